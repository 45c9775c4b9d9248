"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

The FP32 path is compared bit for bit with the oracle's FP32 canonical
mirror: descriptors, every pyramid level (values and argmax codes), the
merged-tuple counts per level, and the final matches.  Against the FP64
oracle the matches must agree except on patches whose decision is nearly
tied (stated tolerance below).
"""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth

pytestmark = pytest.mark.gpu

# FP64 agreement: a patch may differ from the FP64 oracle only where one of the
# decisions behind the oracle's output for it (BestAt, BestAt', a 3x3 argmax on
# its winning path) has a relative top-two gap below this tolerance.
FP64_GAP_TOL = 1e-3


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_1506_07656_gb300 import build, dm
    build.build()
    c = dm.Context(dm.DM_FP32)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_plain(torch_cuda, ctx):
    """FP32 path with plain (uncompensated) child sums."""
    from paper_1506_07656_gb300 import dm
    c = dm.Context(dm.DM_FP32, compensated=0)
    yield c
    c.close()


def _dev(torch, a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def _gpu_descriptors(torch, ctx, img):
    from paper_1506_07656_gb300 import dm
    H, W = img.shape
    d_img = _dev(torch, img)
    out = torch.empty((H, W, 9), dtype=torch.float32, device="cuda")
    tmp = torch.empty(dm.dm_workspace_bytes(ctx.ctx, max(W, 4), max(H, 4), W, H)["desc"], dtype=torch.uint8,
                      device="cuda")
    dm.dm_descriptors(ctx.ctx, d_img, out, tmp)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _gpu_pyramid(torch, ctx, d1, d2):
    from paper_1506_07656_gb300 import dm
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    ws = torch.empty(dm.dm_workspace_bytes(ctx.ctx, W1, H1, W2, H2)["pyramid"], dtype=torch.uint8, device="cuda")
    t1, t2 = _dev(torch, d1), _dev(torch, d2)
    h = dm.dm_correlate_pyramid(ctx.ctx, t1, t2, ws)
    torch.cuda.synchronize()
    g = dm.dm_geometry(W1, H1, W2, H2)
    levels = [dm.read_level(ws, dm.dm_pyramid_level(h, l)) for l in range(g["L"] + 1)]
    return h, ws, levels


def _gpu_backtrack(torch, ctx, h, W1, H1, W2, H2, capacity=None):
    from paper_1506_07656_gb300 import dm
    g = dm.dm_geometry(W1, H1, W2, H2)
    ws = torch.empty(dm.dm_workspace_bytes(ctx.ctx, W1, H1, W2, H2)["backtrack"], dtype=torch.uint8, device="cuda")
    cap = g["n_patch0"] if capacity is None else capacity
    out = torch.zeros((max(cap, 1), 5), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dm.dm_backtrack(ctx.ctx, h, ws, out[:cap] if cap else out[:0], cnt)
    status, reached = dm.dm_read_status(ctx.ctx, ws, g["L"] + 1)
    n = int(cnt.item())
    return out[:min(n, cap)].cpu().numpy().astype(np.float64), n, status, reached


def _compare_pyramids(pyr, levels):
    g = pyr.geom
    for l in range(g.L + 1):
        vals, am, valid = levels[l]
        np.testing.assert_array_equal(valid, pyr.valid[l])
        keep = valid.astype(bool)
        want = pyr.pooled[l] if l < g.L else pyr.top
        np.testing.assert_array_equal(vals[keep], want[keep], err_msg=f"level {l} values")
        if l < g.L:
            np.testing.assert_array_equal(am[keep], pyr.argmax[l][keep], err_msg=f"level {l} argmax")


CASES = [
    # (W1, H1, W2, H2, maker, seed): config-1 pair, ragged sizes, unequal sizes
    (64, 48, 64, 48, "smooth", 1),
    (37, 29, 37, 29, "smooth", 2),
    (41, 23, 53, 35, "smooth", 3),
    (96, 61, 71, 80, "motif", 4),
    (130, 70, 130, 70, "smooth", 5),
]


def _pair(W1, H1, W2, H2, maker, seed):
    if (W1, H1) == (W2, H2):
        pr = synth.make_pair_smooth(W1, H1, seed) if maker == "smooth" else synth.make_pair_motif(W1, H1, seed, 12.0)
        return pr.img1, pr.img2
    rng = np.random.default_rng(seed)
    a = synth.value_noise(W1, H1, rng).astype(np.float32)
    b = synth.value_noise(W2, H2, rng).astype(np.float32)
    return a, b


@pytest.mark.parametrize("case", CASES)
def test_descriptors_bit_exact(torch_cuda, ctx, oracle_mod, case):
    img1, img2 = _pair(*case)
    for img in (img1, img2):
        got = _gpu_descriptors(torch_cuda, ctx, img)
        want = oracle_mod.descriptors(img, "f32")
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("compensated", [True, False])
@pytest.mark.parametrize("case", CASES)
def test_pyramid_and_matches_bit_exact(torch_cuda, ctx, ctx_plain, oracle_mod, case, compensated):
    W1, H1, W2, H2 = case[:4]
    img1, img2 = _pair(*case)
    d1 = oracle_mod.descriptors(img1, "f32")
    d2 = oracle_mod.descriptors(img2, "f32")
    pyr = oracle_mod.pyramid(d1, d2, "f32", compensated=compensated)
    ctx = ctx if compensated else ctx_plain
    h, ws, levels = _gpu_pyramid(torch_cuda, ctx, d1, d2)
    try:
        _compare_pyramids(pyr, levels)
        bt = oracle_mod.backtrack(pyr)
        want = oracle_mod.reciprocal(pyr, bt)
        got, n, status, reached = _gpu_backtrack(torch_cuda, ctx, h, W1, H1, W2, H2)
        assert status == 0
        assert n == len(want)
        np.testing.assert_array_equal(got, want)
        # merged tuples per level (levels 1..L)
        assert reached[1:] == bt.reached[1:].tolist()
    finally:
        from paper_1506_07656_gb300 import dm
        dm.dm_pyramid_free(h)


def test_match_end_to_end_config1(torch_cuda, ctx, oracle_mod):
    """64x48 value-noise pair, smooth warp (max 6 px): images in, matches out."""
    pr = synth.make_pair_smooth(64, 48, seed=1)
    got = ctx.match(pr.img1, pr.img2).cpu().numpy().astype(np.float64)
    want32, _, _ = oracle_mod.match(pr.img1, pr.img2, "f32")
    np.testing.assert_array_equal(got, want32)
    want64, pyr64, bt64 = oracle_mod.match(pr.img1, pr.img2, "f64", gaps=True)
    bad = _disagreeing_patches(got, want64, pyr64.geom)
    excused = [p for p in bad if bt64.gap[p] < FP64_GAP_TOL]
    print(f"FP64 agreement: {1 - len(bad) / pyr64.geom.npatch(0):.4f}, {len(bad)} differing patches, "
          f"{len(excused)} excused by a near tie")
    assert len(excused) == len(bad), [(p, bt64.gap[p]) for p in bad if p not in excused]
    assert synth.accuracy_at(got, pr.flow, 10.0) >= 0.95
    st, reached = ctx.status(64, 48, 64, 48)
    assert st == 0


def _disagreeing_patches(a, b, geom):
    """Atomic patches whose match (or absence of one) differs between two lists."""
    ka = {(int(r[0]), int(r[1])): (r[2], r[3]) for r in a}
    kb = {(int(r[0]), int(r[1])): (r[2], r[3]) for r in b}
    out = []
    for (x1, y1) in set(ka) | set(kb):
        if ka.get((x1, y1)) != kb.get((x1, y1)):
            out.append(((y1 - 2) // 4) * geom.P0x + (x1 - 2) // 4)
    return sorted(out)


def _agreement(a, b):
    """Fraction of atomic patches on which two match lists agree (same match or both none)."""
    ka = {(r[0], r[1]): (r[2], r[3]) for r in a}
    kb = {(r[0], r[1]): (r[2], r[3]) for r in b}
    keys = set(ka) | set(kb)
    if not keys:
        return 1.0
    return sum(ka.get(k) == kb.get(k) for k in keys) / len(keys)


@pytest.mark.slow
def test_match_end_to_end_config2(torch_cuda, ctx, oracle_mod):
    """512x224 pair: noise with a 30% 16x16 repeated motif, 3-bump warp (max 40 px) + similarity."""
    pr = synth.make_pair_motif(512, 224, seed=7)
    got = ctx.match(pr.img1, pr.img2).cpu().numpy().astype(np.float64)
    want32, _, bt = oracle_mod.match(pr.img1, pr.img2, "f32")
    np.testing.assert_array_equal(got, want32)
    st, reached = ctx.status(512, 224, 512, 224)
    assert st == 0
    assert reached[1:] == bt.reached[1:].tolist()


def test_match_host_equals_device(torch_cuda, ctx):
    from paper_1506_07656_gb300 import dm
    pr = synth.make_pair_smooth(64, 48, seed=3)
    dev = ctx.match(pr.img1, pr.img2).cpu().numpy()
    torch = torch_cuda
    h1 = torch.from_numpy(pr.img1).pin_memory()
    h2 = torch.from_numpy(pr.img2).pin_memory()
    ws = ctx.workspace("match", 64, 48, 64, 48)
    out = torch.zeros((192, 5), dtype=torch.float32).pin_memory()
    n = dm.dm_match_host(ctx.ctx, h1, h2, ws, out)
    np.testing.assert_array_equal(out[:n].numpy(), dev)


def test_output_capacity_overflow(torch_cuda, ctx, oracle_mod):
    from paper_1506_07656_gb300 import dm
    pr = synth.make_pair_smooth(64, 48, seed=1)
    d1 = oracle_mod.descriptors(pr.img1, "f32")
    d2 = oracle_mod.descriptors(pr.img2, "f32")
    want = oracle_mod.reciprocal(*(lambda p: (p, oracle_mod.backtrack(p)))(oracle_mod.pyramid(d1, d2, "f32")))
    h, ws, _ = _gpu_pyramid(torch_cuda, ctx, d1, d2)
    try:
        got, n, status, _ = _gpu_backtrack(torch_cuda, ctx, h, 64, 48, 64, 48, capacity=10)
        assert n == len(want)                     # the true count is reported
        assert status & dm.DM_DEV_OUTPUT_OVERFLOW
        np.testing.assert_array_equal(got, want[:10])
    finally:
        dm.dm_pyramid_free(h)


def test_argument_errors(torch_cuda, ctx):
    from paper_1506_07656_gb300 import dm
    torch = torch_cuda
    img = torch.zeros((3, 3), device="cuda")
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    out = torch.empty((4, 5), device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_match(ctx.ctx, img, img, ws, out, cnt)
    assert e.value.status == dm.DM_EINVAL
    img = torch.zeros((48, 64), device="cuda")
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_match(ctx.ctx, img, img, small, out, cnt)
    assert e.value.status == dm.DM_ENOMEM
    with pytest.raises(dm.DmError) as e:
        dm.dm_match(ctx.ctx, img, img, ws[1:], out, cnt)      # misaligned workspace
    assert e.value.status == dm.DM_EINVAL


def test_identity_and_translation_on_gpu(torch_cuda, ctx):
    """Identity warp: every atomic patch matches itself with score L + 1."""
    pr = synth.make_pair_smooth(64, 48, seed=9)
    got = ctx.match(pr.img1, pr.img1).cpu().numpy()
    assert len(got) == 16 * 12
    np.testing.assert_array_equal(got[:, 0], got[:, 2])
    np.testing.assert_array_equal(got[:, 1], got[:, 3])
    assert np.abs(got[:, 4] - 5.0).max() < 1e-5


@pytest.mark.parametrize("dims,seed", [((64, 48, 64, 48), 11), ((41, 23, 53, 35), 12), ((130, 70, 130, 70), 13)])
def test_tie_heavy_fields_bit_exact(torch_cuda, ctx, oracle_mod, dims, seed):
    """Descriptor fields whose entries take three values (0, 1/4, 1/2): the
    correlations are exact small dyadic sums, so the 3x3 maxima of every level
    tie often and the first-maximum rule in scan order (and the backtracking's
    tie rules) decide; the pyramid (values and argmax codes), the merged-tuple
    counts and the matches must still equal the FP32 oracle bit for bit."""
    W1, H1, W2, H2 = dims
    rng = np.random.default_rng(seed)
    d1 = (rng.integers(0, 3, size=(H1, W1, 9)) * 0.25).astype(np.float32)
    d2 = (rng.integers(0, 3, size=(H2, W2, 9)) * 0.25).astype(np.float32)
    pyr = oracle_mod.pyramid(d1, d2, "f32")
    ties = sum(int(np.sum(pyr.pooled[l] == np.roll(pyr.pooled[l], 1, axis=2))) for l in range(pyr.geom.L))
    assert ties > 0
    h, ws, levels = _gpu_pyramid(torch_cuda, ctx, d1, d2)
    try:
        _compare_pyramids(pyr, levels)
        bt = oracle_mod.backtrack(pyr)
        want = oracle_mod.reciprocal(pyr, bt)
        got, n, status, reached = _gpu_backtrack(torch_cuda, ctx, h, W1, H1, W2, H2)
        assert status == 0
        assert n == len(want)
        np.testing.assert_array_equal(got, want)
        assert reached[1:] == bt.reached[1:].tolist()
    finally:
        from paper_1506_07656_gb300 import dm
        dm.dm_pyramid_free(h)

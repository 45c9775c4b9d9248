"""The GPU path against the oracle at the workload sizes.

* Config 2 (512x224 motif pair): the FP32 path's matches agree with the FP64
  oracle's except on patches whose decision is nearly tied (gap < 1e-3).
* Config 3 at 512x224 (the config-1 recipe at half the 1024x436 size, max
  displacement 60 px): the FP32, BF16 and FP8-E4M3 pyramids against the FP64
  oracle's, level by level, and their matches against the FP64 oracle's, with
  tolerances derived from the precision (below).
* The batch sizes 1242x375 (L = 9, W = 2 mod 4, odd H) and 640x480 (L = 8):
  patch existence at every level against the oracle's, sampled patches of
  levels 0..3 bit-exact in FP32 in the tuned launch shapes, and the batch's
  matches equal to the single-pair call's.
* The extensions at bench-like sizes: DM* on a 256x192 pair, the invariant
  form on a 128x96 image against its quarter turn, both bit-exact in FP32.

Derived tolerances (config 3).  Both sides start from the same descriptors
(the FP32 oracle's, which the GPU reproduces bit for bit), so the comparison
isolates the pyramid's arithmetic; the per-level map error bounds and the
decision tolerances follow from the operand rounding of each precision
(precision_bounds.py).  For FP32 the spec rule (gap < 1e-3) is asserted
on top; the share of patches that rule does not excuse is printed for BF16
and FP8.
"""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth
from precision_bounds import argmax_tol, eps_level, match_tol

pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    return torch, dm


def _prec_id(dm, prec):
    return {"fp32": dm.DM_FP32, "bf16": dm.DM_BF16, "fp8": dm.DM_FP8_E4M3}[prec]


def _gpu_match_and_levels(torch, dm, ctx, img1, img2, levels=None, samples=None, descs=None):
    """Images (or given descriptor fields) -> pyramid -> backtracking on the GPU;
    returns the matches, the status and, per level, (values, codes, valid) of
    all patches (levels=None: every level) or of the sampled patches {level:
    indices}, with the existence flags of every level under "valid"."""
    H1, W1 = img1.shape
    H2, W2 = img2.shape
    sizes = dm.dm_workspace_bytes(ctx.ctx, W1, H1, W2, H2)
    if descs is None:
        tmp = torch.empty(sizes["desc"], dtype=torch.uint8, device="cuda")
        d = []
        for img in (img1, img2):
            H, W = img.shape
            t = torch.empty((H, W, 9), dtype=torch.float32, device="cuda")
            dm.dm_descriptors(ctx.ctx, torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda(), t, tmp)
            d.append(t)
    else:
        d = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda() for x in descs]
    ws = torch.empty(sizes["pyramid"], dtype=torch.uint8, device="cuda")
    h = dm.dm_correlate_pyramid(ctx.ctx, d[0], d[1], ws)
    try:
        g = dm.dm_geometry(W1, H1, W2, H2)
        out = {"valid": {}}
        for l in range(g["L"] + 1):
            info = dm.dm_pyramid_level(h, l)
            out["valid"][l] = _valid(ws, info)
            if samples is not None:
                if l in samples:
                    out[l] = dm.read_level(ws, info, samples[l])
            elif levels is None or l in levels:
                out[l] = dm.read_level(ws, info)
        bws = torch.empty(sizes["backtrack"], dtype=torch.uint8, device="cuda")
        m = torch.zeros((g["n_patch0"], 5), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        dm.dm_backtrack(ctx.ctx, h, bws, m, cnt)
        st, _ = dm.dm_read_status(ctx.ctx, bws, 1)
        n = int(cnt.item())
        return m[:n].cpu().numpy().astype(np.float64), st, out
    finally:
        dm.dm_pyramid_free(h)
        del ws
        torch.cuda.empty_cache()


def _valid(ws, info):
    base = ws.data_ptr()
    o = info["valid"] - base
    return ws[o:o + info["n"]].cpu().numpy()


def _differing_patches(a, b, P0x):
    ka = {(int(r[0]), int(r[1])): (r[2], r[3]) for r in a}
    kb = {(int(r[0]), int(r[1])): (r[2], r[3]) for r in b}
    return sorted(((y - 2) // 4) * P0x + (x - 2) // 4 for (x, y) in set(ka) | set(kb) if ka.get((x, y)) != kb.get((x, y)))


# --------------------------------------------------------------------------- #
# Config 2: FP32 against FP64 at 512x224                                      #
# --------------------------------------------------------------------------- #
def test_config2_fp32_agrees_with_fp64_up_to_near_ties(env, oracle_mod):
    torch, dm = env
    pr = synth.make_pair_motif(512, 224, seed=7)
    ctx = dm.Context(dm.DM_FP32)
    try:
        got = ctx.match(pr.img1, pr.img2).cpu().numpy().astype(np.float64)
        st, _ = ctx.status(512, 224, 512, 224)
    finally:
        ctx.close()
    assert st == 0
    want, pyr, bt = oracle_mod.match(pr.img1, pr.img2, "f64", gaps=True)
    g = pyr.geom
    bad = _differing_patches(got, want, g.P0x)
    unexcused = [p for p in bad if bt.gap[p] >= 1e-3]
    print(f"config 2 FP32 vs FP64: agreement {1 - len(bad) / g.npatch(0):.5f}, {len(bad)} differing patches, "
          f"{len(unexcused)} not excused by a near tie")
    assert not unexcused, [(p, bt.gap[p]) for p in unexcused]


# --------------------------------------------------------------------------- #
# Config 3 at 512x224: FP32 / BF16 / FP8 against the FP64 oracle              #
# --------------------------------------------------------------------------- #
@pytest.fixture(scope="module")
def config3(oracle_mod):
    pr = synth.make_pair_smooth(512, 224, seed=3000, max_disp=60.0)
    d1 = oracle_mod.descriptors(pr.img1, "f32")
    d2 = oracle_mod.descriptors(pr.img2, "f32")
    pyr = oracle_mod.pyramid(d1.astype(np.float64), d2.astype(np.float64), "f64", gaps=True)
    bt = oracle_mod.backtrack(pyr)                      # with the per-patch decision gaps
    want = oracle_mod.reciprocal(pyr, bt)
    return pr, (d1, d2), pyr, bt, want


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp8"])
def test_config3_levels_and_matches_vs_fp64(env, config3, prec):
    torch, dm = env
    pr, descs, pyr, bt, want = config3
    g = pyr.geom
    ctx = dm.Context(_prec_id(dm, prec))
    try:
        got, st, lv = _gpu_match_and_levels(torch, dm, ctx, pr.img1, pr.img2, descs=descs)
    finally:
        ctx.close()
    assert st == 0
    for l in range(g.L + 1):
        vals, codes, valid = lv[l]
        np.testing.assert_array_equal(valid, pyr.valid[l])
        keep = valid.astype(bool)
        ref = pyr.pooled[l] if l < g.L else pyr.top
        x, y = ref[keep], vals[keep].astype(np.float64)
        pos = x > 0
        rel = np.abs(y[pos] - x[pos]) / x[pos]
        eps = eps_level(prec, l)
        line = f"{prec} level {l}: max rel err {rel.max():.3e} mean {rel.mean():.3e} (bound {eps:.3e})"
        assert np.all(y[~pos] == 0.0)                      # zero exactly where every child is out of domain
        assert rel.max() <= eps, line
        if l < g.L:
            diff = codes[keep] != pyr.argmax[l][keep]
            gaps = pyr.gap[l][keep][diff]
            tol = argmax_tol(prec, l)
            line += f"; argmax differs at {int(diff.sum())} of {diff.size} (all with FP64 gap < {tol:.2e})"
            assert np.all(gaps < tol), (l, gaps.max() if gaps.size else None)
        print(line)
    bad = _differing_patches(got, want, g.P0x)
    tol = match_tol(prec, g.L)
    unexcused = [p for p in bad if bt.gap[p] >= tol]
    strict = [p for p in bad if bt.gap[p] >= 1e-3]
    agree = 1 - len(bad) / g.npatch(0)
    floor = 1 - np.count_nonzero(bt.gap < tol) / g.npatch(0)
    print(f"{prec} matches vs FP64: agreement {agree:.4f} (derived floor {floor:.4f}), {len(bad)} differing, "
          f"{len(strict)} not excused by the 1e-3 rule ({len(strict) / g.npatch(0):.4f} of the patches), "
          f"{len(unexcused)} not excused by the {tol:.2e} rule")
    assert not unexcused
    assert agree >= floor
    if prec == "fp32":
        assert not strict


# --------------------------------------------------------------------------- #
# The batch sizes: 1242x375 (L = 9) and 640x480 (L = 8)                        #
# --------------------------------------------------------------------------- #
BATCH_SIZES = [(1242, 375, 4100), (640, 480, 4200)]


def _batch_pair(W, H, seed):
    return synth.make_pair_smooth(W, H, seed=seed, max_disp=120.0, with_flow=False)


@pytest.mark.parametrize("W,H,seed", BATCH_SIZES)
def test_batch_size_sampled_levels_bit_exact(env, oracle_mod, W, H, seed):
    torch, dm = env
    pr = _batch_pair(W, H, seed)
    g = dm.dm_geometry(W, H, W, H)
    rng = np.random.default_rng(seed)
    samples = {0: np.sort(rng.choice(g["n_patch0"], 4, replace=False))}
    for l, k in ((1, 3), (2, 2), (3, 2)):
        samples[l] = np.sort(rng.choice(g["n_patch"], k, replace=False))
    ctx = dm.Context(dm.DM_FP32)
    try:
        ctx.autotune(pr.img1, pr.img2)                 # the launch shapes the batch runs for this size
        m, st, lv = _gpu_match_and_levels(torch, dm, ctx, pr.img1, pr.img2, samples=samples)
    finally:
        ctx.close()
    assert st == 0
    vf = oracle_mod.valid_flags(W, H, W, H)
    for l in range(g["L"] + 1):
        np.testing.assert_array_equal(lv["valid"][l], vf[l], err_msg=f"existence, level {l}")
    d1 = oracle_mod.descriptors(pr.img1, "f32")
    d2 = oracle_mod.descriptors(pr.img2, "f32")
    for l, sel in samples.items():
        v, a, e = oracle_mod.levels_sampled(d1, d2, l, sel, "f32")
        vals, codes, valid = lv[l]
        np.testing.assert_array_equal(valid, e)
        keep = e.astype(bool)
        np.testing.assert_array_equal(vals[keep], v[keep], err_msg=f"level {l} values")
        np.testing.assert_array_equal(codes[keep], a[keep], err_msg=f"level {l} codes")
    # well-formed matches
    assert len(m) > 0.3 * g["n_patch0"]
    assert len({(int(r[0]), int(r[1])) for r in m}) == len(m)
    assert np.all((m[:, 2] >= 0) & (m[:, 2] < W) & (m[:, 3] >= 0) & (m[:, 3] < H))
    assert np.all((m[:, 4] > 0) & (m[:, 4] <= g["L"] + 1 + 1e-5))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_of_the_large_sizes_equals_single_pairs(env, prec):
    torch, dm = env
    ctx = dm.Context(_prec_id(dm, prec))
    try:
        items, prs = [], []
        for W, H, seed in BATCH_SIZES:
            pr = _batch_pair(W, H, seed)
            ctx.autotune(pr.img1, pr.img2)
            n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
            items.append((torch.from_numpy(pr.img1).cuda(), torch.from_numpy(pr.img2).cuda(),
                          torch.zeros((n0, 5), dtype=torch.float32, device="cuda"),
                          torch.zeros(1, dtype=torch.int32, device="cuda")))
            prs.append(pr)
        pairs = dm.make_pairs(items)
        ws = torch.empty(dm.dm_batch_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
        dm.dm_match_batch(ctx.ctx, pairs, ws)
        torch.cuda.synchronize()
        got = [it[2][:int(it[3].item())].cpu().numpy() for it in items]
        del ws
        torch.cuda.empty_cache()
        for gm, pr in zip(got, prs):
            np.testing.assert_array_equal(gm, ctx.match(pr.img1, pr.img2).cpu().numpy())
    finally:
        ctx.close()
        torch.cuda.empty_cache()


# --------------------------------------------------------------------------- #
# Extensions at bench-like sizes                                              #
# --------------------------------------------------------------------------- #
def test_dmstar_256x192_bit_exact(env, oracle_mod):
    torch, dm = env
    pr = synth.make_pair_smooth(256, 192, seed=31)
    img1, img2 = pr.img1.astype(np.float32), pr.img2.astype(np.float32)
    want = oracle_mod.dmstar_match(img1, img2, "f32")
    ctx = dm.Context(dm.DM_FP32)
    try:
        got = ctx.match_star(img1, img2).cpu().numpy().astype(np.float64)
    finally:
        ctx.close()
    assert len(want) > 0
    np.testing.assert_array_equal(got, want.astype(np.float32).astype(np.float64))


def test_invariant_128x96_quarter_turn_bit_exact(env, oracle_mod):
    torch, dm = env
    img1 = synth.make_pair_smooth(128, 96, seed=9, max_disp=1.0).img1.astype(np.float32)
    img2 = np.ascontiguousarray(np.rot90(img1, 1))
    want = oracle_mod.invariant_match(img1, img2, "f32")
    ctx = dm.Context(dm.DM_FP32)
    try:
        got = ctx.match_invariant(img1, img2).cpu().numpy().astype(np.float64)
    finally:
        ctx.close()
    assert len(want) > 0
    np.testing.assert_array_equal(got, want.astype(np.float32).astype(np.float64))
    # the quarter turn is recovered: (x2, y2) = (y1, W1 - 1 - x1) within 3 px
    ok = (np.abs(got[:, 2] - got[:, 1]) <= 3) & (np.abs(got[:, 3] - (127 - got[:, 0])) <= 3)
    assert ok.mean() >= 0.9

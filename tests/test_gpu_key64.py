"""64-bit merge keys of the backtracking (Sec. 3.3 "Merging correspondences":
tuples equal in (level, patch, position) are merged keeping the highest score).

The key of a tuple of level l is patch * |domain of l| + position.  Where every
level's keys fit 32 bits the tables hold 8-byte slots; larger pairs (and the
rotated canvases of the invariant form) take 64-bit keys in 16-byte slots.
dm_set_merge_keys(64) forces the wide form at any size, so it is checked

* bit for bit against the FP32 oracle on small pairs (matches and merged-tuple
  counts per level), in both child-sum modes and in the invariant form;
* against the 32-bit form at the bench's 1024 x 436 (identical matches and
  counts);

and where 64 bits are needed it runs: the invariant form at 1024 x 436,
whose 45-degree canvas (1032 x 1032 against 1024 x 436) has 7.4e9 keys at
level 1 and was refused with 32-bit keys, recovers a quarter turn.
"""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build
    build.build()
    return torch


def _ctx(prec="fp32", bits=64, **kw):
    from paper_1506_07656_gb300 import dm
    c = dm.Context({"fp32": dm.DM_FP32, "bf16": dm.DM_BF16}[prec], **kw)
    c.set_merge_keys(bits)
    return c


def _match_with_counts(torch, ctx, img1, img2):
    from paper_1506_07656_gb300 import dm
    H1, W1 = img1.shape
    H2, W2 = img2.shape
    got = ctx.match(img1, img2).cpu().numpy().astype(np.float64)
    g = dm.dm_geometry(W1, H1, W2, H2)
    status, reached = dm.dm_read_status(ctx.ctx, ctx.workspace("match", W1, H1, W2, H2), g["L"] + 1)
    return got, status, reached


CASES = [(64, 48, 64, 48, 1), (37, 29, 37, 29, 2), (130, 70, 130, 70, 5)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("comp", [1, 0])
def test_forced_64bit_keys_equal_the_oracle(torch_cuda, oracle_mod, case, comp):
    W1, H1, W2, H2, seed = case
    pr = synth.make_pair_smooth(W1, H1, seed)
    want, _, bt = oracle_mod.match(pr.img1, pr.img2, "f32", compensated=comp)
    ctx = _ctx("fp32", 64, compensated=comp)
    try:
        got, status, reached = _match_with_counts(torch_cuda, ctx, pr.img1, pr.img2)
    finally:
        ctx.close()
    assert status == 0
    np.testing.assert_array_equal(got, want)
    assert reached[1:] == bt.reached[1:].tolist()


def test_forced_64bit_keys_unequal_sizes(torch_cuda, oracle_mod):
    rng = np.random.default_rng(3)
    a = synth.value_noise(41, 23, rng).astype(np.float32)
    b = synth.value_noise(53, 35, rng).astype(np.float32)
    want, _, bt = oracle_mod.match(a, b, "f32")
    ctx = _ctx("fp32", 64)
    try:
        got, status, reached = _match_with_counts(torch_cuda, ctx, a, b)
    finally:
        ctx.close()
    assert status == 0
    np.testing.assert_array_equal(got, want)
    assert reached[1:] == bt.reached[1:].tolist()


def test_forced_64bit_keys_in_the_invariant_form(torch_cuda, oracle_mod):
    img1 = synth.make_pair_smooth(48, 40, seed=9, max_disp=1.0).img1
    img2 = np.ascontiguousarray(np.rot90(img1, 1))
    want = oracle_mod.invariant_match(img1.astype(np.float32), img2.astype(np.float32), "f32")
    ctx = _ctx("fp32", 64)
    try:
        got = ctx.match_invariant(img1, img2).cpu().numpy().astype(np.float64)
    finally:
        ctx.close()
    assert len(want) > 0
    np.testing.assert_array_equal(got, want)


def test_64bit_keys_equal_32bit_keys_at_1024x436(torch_cuda):
    pr = synth.make_pair_smooth(1024, 436, seed=1000, max_disp=120.0, with_flow=False)
    runs = {}
    for bits in (0, 64):
        ctx = _ctx("bf16", bits)
        try:
            runs[bits] = _match_with_counts(torch_cuda, ctx, pr.img1, pr.img2)
        finally:
            ctx.close()
    (a, sa, ra), (b, sb, rb) = runs[0], runs[64]
    assert sa == 0 and sb == 0
    assert len(a) > 10000
    np.testing.assert_array_equal(a, b)
    assert ra == rb


def test_star_refuses_64bit_keys(torch_cuda):
    from paper_1506_07656_gb300 import dm
    ctx = _ctx("fp32", 64)
    try:
        with pytest.raises(dm.DmError) as e:
            dm.dm_star_workspace_bytes(ctx.ctx, 64, 48, 64, 48)
        assert e.value.status == dm.DM_EUNSUPPORTED
        ctx.set_merge_keys(0)
        dm.dm_star_workspace_bytes(ctx.ctx, 64, 48, 64, 48)
        with pytest.raises(dm.DmError) as e:
            ctx.set_merge_keys(32)
        assert e.value.status == dm.DM_EINVAL
    finally:
        ctx.close()


def test_invariant_form_at_1024x436_recovers_a_quarter_turn(torch_cuda):
    """Image 2 is image 1 turned by 90 degrees (436 x 1024): the 45-degree
    canvases need 64-bit keys.  The matches are consistent with the turn
    (x2 = y1, y2 = W1 - 1 - x1 within 3 px) on most patches, like the small
    quarter-turn pairs that are checked bit for bit."""
    from paper_1506_07656_gb300 import dm
    img1 = synth.make_pair_smooth(1024, 436, seed=21, max_disp=1.0, with_flow=False).img1
    img2 = np.ascontiguousarray(np.rot90(img1, 1))
    ctx = _ctx("bf16", 0)
    try:
        dm.dm_set_batch_lanes(ctx.ctx, 1)
        got = ctx.match_invariant(img1, img2).cpu().numpy().astype(np.float64)
        ws = ctx._ws[("invariant", 1024, 436, 436, 1024)]
        status, _ = dm.dm_read_status(ctx.ctx, ws, 1)
    finally:
        ctx.close()
    assert status == 0
    n0 = dm.dm_geometry(1024, 436, 436, 1024)["n_patch0"]
    consistent = np.mean((np.abs(got[:, 2] - got[:, 1]) <= 3.0) & (np.abs(got[:, 3] - (1023 - got[:, 0])) <= 3.0))
    print(f"invariant 1024x436 quarter turn: {len(got)} matches of {n0} patches, {consistent:.3f} consistent")
    assert len(got) >= 0.2 * n0
    assert consistent >= 0.7

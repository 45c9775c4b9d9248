"""Parity at the bench's full size: one 1024x436 pair (the bench recipe: value
noise, smooth warp up to 120 px), matched in the launch configuration the
bench times.  The oracle cannot produce the whole pyramid of such a pair in
seconds, so sampled outputs are checked one by one and the rest by properties
that hold at any size.

FP32 path: the pooled maps and argmax codes of sampled patches of levels 0
to 3 are bit-exact with the FP32 oracle (which builds a level-l map from the
4^l atomic descendants of the patch); the existence of every patch at every
level, including the top-level patches that drop out for lack of a child
(reading c8), equals the oracle's; every stored level value lies in
[0, 1]; the matches are well formed (at most one per atomic patch, centres on
the atomic grid, targets inside I', scores in (0, L+1]).  BF16 path: the same
sampled level-0 maps are within the BF16 error bound of the FP32 oracle
(derived from the operand rounding, precision_bounds.py); its argmax and
match agreement with the FP32 path are printed."""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth
from precision_bounds import eps_level

pytestmark = pytest.mark.gpu

W, H = 1024, 436


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    pr = synth.make_pair_smooth(W, H, seed=1000, max_disp=120.0, with_flow=False)
    d1 = oracle_mod.descriptors(pr.img1, "f32")
    d2 = oracle_mod.descriptors(pr.img2, "f32")
    return torch, dm, pr, d1, d2


def _run(torch, dm, precision, d1, d2, samples, pr):
    ctx = dm.Context(precision)
    vmax = 1.0 + (1e-6 if precision == dm.DM_FP32 else 2e-2)   # BF16/FP8 operands can push C0 a little past 1
    try:
        ctx.autotune(pr.img1, pr.img2)                           # the launch shapes the bench times
        t1 = torch.as_tensor(d1, device="cuda")
        t2 = torch.as_tensor(d2, device="cuda")
        sizes = dm.dm_workspace_bytes(ctx.ctx, W, H, W, H)
        ws = torch.empty(sizes["pyramid"], dtype=torch.uint8, device="cuda")
        h = dm.dm_correlate_pyramid(ctx.ctx, t1, t2, ws)
        torch.cuda.synchronize()
        g = dm.dm_geometry(W, H, W, H)
        lv = {l: dm.read_level(ws, dm.dm_pyramid_level(h, l), sel) for l, sel in samples.items()}
        valid = []
        # every stored level value in [0, 1] (all rows of every level, on the device)
        for l in range(g["L"] + 1):
            info = dm.dm_pyramid_level(h, l)
            base = ws.data_ptr()
            n, mh, pitch = info["n"], info["mh"], info["pitch"]
            v = ws[info["vals"] - base:info["vals"] - base + n * mh * pitch * 4].view(torch.float32)
            assert float(v.min()) >= 0.0 and float(v.max()) <= vmax, l
            valid.append(ws[info["valid"] - base:info["valid"] - base + n].cpu().numpy())
        wsb = torch.empty(sizes["backtrack"], dtype=torch.uint8, device="cuda")
        out = torch.zeros((g["n_patch0"], 5), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        dm.dm_backtrack(ctx.ctx, h, wsb, out, cnt)
        st, _ = dm.dm_read_status(ctx.ctx, wsb, 1)
        n = int(cnt.item())
        dm.dm_pyramid_free(h)
        return lv, valid, out[:n].cpu().numpy().astype(np.float64), st, g
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def _samples(g):
    """Sampled patches per level: 12 atomic patches, 5 of level 1, and two each
    of levels 2 and 3 (16 and 64 atomic descendants), one of them at the right
    border of the lattice."""
    rng = np.random.default_rng(3)
    s = {0: np.sort(rng.choice(g["n_patch0"], size=12, replace=False)),
         1: np.sort(rng.choice(g["n_patch"], size=5, replace=False))}
    Lx = (W - 1) // 4 + 1
    s[2] = np.sort(np.append(rng.choice(g["n_patch"], size=1), 37 * Lx + Lx - 1))
    s[3] = np.sort(rng.choice(g["n_patch"], size=2, replace=False))
    return s


def _check_matches(m, g):
    assert len(m) > 0.3 * g["n_patch0"]
    keys = {(int(r[0]), int(r[1])) for r in m}
    assert len(keys) == len(m)                                  # at most one match per atomic patch
    assert np.all((m[:, 0] - 2) % 4 == 0) and np.all((m[:, 1] - 2) % 4 == 0)
    assert np.all((m[:, 2] >= 0) & (m[:, 2] < W) & (m[:, 3] >= 0) & (m[:, 3] < H))
    assert np.all((m[:, 4] > 0) & (m[:, 4] <= g["L"] + 1 + 1e-5))


def test_fp32_full_size_sampled_bit_exact(env, oracle_mod):
    torch, dm, pr, d1, d2 = env
    g = dm.dm_geometry(W, H, W, H)
    samples = _samples(g)
    lv, valid, m, st, _ = _run(torch, dm, dm.DM_FP32, d1, d2, samples, pr)
    vf = oracle_mod.valid_flags(W, H, W, H)
    for l in range(g["L"] + 1):
        np.testing.assert_array_equal(valid[l], vf[l], err_msg=f"existence, level {l}")
    assert not vf[g["L"]].all()                                 # some top-level patches drop out (c8)
    for l, sel in samples.items():
        want, codes, ex = oracle_mod.levels_sampled(d1, d2, l, sel, "f32")
        v, a, e = lv[l]
        np.testing.assert_array_equal(e, ex)
        keep = ex.astype(bool)
        np.testing.assert_array_equal(v[keep], want[keep], err_msg=f"level {l} values")
        np.testing.assert_array_equal(a[keep], codes[keep], err_msg=f"level {l} codes")
    assert st == 0
    _check_matches(m, g)


def test_bf16_full_size_sampled_within_tolerance(env, oracle_mod):
    torch, dm, pr, d1, d2 = env
    g = dm.dm_geometry(W, H, W, H)
    s = _samples(g)
    lv, _, m16, st, _ = _run(torch, dm, dm.DM_BF16, d1, d2, {0: s[0]}, pr)
    v0, a0, _ = lv[0]
    w0, b0 = oracle_mod.level0_pooled(d1, d2, s[0], "f32")
    rel = np.abs(v0 - w0) / np.maximum(np.abs(w0), 1e-30)
    # the BF16 bound of the level-0 maps plus the FP32 oracle's own (precision_bounds.py)
    assert rel.max() <= eps_level("bf16", 0) + eps_level("fp32", 0), rel.max()
    assert st == 0
    _check_matches(m16, g)
    _, _, m32, _, _ = _run(torch, dm, dm.DM_FP32, d1, d2, {0: s[0][:1]}, pr)
    k32 = {(r[0], r[1]): (r[2], r[3]) for r in m32}
    k16 = {(r[0], r[1]): (r[2], r[3]) for r in m16}
    keys = set(k32) | set(k16)
    print(f"1024x436 BF16: level-0 max rel err {rel.max():.3e}, argmax agreement {np.mean(a0 == b0):.4f}, "
          f"match agreement with FP32 {sum(k32.get(k) == k16.get(k) for k in keys) / len(keys):.4f}")

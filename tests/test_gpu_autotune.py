"""Autotuner of the batched form: every launch-shape candidate computes the
same results, and the tuner only ever picks among the candidates.

FP32: the matches and every pyramid level under each forced shape are bit-exact
with the FP32 oracle.  BF16: each forced shape gives bit-identical output to
the default shape (the tensor-core arithmetic of a tile does not depend on
which CTA computes it)."""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [
    {"m_chunk": 1, "level_tile_rows": 8, "bt_ctas_per_sm": 2, "level_ring": 3},
    {"m_chunk": 3, "level_tile_rows": 16, "bt_ctas_per_sm": 32, "level_ring": 2},
    {"m_chunk": 1000, "level_tile_rows": 8, "bt_ctas_per_sm": 1, "level_ring": 2},
    {"m_chunk": 2, "level_tile_rows": 0, "bt_ctas_per_sm": 8, "level_ring": 2},      # row-streaming level kernel
    {"m_chunk": 2, "level_tile_rows": 4, "bt_ctas_per_sm": 8, "level_ring": 2},      # 4-row tiles on 2 warps
    {"m_chunk": 1, "level_tile_rows": 4, "bt_ctas_per_sm": 4, "level_ring": 3},
]


@pytest.fixture(scope="module")
def dm_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    return dm


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("W,H,seed", [(130, 70, 1), (97, 61, 2)])
def test_forced_shapes_fp32_bit_exact(dm_mod, oracle_mod, shape, W, H, seed):
    dm = dm_mod
    pr = synth.make_pair_smooth(W, H, seed)
    want, pyr, _ = oracle_mod.match(pr.img1, pr.img2, "f32")
    ctx = dm.Context(dm.DM_FP32)
    try:
        dm.dm_set_tuned_config(ctx.ctx, W, H, W, H, shape)
        assert dm.dm_tuned_config(ctx.ctx, W, H, W, H) == shape
        got = ctx.match(pr.img1, pr.img2).cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(got, want)
        st, reached = ctx.status(W, H, W, H)
        assert st == 0
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_forced_shapes_tensorcore_identical(dm_mod, prec):
    dm = dm_mod
    W, H = 256, 160
    pr = synth.make_pair_smooth(W, H, 3, max_disp=20.0)
    code = dm.DM_BF16 if prec == "bf16" else dm.DM_FP8_E4M3
    ctx = dm.Context(code)
    try:
        ref = ctx.match(pr.img1, pr.img2).cpu().numpy()
        for shape in SHAPES:
            dm.dm_set_tuned_config(ctx.ctx, W, H, W, H, shape)
            got = ctx.match(pr.img1, pr.img2).cpu().numpy()
            np.testing.assert_array_equal(got, ref)
    finally:
        ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_autotune_picks_a_candidate_and_keeps_results(dm_mod, prec):
    dm = dm_mod
    W, H = 320, 240
    pr = synth.make_pair_smooth(W, H, 4, max_disp=20.0)
    ctx = dm.Context(dm.DM_FP32 if prec == "fp32" else dm.DM_BF16)
    try:
        n_mtiles = -(-dm.dm_geometry(W, H, W, H)["n_patch0"] // 128)
        assert dm.dm_tuned_config(ctx.ctx, W, H, W, H) == {"m_chunk": n_mtiles, "level_tile_rows": 8,
                                                            "bt_ctas_per_sm": 8, "level_ring": 2}
        before = ctx.match(pr.img1, pr.img2).cpu().numpy()
        chosen = ctx.autotune(pr.img1, pr.img2)
        assert chosen["m_chunk"] in {-(-n_mtiles // k) for k in (1, 2, 3, 4, 6, 8)}
        assert chosen["level_tile_rows"] in (0, 4, 8, 16)
        assert chosen["bt_ctas_per_sm"] in (2, 4, 8, 16, 32)
        assert chosen["level_ring"] in (2, 3)
        assert dm.dm_tuned_config(ctx.ctx, W, H, W, H) == chosen
        after = ctx.match(pr.img1, pr.img2).cpu().numpy()
        np.testing.assert_array_equal(after, before)
    finally:
        ctx.close()


def test_set_tuned_config_rejects_bad_shapes(dm_mod):
    dm = dm_mod
    ctx = dm.Context(dm.DM_FP32)
    try:
        for bad in ({"m_chunk": 0, "level_tile_rows": 16, "bt_ctas_per_sm": 8, "level_ring": 2},
                    {"m_chunk": 4, "level_tile_rows": 12, "bt_ctas_per_sm": 8, "level_ring": 2},
                    {"m_chunk": 4, "level_tile_rows": 16, "bt_ctas_per_sm": 65, "level_ring": 3},
                    {"m_chunk": 4, "level_tile_rows": 16, "bt_ctas_per_sm": 8, "level_ring": 4}):
            with pytest.raises(dm.DmError):
                dm.dm_set_tuned_config(ctx.ctx, 64, 48, 64, 48, bad)
    finally:
        ctx.close()


STREAM = {"m_chunk": 1, "level_tile_rows": 0, "bt_ctas_per_sm": 8, "level_ring": 2}


@pytest.mark.parametrize("compensated", [True, False])
@pytest.mark.parametrize("W1,H1,W2,H2,seed", [(64, 48, 64, 48, 1), (37, 29, 37, 29, 2), (41, 23, 53, 35, 3),
                                              (96, 61, 71, 80, 4), (130, 70, 130, 70, 5), (300, 90, 257, 131, 6)])
def test_row_streaming_level_kernel_bit_exact(dm_mod, oracle_mod, W1, H1, W2, H2, seed, compensated):
    """The row-streaming level kernel: every level (values, argmax codes,
    existence) bit-exact with the FP32 oracle, in both child-sum modes, on
    equal, ragged and unequal sizes (strips that end inside the map, patches
    with fewer than four children, odd map sizes)."""
    import torch
    dm = dm_mod
    rng = np.random.default_rng(seed)
    a = synth.value_noise(W1, H1, rng).astype(np.float32)
    b = synth.value_noise(W2, H2, rng).astype(np.float32)
    d1 = oracle_mod.descriptors(a, "f32")
    d2 = oracle_mod.descriptors(b, "f32")
    pyr = oracle_mod.pyramid(d1, d2, "f32", compensated=compensated)
    ctx = dm.Context(dm.DM_FP32, compensated=int(compensated))
    try:
        dm.dm_set_tuned_config(ctx.ctx, W1, H1, W2, H2, STREAM)
        ws = torch.empty(dm.dm_workspace_bytes(ctx.ctx, W1, H1, W2, H2)["pyramid"], dtype=torch.uint8, device="cuda")
        h = dm.dm_correlate_pyramid(ctx.ctx, torch.from_numpy(d1).cuda(), torch.from_numpy(d2).cuda(), ws)
        try:
            for l in range(pyr.geom.L + 1):
                vals, am, valid = dm.read_level(ws, dm.dm_pyramid_level(h, l))
                np.testing.assert_array_equal(valid, pyr.valid[l])
                keep = valid.astype(bool)
                want = pyr.pooled[l] if l < pyr.geom.L else pyr.top
                np.testing.assert_array_equal(vals[keep], want[keep], err_msg=f"level {l}")
                if l < pyr.geom.L:
                    np.testing.assert_array_equal(am[keep], pyr.argmax[l][keep], err_msg=f"level {l} codes")
        finally:
            dm.dm_pyramid_free(h)
    finally:
        ctx.close()

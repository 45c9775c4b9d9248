"""Failure paths, driven by the library's fault-injection hooks (dm_inject_fault)
without faulting the GPU: the host reports an injected launch or allocation
failure, a merge table that is too small fills up, a bounded device wait on a
barrier nothing completes runs out.  Each case checks the reported status and
that the same context then gives the oracle's results again.
"""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth

pytestmark = pytest.mark.gpu

W, H = 64, 48


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    pr = synth.make_pair_smooth(W, H, seed=1)
    want, _, _ = oracle_mod.match(pr.img1, pr.img2, "f32")
    ctx = dm.Context(dm.DM_FP32)
    yield torch, dm, ctx, pr, want
    dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_NONE)
    ctx.close()


def _match_status(torch, dm, ctx, pr):
    """dm_match through the C ABI; returns (matches, status word)."""
    ws = ctx.workspace("match", W, H, W, H)
    n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
    out = torch.zeros((n0, 5), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dm.dm_match(ctx.ctx, torch.from_numpy(pr.img1).cuda(), torch.from_numpy(pr.img2).cuda(), ws, out, cnt)
    st, _ = dm.dm_read_status(ctx.ctx, ws, 1)
    n = int(cnt.item())
    return out[:min(n, n0)].cpu().numpy().astype(np.float64), st


def test_merge_table_overflow_is_reported(env):
    torch, dm, ctx, pr, want = env
    dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_CAPACITY, 64)
    try:
        got, st = _match_status(torch, dm, ctx, pr)
    finally:
        dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_CAPACITY, 0)
    assert st & dm.DM_DEV_FRONTIER_OVERFLOW
    # the tuples that fitted still give well-formed matches
    assert len({(r[0], r[1]) for r in got}) == len(got)
    assert np.all((got[:, 0] - 2) % 4 == 0) and np.all((got[:, 1] - 2) % 4 == 0)
    # the context is unharmed
    again, st = _match_status(torch, dm, ctx, pr)
    assert st == 0
    np.testing.assert_array_equal(again, want)


def test_wait_that_runs_out_reports_timeout(env, oracle_mod):
    torch, dm, ctx, pr, want = env
    d1 = oracle_mod.descriptors(pr.img1, "f32")
    d2 = oracle_mod.descriptors(pr.img2, "f32")
    t1, t2 = torch.from_numpy(d1).cuda(), torch.from_numpy(d2).cuda()
    ws = torch.empty(dm.dm_workspace_bytes(ctx.ctx, W, H, W, H)["pyramid"], dtype=torch.uint8, device="cuda")
    dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_WAIT, 2000)
    try:
        # (no backtracking on this pyramid: the tiles of the CTAs that gave up were never written)
        h = dm.dm_correlate_pyramid(ctx.ctx, t1, t2, ws)
        dm.dm_pyramid_free(h)
        st, _ = dm.dm_read_status(ctx.ctx, ws, 1)
        assert st & dm.DM_DEV_TIMEOUT
    finally:
        dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_WAIT, 0)
    torch.cuda.synchronize()
    # the same context and workspace, without the hook: the oracle's pyramid
    h = dm.dm_correlate_pyramid(ctx.ctx, t1, t2, ws)
    try:
        st, _ = dm.dm_read_status(ctx.ctx, ws, 1)
        assert st == 0
        pyr = oracle_mod.pyramid(d1, d2, "f32")
        for l in range(pyr.geom.L + 1):
            vals, am, valid = dm.read_level(ws, dm.dm_pyramid_level(h, l))
            keep = valid.astype(bool)
            ref = pyr.pooled[l] if l < pyr.geom.L else pyr.top
            np.testing.assert_array_equal(vals[keep], ref[keep])
    finally:
        dm.dm_pyramid_free(h)
    again, st = _match_status(torch, dm, ctx, pr)
    assert st == 0
    np.testing.assert_array_equal(again, want)


@pytest.mark.parametrize("site,stage", [(1, "level-0 correlation"), (2, "pyramid levels"), (3, "backtracking")])
def test_injected_launch_failure(env, site, stage):
    torch, dm, ctx, pr, want = env
    dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_LAUNCH, site)
    try:
        with pytest.raises(dm.DmError) as e:
            _match_status(torch, dm, ctx, pr)
    finally:
        dm.dm_inject_fault(ctx.ctx, dm.DM_FAULT_LAUNCH, 0)
    assert e.value.status == dm.DM_ECUDA
    assert "injected" in str(e.value) and stage in str(e.value)
    torch.cuda.synchronize()                      # whatever was queued before the failure completes
    again, st = _match_status(torch, dm, ctx, pr)
    assert st == 0
    np.testing.assert_array_equal(again, want)


def test_injected_allocation_failure(env):
    torch, dm, ctx, pr, want = env
    dm.dm_inject_fault(None, dm.DM_FAULT_ALLOC, 1)
    with pytest.raises(dm.DmError) as e:
        dm.dm_create()
    assert e.value.status == dm.DM_ENOMEM
    h = dm.dm_create()                             # the hook fired once; creation works again
    dm.dm_destroy(h)
    # armed for the second creation: the context (first) is created, the first
    # event dm_timing_start creates (second) fails; the context keeps working
    dm.dm_inject_fault(None, dm.DM_FAULT_ALLOC, 2)
    c2 = dm.Context(dm.DM_FP32)
    try:
        with pytest.raises(dm.DmError) as e:
            dm.dm_timing_start(c2.ctx, 3)
        assert e.value.status == dm.DM_ENOMEM and "injected" in str(e.value)
        dm.dm_timing_start(c2.ctx, 3)
        np.testing.assert_array_equal(c2.match(pr.img1, pr.img2).cpu().numpy().astype(np.float64), want)
    finally:
        dm.dm_inject_fault(None, dm.DM_FAULT_ALLOC, 0)
        c2.close()

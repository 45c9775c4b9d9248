"""dm_backtrack_noalloc: backtracking for callers that cannot allocate.

Some callers cannot give the library a device workspace (plug-ins in a host
application that owns all device memory, loops that must never call
cudaMalloc).  dm_backtrack_noalloc uses a fixed scratch array inside the
library instead.  These checks call it through the C ABI and compare its
matches with those of dm_backtrack on the same pyramid -- bit for bit, the
FP32 tolerance of the other parity tests -- on three calls in a row (a
small pair, a larger one, the small one again), so that nothing left in the
shared scratch by an earlier call can leak into a later one.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    ctx = dm.Context(dm.DM_FP32)
    yield torch, dm, ctx
    ctx.close()


def _pyramid(torch, dm, ctx, img1, img2):
    H1, W1 = img1.shape
    H2, W2 = img2.shape
    ws = ctx.workspace("desc", W1, H1, W2, H2)
    descs = []
    for img in (img1, img2):
        H, W = img.shape
        d = torch.empty((H, W, 9), dtype=torch.float32, device="cuda")
        dm.dm_descriptors(ctx.ctx, torch.from_numpy(img).cuda(), d, ws)
        descs.append(d)
    pws = torch.empty(dm.dm_workspace_bytes(ctx.ctx, W1, H1, W2, H2)["pyramid"], dtype=torch.uint8, device="cuda")
    h = dm.dm_correlate_pyramid(ctx.ctx, descs[0], descs[1], pws)
    return h, pws, descs


def _with_workspace(torch, dm, ctx, h, W1, H1, W2, H2, n0):
    ws = torch.empty(dm.dm_workspace_bytes(ctx.ctx, W1, H1, W2, H2)["backtrack"], dtype=torch.uint8, device="cuda")
    out = torch.zeros((n0, 5), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dm.dm_backtrack(ctx.ctx, h, ws, out, cnt)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return out[:n].cpu().numpy()


def _no_alloc(torch, dm, ctx, h, n0):
    out = torch.full((n0, 5), -1.0, dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    dm.dm_backtrack_noalloc(ctx.ctx, h, out, cnt)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return out[:n].cpu().numpy()


def test_no_alloc_matches_workspace_version_repeatedly(env):
    torch, dm, ctx = env
    # the smaller pair again after the larger one: entries a larger earlier call
    # left in the shared scratch are the risky direction
    small = synth.make_pair_smooth(64, 48, seed=21)
    pairs = [small, synth.make_pair_motif(96, 72, seed=22, max_disp=10.0), small]
    for pr in pairs:
        H, W = pr.img1.shape
        n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
        h, _pws, _d = _pyramid(torch, dm, ctx, pr.img1, pr.img2)
        try:
            want = _with_workspace(torch, dm, ctx, h, W, H, W, H, n0)
            got = _no_alloc(torch, dm, ctx, h, n0)
            assert len(want) > 0
            np.testing.assert_array_equal(got, want)
        finally:
            dm.dm_pyramid_free(h)


def test_no_alloc_refuses_pairs_beyond_its_scratch(env):
    torch, dm, ctx = env
    pr = synth.make_pair_smooth(256, 192, seed=23)
    need = dm.dm_workspace_bytes(ctx.ctx, 256, 192, 256, 192)["backtrack"]
    assert need > dm.NOALLOC_SCRATCH_BYTES
    h, _pws, _d = _pyramid(torch, dm, ctx, pr.img1, pr.img2)
    try:
        out = torch.zeros((10, 5), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pytest.raises(dm.DmError) as e:
            dm.dm_backtrack_noalloc(ctx.ctx, h, out, cnt)
        assert e.value.status == dm.DM_ENOMEM
        assert "scratch" in str(e.value)
    finally:
        torch.cuda.synchronize()
        dm.dm_pyramid_free(h)

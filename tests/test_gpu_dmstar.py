"""DM* (Sec. 5.3: local-maximum entry points at every level, start + end
scoring) on the GPU, through the C ABI.

* FP32: dm_match_star equals, bit for bit, the oracle's FP32 DM* chain, with
  compensated and plain child sums, on equal, ragged and unequal sizes.
* dm_backtrack_star on a pyramid of dm_correlate_pyramid gives the same
  matches as dm_match_star.
* BF16 level 0: the matches agree with the FP32 path on most patches.
* Argument and workspace checks.
"""
import numpy as np
import pytest

import oracle
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


def _ctx(prec, compensated=True):
    from paper_1506_07656_gb300 import dm
    return dm.Context({"fp32": dm.DM_FP32, "bf16": dm.DM_BF16}[prec], compensated=compensated)


CASES = [(40, 32, 40, 32, 1), (37, 29, 37, 29, 2), (41, 23, 53, 35, 3), (64, 48, 64, 48, 4), (130, 70, 130, 70, 5)]


def _pair(W1, H1, W2, H2, seed):
    if (W1, H1) == (W2, H2):
        pr = synth.make_pair_smooth(W1, H1, seed)
        return pr.img1.astype(np.float32), pr.img2.astype(np.float32)
    a = synth.make_pair_smooth(W1, H1, seed).img1
    b = synth.make_pair_smooth(W2, H2, seed + 100).img2
    return a.astype(np.float32), b.astype(np.float32)


def _run(torch, ctx, img1, img2):
    t = ctx.match_star(img1, img2)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("compensated", [True, False])
@pytest.mark.parametrize("case", CASES)
def test_fp32_bit_exact_with_oracle(torch_cuda, case, compensated):
    W1, H1, W2, H2, seed = case
    img1, img2 = _pair(W1, H1, W2, H2, seed)
    want = oracle.dmstar_match(img1, img2, "f32", compensated=compensated)
    got = _run(torch_cuda, _ctx("fp32", compensated), img1, img2)
    assert len(want) > 0
    np.testing.assert_array_equal(got, want.astype(np.float32).astype(np.float64))


def test_backtrack_star_on_a_pyramid_equals_match_star(torch_cuda):
    from paper_1506_07656_gb300 import dm
    torch = torch_cuda
    W, H = 64, 48
    img1, img2 = _pair(W, H, W, H, 4)
    ctx = _ctx("fp32")
    want = _run(torch, ctx, img1, img2)
    sizes = dm.dm_workspace_bytes(ctx.ctx, W, H, W, H)
    d1 = torch.empty((H, W, 9), dtype=torch.float32, device="cuda")
    d2 = torch.empty((H, W, 9), dtype=torch.float32, device="cuda")
    tmp = torch.empty(sizes["desc"], dtype=torch.uint8, device="cuda")
    dm.dm_descriptors(ctx.ctx, torch.from_numpy(img1).cuda(), d1, tmp)
    dm.dm_descriptors(ctx.ctx, torch.from_numpy(img2).cuda(), d2, tmp)
    pws = torch.empty(sizes["pyramid"], dtype=torch.uint8, device="cuda")
    h = dm.dm_correlate_pyramid(ctx.ctx, d1, d2, pws)
    bws = torch.empty(dm.dm_star_workspace_bytes(ctx.ctx, W, H, W, H)["backtrack"], dtype=torch.uint8, device="cuda")
    n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
    out = torch.zeros((n0, 5), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dm.dm_backtrack_star(ctx.ctx, h, bws, out, cnt)
    torch.cuda.synchronize()
    got = out[:int(cnt.item())].cpu().numpy().astype(np.float64)
    dm.dm_pyramid_free(h)
    np.testing.assert_array_equal(got, want)
    status, reached = dm.dm_read_status(ctx.ctx, bws, 2)
    assert status == 0 and reached[0] > 0


def test_bf16_agrees_with_fp32(torch_cuda):
    img1, img2 = _pair(130, 70, 130, 70, 5)
    m32 = _run(torch_cuda, _ctx("fp32"), img1, img2)
    m16 = _run(torch_cuda, _ctx("bf16"), img1, img2)
    key = {(r[0], r[1]): (r[2], r[3]) for r in m32}
    agree = np.mean([key.get((r[0], r[1])) == (r[2], r[3]) for r in m16])
    assert agree >= 0.8, agree
    assert abs(len(m16) - len(m32)) <= 0.2 * len(m32)


def test_argument_and_workspace_checks(torch_cuda):
    from paper_1506_07656_gb300 import dm
    torch = torch_cuda
    ctx = _ctx("fp32")
    img1, img2 = _pair(40, 32, 40, 32, 1)
    i1 = torch.as_tensor(img1, device="cuda")
    i2 = torch.as_tensor(img2, device="cuda")
    sizes = dm.dm_star_workspace_bytes(ctx.ctx, 40, 32, 40, 32)
    assert sizes["match"] > dm.dm_workspace_bytes(ctx.ctx, 40, 32, 40, 32)["match"]
    out = torch.empty((100, 5), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    small = torch.empty(sizes["match"] - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_match_star(ctx.ctx, i1, i2, small, out, cnt)
    assert e.value.status == dm.DM_ENOMEM
    ws = torch.empty(sizes["match"] + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_match_star(ctx.ctx, i1, i2, ws[16:], out, cnt)
    assert e.value.status == dm.DM_EINVAL
    with pytest.raises(dm.DmError) as e:
        dm.dm_match_star(ctx.ctx, torch.zeros((3, 40), device="cuda"), i2, ws, out, cnt)
    assert e.value.status == dm.DM_EINVAL

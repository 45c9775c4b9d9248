"""DeepFlow (Sec. 4.3) on the GPU, through the C ABI (dm_deepflow).

* FP32: the flow equals, bit for bit, the oracle's FP32 DeepFlow -- without
  matches, with the oracle's own DeepMatching matches as the matching term,
  on ragged sizes, with the brightness term switched on, and on sizes whose
  finest levels take the temporally blocked multi-launch path (more pixels
  than one CTA holds), with partial and full blocks of half-sweeps, and with
  more tiles than resident CTAs (the halos of later waves must not see the
  updates of earlier ones).
* identical images: zero flow.
* chaining: the matches of dm_match passed on the device (its count read on
  the device) give the same flow as the same matches passed from the host.
* argument and workspace checks.
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


def _ctx():
    from paper_1506_07656_gb300 import dm
    return dm.Context(dm.DM_FP32)


def _tex(W, H, t=(0.0, 0.0)):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    x, y = x - t[0], y - t[1]
    return (0.5 + 0.2 * np.sin(0.31 * x + 0.17 * y) + 0.15 * np.cos(0.23 * y - 0.11 * x)).astype(np.float32)


def _flow(torch, ctx, i1, i2, m=None, **kw):
    u, v = ctx.deepflow(i1, i2, m, **kw)
    torch.cuda.synchronize()
    return u.cpu().numpy(), v.cpu().numpy()


CASES = ["translation_64x48", "dm_matches_64x48", "ragged_37x29", "brightness_term_48x40", "multi_launch_320x240",
         "blocked_sor_97x75", "many_tiles_1024x436"]


def _case(name):
    if name == "translation_64x48":
        return _tex(64, 48), _tex(64, 48, (1.5, -0.7)), None, {}
    if name == "dm_matches_64x48":
        pr = synth.make_pair_smooth(64, 48, seed=3, max_disp=4.0)
        m, _, _ = oracle.match(pr.img1, pr.img2, "f32")
        return pr.img1.astype(np.float32), pr.img2.astype(np.float32), m, {}
    if name == "ragged_37x29":
        pr = synth.make_pair_smooth(37, 29, seed=4, max_disp=3.0)
        m, _, _ = oracle.match(pr.img1, pr.img2, "f32")
        return pr.img1.astype(np.float32), pr.img2.astype(np.float32), m, {"min_size": 8}
    if name == "brightness_term_48x40":
        return _tex(48, 40), _tex(48, 40, (-0.8, 1.2)), None, {"delta": 0.5, "gamma": 0.3}
    if name == "multi_launch_320x240":
        pr = synth.make_pair_smooth(320, 240, seed=6, max_disp=6.0)
        rng = np.random.default_rng(1)
        xs, ys = rng.integers(0, 320, 400), rng.integers(0, 240, 400)
        m = np.stack([xs, ys, np.clip(xs + 2, 0, 319), np.clip(ys - 1, 0, 239), rng.random(400)], 1)
        return pr.img1.astype(np.float32), pr.img2.astype(np.float32), m, {"n_fixed": 2, "n_sor": 5}
    if name == "blocked_sor_97x75":                   # default parameters, finest levels above one CTA's size
        pr = synth.make_pair_smooth(97, 75, seed=12, max_disp=4.0)
        m, _, _ = oracle.match(pr.img1, pr.img2, "f32")
        return pr.img1.astype(np.float32), pr.img2.astype(np.float32), m, {}
    if name == "many_tiles_1024x436":                 # more SOR tiles than resident CTAs (several waves), 2 levels
        pr = synth.make_pair_smooth(1024, 436, seed=21, max_disp=8.0)
        return pr.img1.astype(np.float32), pr.img2.astype(np.float32), None, {"min_size": 400}
    raise KeyError(name)


@pytest.mark.parametrize("case", CASES)
def test_fp32_bit_exact_with_oracle(torch_cuda, case):
    i1, i2, m, kw = _case(case)
    want_u, want_v = oracle.deepflow(i1, i2, m, "f32", **kw)
    got_u, got_v = _flow(torch_cuda, _ctx(), i1, i2, m, **kw)
    np.testing.assert_array_equal(got_u, want_u)
    np.testing.assert_array_equal(got_v, want_v)


def test_identical_images_zero_flow(torch_cuda):
    i1 = _tex(64, 48)
    u, v = _flow(torch_cuda, _ctx(), i1, i1)
    assert np.all(u == 0) and np.all(v == 0)


def test_chained_device_matches(torch_cuda):
    from paper_1506_07656_gb300 import dm
    torch = torch_cuda
    pr = synth.make_pair_smooth(64, 48, seed=8, max_disp=4.0)
    ctx = _ctx()
    i1 = torch.as_tensor(pr.img1, dtype=torch.float32, device="cuda")
    i2 = torch.as_tensor(pr.img2, dtype=torch.float32, device="cuda")
    n0 = dm.dm_geometry(64, 48, 64, 48)["n_patch0"]
    out = torch.zeros((n0, 5), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    dm.dm_match(ctx.ctx, i1, i2, ctx.workspace("match", 64, 48, 64, 48), out, cnt)
    prm = dm.dm_flow_params()
    ws = torch.empty(dm.dm_deepflow_workspace_bytes(ctx.ctx, 64, 48, n0, prm), dtype=torch.uint8, device="cuda")
    u = torch.empty((48, 64), dtype=torch.float32, device="cuda")
    v = torch.empty_like(u)
    dm.dm_deepflow(ctx.ctx, i1, i2, out, cnt, u, v, ws, prm)          # no host round trip in between
    torch.cuda.synchronize()
    m = out[:int(cnt.item())].cpu().numpy()
    u2, v2 = _flow(torch, ctx, pr.img1, pr.img2, m)
    np.testing.assert_array_equal(u.cpu().numpy(), u2)
    np.testing.assert_array_equal(v.cpu().numpy(), v2)


def test_argument_and_workspace_checks(torch_cuda):
    from paper_1506_07656_gb300 import dm
    torch = torch_cuda
    ctx = _ctx()
    i1 = torch.as_tensor(_tex(40, 30), device="cuda")
    u = torch.empty((30, 40), dtype=torch.float32, device="cuda")
    v = torch.empty_like(u)
    prm = dm.dm_flow_params()
    need = dm.dm_deepflow_workspace_bytes(ctx.ctx, 40, 30, 0, prm)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_deepflow(ctx.ctx, i1, i1, None, None, u, v, small, prm)
    assert e.value.status == dm.DM_ENOMEM
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dm.DmError) as e:
        dm.dm_deepflow(ctx.ctx, i1, i1, None, None, u, v, ws[16:], prm)
    assert e.value.status == dm.DM_EINVAL
    bad = dm.dm_flow_params(eta=1.5)
    with pytest.raises(dm.DmError) as e:
        dm.dm_deepflow_workspace_bytes(ctx.ctx, 40, 30, 0, bad)
    assert e.value.status == dm.DM_EINVAL

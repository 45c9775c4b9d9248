"""Batched form: dm_match_batch over pairs of mixed sizes, and its CUDA-graph replay.

Each pair of a batch must give exactly the matches dm_match gives for it
alone; a captured graph of the batch, replayed on new image contents written
into the same input buffers, must give the matches of those new images.
"""
import numpy as np
import pytest

from paper_1506_07656_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (37, 29), (96, 72), (130, 70), (64, 48)]


@pytest.fixture(scope="module", params=["fp32", "bf16", "fp8"])
def env(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    ctx = dm.Context({"fp32": dm.DM_FP32, "bf16": dm.DM_BF16, "fp8": dm.DM_FP8_E4M3}[request.param])
    yield torch, dm, ctx
    ctx.close()


def _alloc(torch, dm, sizes, seed0):
    items, host = [], []
    for k, (W, H) in enumerate(sizes):
        pr = synth.make_pair_smooth(W, H, seed=seed0 + k)
        n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
        i1 = torch.from_numpy(pr.img1).cuda()
        i2 = torch.from_numpy(pr.img2).cuda()
        out = torch.zeros((n0, 5), dtype=torch.float32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        items.append((i1, i2, out, cnt))
        host.append(pr)
    return items, host


def _single(ctx, pr):
    return ctx.match(pr.img1, pr.img2).cpu().numpy()


def test_batch_equals_single_pairs(env):
    torch, dm, ctx = env
    items, host = _alloc(torch, dm, SIZES, 40)
    pairs = dm.make_pairs(items)
    ws = torch.empty(dm.dm_batch_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
    dm.dm_match_batch(ctx.ctx, pairs, ws)
    torch.cuda.synchronize()
    for (i1, i2, out, cnt), pr in zip(items, host):
        n = int(cnt.item())
        np.testing.assert_array_equal(out[:n].cpu().numpy(), _single(ctx, pr))


def test_batch_graph_replay(env):
    torch, dm, ctx = env
    items, host = _alloc(torch, dm, SIZES, 60)
    pairs = dm.make_pairs(items)
    ws = torch.empty(dm.dm_batch_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        dm.dm_match_batch(ctx.ctx, pairs, ws, side)       # uncaptured first call
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        dm.dm_match_batch(ctx.ctx, pairs, ws, side)
    for rep, seed0 in enumerate((80, 100)):
        new = [synth.make_pair_smooth(W, H, seed=seed0 + k) for k, (W, H) in enumerate(SIZES)]
        for (i1, i2, out, cnt), pr in zip(items, new):
            i1.copy_(torch.from_numpy(pr.img1))
            i2.copy_(torch.from_numpy(pr.img2))
            out.zero_()
            cnt.zero_()
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        for (i1, i2, out, cnt), pr in zip(items, new):
            n = int(cnt.item())
            np.testing.assert_array_equal(out[:n].cpu().numpy(), _single(ctx, pr))


def test_batch_rejects_bad_pair_before_launch(env):
    torch, dm, ctx = env
    items, _ = _alloc(torch, dm, [(64, 48)], 120)
    bad = list(items) + [(torch.zeros((3, 3), device="cuda"), torch.zeros((3, 3), device="cuda"),
                          torch.zeros((1, 5), device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))]
    pairs = dm.make_pairs(bad)
    ws = torch.empty(1 << 24, dtype=torch.uint8, device="cuda")
    items[0][3].fill_(-7)
    with pytest.raises(dm.DmError) as e:
        dm.dm_match_batch(ctx.ctx, pairs, ws)
    assert e.value.status == dm.DM_EINVAL
    torch.cuda.synchronize()
    assert int(items[0][3].item()) == -7        # nothing ran for the valid first pair either


@pytest.mark.parametrize("lanes", [1, 3, 4])
def test_batch_lanes_give_identical_matches(env, lanes):
    """Any number of concurrent lanes, and a workspace too small for all of
    them (fewer lanes run), gives the matches of the single-pair calls."""
    torch, dm, ctx = env
    items, host = _alloc(torch, dm, SIZES, 140)
    pairs = dm.make_pairs(items)
    try:
        dm.dm_set_batch_lanes(ctx.ctx, lanes)
        full = dm.dm_batch_workspace_bytes(ctx.ctx, pairs)
        for nbytes in (full, full // lanes + 256):
            ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            for it in items:
                it[2].zero_()
                it[3].zero_()
            dm.dm_match_batch(ctx.ctx, pairs, ws)
            torch.cuda.synchronize()
            for (i1, i2, out, cnt), pr in zip(items, host):
                n = int(cnt.item())
                np.testing.assert_array_equal(out[:n].cpu().numpy(), _single(ctx, pr))
    finally:
        dm.dm_set_batch_lanes(ctx.ctx, 2)
    with pytest.raises(dm.DmError):
        dm.dm_set_batch_lanes(ctx.ctx, 5)


def _host_items(torch, dm, sizes, seed0):
    items, host = [], []
    for k, (W, H) in enumerate(sizes):
        pr = synth.make_pair_smooth(W, H, seed=seed0 + k)
        n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
        items.append((torch.from_numpy(pr.img1).pin_memory(), torch.from_numpy(pr.img2).pin_memory(),
                      torch.full((n0, 5), -1.0, dtype=torch.float32).pin_memory(),
                      torch.full((1,), -1, dtype=torch.int32).pin_memory()))
        host.append(pr)
    return items, host


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_host_batch_equals_single_pairs(env, lanes):
    """dm_match_batch_host: images from (page-locked) host memory, matches and
    counts back to host memory, inside the lanes; every pair equals dm_match."""
    torch, dm, ctx = env
    items, host = _host_items(torch, dm, SIZES, 200)
    pairs = dm.make_pairs_host(items)
    try:
        dm.dm_set_batch_lanes(ctx.ctx, lanes)
        ws = torch.empty(dm.dm_batch_host_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
        dm.dm_match_batch_host(ctx.ctx, pairs, ws)
        torch.cuda.synchronize()
    finally:
        dm.dm_set_batch_lanes(ctx.ctx, 2)
    for (h1, h2, out, cnt), pr in zip(items, host):
        n = int(cnt.item())
        np.testing.assert_array_equal(out[:n].numpy(), _single(ctx, pr))


def test_host_batch_graph_replay(env):
    """The host-buffer batch captured in a CUDA graph (copies included) and
    replayed on new image contents written into the same host buffers."""
    torch, dm, ctx = env
    items, _ = _host_items(torch, dm, SIZES, 220)
    pairs = dm.make_pairs_host(items)
    ws = torch.empty(dm.dm_batch_host_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        dm.dm_match_batch_host(ctx.ctx, pairs, ws, side)      # uncaptured first call
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        dm.dm_match_batch_host(ctx.ctx, pairs, ws, side)
    for seed0 in (240, 260):
        new = [synth.make_pair_smooth(W, H, seed=seed0 + k) for k, (W, H) in enumerate(SIZES)]
        for (h1, h2, out, cnt), pr in zip(items, new):
            h1.copy_(torch.from_numpy(pr.img1))
            h2.copy_(torch.from_numpy(pr.img2))
            cnt.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        for (h1, h2, out, cnt), pr in zip(items, new):
            n = int(cnt.item())
            assert n >= 0
            np.testing.assert_array_equal(out[:n].numpy(), _single(ctx, pr))


@pytest.mark.parametrize("wave", [1, 2, 3, 8])
def test_batch_wave_widths_give_identical_matches(env, wave):
    """Cross-pair waves of any width (1: every pair its own launches) give the
    matches of the single-pair calls; a wave issues one launch per step for all
    of its pairs."""
    torch, dm, ctx = env
    items, host = _alloc(torch, dm, SIZES, 300)
    pairs = dm.make_pairs(items)
    try:
        dm.dm_set_batch_wave(ctx.ctx, wave)
        dm.dm_set_batch_lanes(ctx.ctx, 1)
        ws = torch.empty(dm.dm_batch_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
        dm.dm_match_batch(ctx.ctx, pairs, ws)            # (one-time set-up outside the count)
        torch.cuda.synchronize()
        l0 = dm.dm_timing_read(ctx.ctx)[2]
        dm.dm_match_batch(ctx.ctx, pairs, ws)
        torch.cuda.synchronize()
        launches = dm.dm_timing_read(ctx.ctx)[2] - l0
    finally:
        dm.dm_set_batch_wave(ctx.ctx, 1)
        dm.dm_set_batch_lanes(ctx.ctx, 2)
    for (i1, i2, out, cnt), pr in zip(items, host):
        n = int(cnt.item())
        np.testing.assert_array_equal(out[:n].cpu().numpy(), _single(ctx, pr))
    l1 = dm.dm_timing_read(ctx.ctx)[2]
    for pr in host:
        _single(ctx, pr)
    singles = dm.dm_timing_read(ctx.ctx)[2] - l1
    print(f"wave {wave}: {launches} launches for {len(SIZES)} pairs, {singles} one pair at a time")
    if wave >= len(SIZES):
        assert launches * 2 < singles
    with pytest.raises(dm.DmError):
        dm.dm_set_batch_wave(ctx.ctx, 9)


def test_batch_wave_equals_oracle_on_uneven_pairs(oracle_mod):
    """FP32 cross-pair wave over pairs of different sizes, image 2 of another
    size than image 1 included: every pair equals the FP32 oracle bit for bit."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    rng = np.random.default_rng(17)
    imgs = [(synth.make_pair_smooth(64, 48, seed=1).img1, synth.make_pair_smooth(64, 48, seed=1).img2),
            (synth.value_noise(41, 23, rng).astype(np.float32), synth.value_noise(53, 35, rng).astype(np.float32)),
            (synth.make_pair_smooth(37, 29, seed=2).img1, synth.make_pair_smooth(37, 29, seed=2).img2),
            (synth.value_noise(96, 61, rng).astype(np.float32), synth.value_noise(71, 80, rng).astype(np.float32))]
    ctx = dm.Context(dm.DM_FP32)
    try:
        items = []
        for a, b in imgs:
            n0 = dm.dm_geometry(a.shape[1], a.shape[0], b.shape[1], b.shape[0])["n_patch0"]
            items.append((torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(),
                          torch.zeros((n0, 5), dtype=torch.float32, device="cuda"),
                          torch.zeros(1, dtype=torch.int32, device="cuda")))
        pairs = dm.make_pairs(items)
        dm.dm_set_batch_wave(ctx.ctx, 4)
        ws = torch.empty(dm.dm_batch_workspace_bytes(ctx.ctx, pairs), dtype=torch.uint8, device="cuda")
        dm.dm_match_batch(ctx.ctx, pairs, ws)
        torch.cuda.synchronize()
        for (a, b), (i1, i2, out, cnt) in zip(imgs, items):
            want, _, _ = oracle_mod.match(a, b, "f32")
            n = int(cnt.item())
            np.testing.assert_array_equal(out[:n].cpu().numpy().astype(np.float64), want)
    finally:
        ctx.close()


def test_batch_wave_at_workload_sizes():
    """BF16 wave of the four workload sizes (1024x436, 640x480, 1242x375 with
    L = 8 after the top-level rule, 512x224 with L = 7): each pair equals its
    single-pair dm_match bit for bit and reports a clean status."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_07656_gb300 import build, dm
    build.build()
    sizes = [(1024, 436), (640, 480), (1242, 375), (512, 224)]
    prs = [synth.make_pair_smooth(W, H, seed=400 + k, max_disp=40.0, with_flow=False) for k, (W, H) in enumerate(sizes)]
    ctx = dm.Context(dm.DM_BF16)
    try:
        want = [ctx.match(pr.img1, pr.img2).cpu().numpy() for pr in prs]
        ctx._ws.clear()
        torch.cuda.empty_cache()
        items = []
        for (W, H), pr in zip(sizes, prs):
            n0 = dm.dm_geometry(W, H, W, H)["n_patch0"]
            items.append((torch.from_numpy(pr.img1).cuda(), torch.from_numpy(pr.img2).cuda(),
                          torch.zeros((n0, 5), dtype=torch.float32, device="cuda"),
                          torch.zeros(1, dtype=torch.int32, device="cuda")))
        pairs = dm.make_pairs(items)
        dm.dm_set_batch_lanes(ctx.ctx, 1)
        dm.dm_set_batch_wave(ctx.ctx, len(sizes))
        slice_bytes = dm.dm_batch_workspace_bytes(ctx.ctx, pairs) // len(sizes)
        ws = torch.empty(slice_bytes * len(sizes), dtype=torch.uint8, device="cuda")
        dm.dm_match_batch(ctx.ctx, pairs, ws)
        torch.cuda.synchronize()
        for j, ((i1, i2, out, cnt), w) in enumerate(zip(items, want)):
            n = int(cnt.item())
            assert n > 0.3 * out.shape[0]
            np.testing.assert_array_equal(out[:n].cpu().numpy(), w)
            st, _ = dm.dm_read_status(ctx.ctx, ws[j * slice_bytes:], 1)
            assert st == 0
    finally:
        ctx.close()


def test_batch_autotuner_picks_a_shape_within_the_workspace(env):
    """dm_autotune_batch keeps a (wave width, lanes) whose slices fit the
    workspace, and the batch then still gives the single-pair matches."""
    torch, dm, ctx = env
    items, host = _alloc(torch, dm, SIZES, 500)
    pairs = dm.make_pairs(items)
    try:
        dm.dm_set_batch_wave(ctx.ctx, 1)
        dm.dm_set_batch_lanes(ctx.ctx, 1)
        lane = dm.dm_batch_workspace_bytes(ctx.ctx, pairs)
        ws = torch.empty(4 * lane, dtype=torch.uint8, device="cuda")
        shape = dm.dm_autotune_batch(ctx.ctx, pairs, ws)
        assert shape["wave"] in (1, 2, 3, 4) and 1 <= shape["lanes"] <= 4
        assert shape["wave"] * shape["lanes"] <= 4
        for it in items:
            it[2].zero_()
            it[3].zero_()
        dm.dm_match_batch(ctx.ctx, pairs, ws)
        torch.cuda.synchronize()
        for (i1, i2, out, cnt), pr in zip(items, host):
            n = int(cnt.item())
            np.testing.assert_array_equal(out[:n].cpu().numpy(), _single(ctx, pr))
        with pytest.raises(dm.DmError) as e:
            dm.dm_autotune_batch(ctx.ctx, pairs, ws[:lane // 2])
        assert e.value.status == dm.DM_ENOMEM
    finally:
        dm.dm_set_batch_wave(ctx.ctx, 1)
        dm.dm_set_batch_lanes(ctx.ctx, 2)

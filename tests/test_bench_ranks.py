"""Replicas-only multi-GPU form of the bench, host side, on CPU: two gloo
ranks on 127.0.0.1 take the maximum of their step times and report the
whole-job throughput (every rank matches its own pairs; no data-path
collective)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 150.0][rank]                 # rank 1 is the slower replica
    ms_max = bench._max_over_ranks(torch, dist, local_ms, world, "cpu")
    value = bench._job_throughput(world, 20, ms_max / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms_max": ms_max, "value": value}, f)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["ms_max"] == 150.0
        assert abs(d["value"] - 2 * 20 / 0.150) < 1e-9


def test_single_rank_needs_no_process_group():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(torch, None, 3.5, 1, "cpu") == 3.5
    assert bench._job_throughput(1, 10, 2.0) == 5.0

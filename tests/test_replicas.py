"""The benchmark's multi-GPU host path on the CPU (gloo, world size 2).  Several GPUs run replicas:
every rank solves its own batch of wavelengths and nothing is exchanged on the data path, so the
only collective is the timing one: the job's time is the slowest rank's, and the whole-job rate
counts every rank's wavelengths."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r took 1000 + 500 r ms for its timed steps and 2 - r s end to end
        t_ms = bench.max_over_ranks(1000.0 + 500.0 * rank, world, "cpu")
        e2e_s = bench.max_over_ranks(2.0 - rank, world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"t_ms": t_ms, "e2e_s": e2e_s,
                   "value": bench.replica_rate(64, 20, world, t_ms / 1e3)}, f)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_rate(64, 20, 1, 2.0) == 640.0


@pytest.mark.timeout(300)
def test_two_replicas_take_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            got = json.load(f)
        assert got["t_ms"] == 1500.0
        assert got["e2e_s"] == 2.0
        # 64 wavelengths x 20 steps on each of the 2 ranks in the slowest rank's 1.5 s
        assert got["value"] == pytest.approx(64 * 20 * 2 / 1.5)

"""The N-GPU benchmark's host logic on two CPU ranks over gloo: every rank its
own energy grid, the job time is the slowest rank's, the whole-job
throughput counts all ranks' energies, and the reference arm's non-zero
ranks exit without work."""
import json
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    E = np.linspace(-2.0, 2.0, 5) + 1e-6j
    mine = bench.rank_energies(E, rank, world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"e0": [mine[0].real, mine[0].imag], "ms": ms,
                   "value": bench.job_throughput(world, 5, 64, ms)}, f)


def test_two_gloo_ranks_share_the_max_time_and_own_energy_grids(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(world)]
    assert r[0]["ms"] == r[1]["ms"] == 15.0                 # the slowest rank
    assert abs(r[0]["e0"][0] - (-2.0)) < 1e-15
    assert abs(r[1]["e0"][0] - (-2.0 + 1e-3)) < 1e-15      # rank 1: its own grid
    assert r[0]["value"] == pytest.approx(2 * 5 * 64 / 15e-3)


def test_reference_arm_nonzero_rank_does_no_work():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    class A:
        workload = "batched64x64"
        cpu_energies = 8
        steps = 1
        warmup = 0
    assert bench.run_reference(A(), 1, 2) is None

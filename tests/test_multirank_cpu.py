"""The N-GPU benchmark's host logic on two CPU ranks over gloo: the ranks
split one energy list into contiguous shares that concatenate to it, the job
time is the slowest rank's, the whole-job throughput counts every energy
once, and the reference arm's non-zero ranks exit without work."""
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
    E1 = np.linspace(-2.0, 2.0, 5) + 1e-6j          # one rank's workload list
    job = bench.job_energies(E1, world)                # the job's list: world x 5 energies
    mine = bench.rank_energies(job, rank, world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"mine": [[z.real, z.imag] for z in mine], "job": [[z.real, z.imag] for z in job], "ms": ms,
                   "value": bench.job_throughput(world, len(mine), 64, ms)}, f)


def test_two_gloo_ranks_split_one_energy_list_and_share_the_max_time(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(world)]
    assert r[0]["ms"] == r[1]["ms"] == 15.0                 # the slowest rank
    job = r[0]["job"]
    assert job == r[1]["job"] and len(job) == 10
    assert job[0] == [-2.0, 1e-6] and job[-1] == [2.0, 1e-6]
    # contiguous shares that concatenate to the job's list: every energy once
    assert r[0]["mine"] + r[1]["mine"] == job
    assert len(r[0]["mine"]) == len(r[1]["mine"]) == 5
    assert r[0]["value"] == pytest.approx(10 * 64 / 15e-3)


def test_energy_shards_cover_the_list_once():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import paper_2605_19910_gb300 as P
    for n in (1, 7, 512, 1000):
        for world in (1, 2, 3, 8):
            shards = [P.energy_shard(n, r, world) for r in range(world)]
            assert shards[0][0] == 0 and shards[-1][1] == n
            assert all(shards[k][1] == shards[k + 1][0] for k in range(world - 1))
            sizes = [hi - lo for lo, hi in shards]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        P.energy_shard(8, 2, 2)


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

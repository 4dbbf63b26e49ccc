"""The N > 1 path of bench.py on CPU: two gloo ranks in separate processes.

Every rank multiplies its own product (seed + rank), so the products shard
across ranks with no data-path collective; the only exchange is the timing
reduction, which takes the slowest rank's time, and the whole-job rate counts
every rank's products over that time.  Under torchrun the reference arm runs
on rank 0 alone and the other ranks return without work."""
import argparse
import os
import socket
import time

import numpy as np
import pytest

import bench


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a rank's own step time: rank r takes (r + 1) * 40 ms per step
        steps = 3
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            time.sleep(0.04 * (rank + 1))
        dist.barrier()
        mine = time.perf_counter() - t0
        slowest = bench.max_over_ranks(dist, mine, "cpu")
        rate = bench.whole_job_rate(world, steps, slowest)
        seed = bench.rank_seed(1, rank)
        case = bench.make_workload("16x16", seed)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), mine=mine, slowest=slowest, rate=rate, seed=seed,
                 A=case.A, B=case.B)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_shard_products(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [np.load(tmp_path / ("rank%d.npz" % k)) for k in range(world)]
    slowest = max(float(x["mine"]) for x in r)
    for x in r:
        assert float(x["slowest"]) == pytest.approx(slowest, rel=0, abs=1e-12)
        assert float(x["rate"]) == pytest.approx(world * 3 / slowest)
    # the slowest rank sleeps 2 x 3 x 40 ms between the barriers
    assert slowest >= 0.24
    # each rank multiplies its own product
    assert int(r[0]["seed"]) != int(r[1]["seed"])
    assert not np.array_equal(r[0]["A"], r[1]["A"]) or not np.array_equal(r[0]["B"], r[1]["B"])


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(None, 2.5, "cpu") == 2.5
    assert bench.whole_job_rate(1, 4, 2.0) == 2.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    # a rank other than 0 returns before touching the workload or the oracle
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="no such workload", seed=0, rot_base=256, warmup=3, steps=1, gpus=2)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""

"""The multi-process path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Snapshots are independent, so N GPUs run N replicas with no collective on
the data path (weak scaling).  What the ranks do share is host logic, checked
here without a GPU:
  * the ranks' snapshot recipes are disjoint (no seed is filtered twice) and
    every rank sees the same workload shape;
  * the job's step time is the maximum over ranks, identical on every rank;
  * the reported value counts the units of all ranks.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns = bench.WORKLOADS["re550_d64"][-1]
        recipe = bench.snapshot_recipe(rank, ns)
        recipes = [None] * world
        dist.all_gather_object(recipes, recipe)
        ms = bench.max_over_ranks(1.5 + rank, "cpu", world)      # rank 1 is the slow one
        rate = bench.whole_job_rate(world, 1000, 4, ms)
        out[rank] = (recipes, ms, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_bench_logic():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    recipes, ms0, rate0 = out[0]
    _, ms1, rate1 = out[1]
    seeds = [{seed for seed, _, _ in r} for r in recipes]
    assert not (seeds[0] & seeds[1])                            # disjoint snapshots
    assert len(recipes[0]) == len(recipes[1])
    assert ms0 == ms1 == 2.5                                    # the slowest rank's time, everywhere
    assert rate0 == rate1 == 2 * 1000 * 4 / 2.5e-3              # all ranks' units over that time

"""The multi-rank host logic of bench.py (one process per GPU, weak scaling):
each rank's jobs have their own seeds, the job's time is the slowest rank's
(max over ranks), and the whole-job rate counts the attempts of every rank.
Run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    specs, _ = bench.workload_specs("chains", rank, None)
    step_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    slow = bench.rank_max(step_ms, world, dev)
    fast_rate = bench.rank_min(1000.0 * (rank + 1), world, dev)
    att_step = sum(s.L * s.R for s in specs)
    value = bench.job_rate(world * 3 * att_step, slow)
    out[rank] = ([s.seed for s in specs], slow, fast_rate, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    seeds0, slow0, fast0, value0 = out[0]
    seeds1, slow1, fast1, value1 = out[1]
    assert seeds0 == list(range(1, 9)) and seeds1 == list(range(9, 17))  # disjoint chains per rank
    assert slow0 == slow1 == 15.0     # max over ranks, seen by both
    assert fast0 == fast1 == 1000.0   # min over ranks
    att = 8 * 1024 * 64
    assert value0 == value1 == pytest.approx(2 * 3 * att / 0.015)

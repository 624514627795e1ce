"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path shards by evidence cases: every rank draws its own batch, runs it
alone, and the job's throughput is all ranks' cases over the slowest rank's
time.  No collective touches the data; only the timing is reduced.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from synth import configs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=16, seed=bench.rank_evidence_seed("bn60", rank))
    ms = 10.0 + 5.0 * rank   # the rank's own timed region
    dist.barrier()
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (slowest, bench.aggregate_rate(16, world, slowest / 4), ev.tobytes())
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 15.0          # max over ranks
    assert out[0][1] == out[1][1] == 16 * 2 / (15.0 / 4 / 1e3)
    assert out[0][2] != out[1][2]                  # independent batches


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.aggregate_rate(100, 1, 10.0) == 100 / 0.01

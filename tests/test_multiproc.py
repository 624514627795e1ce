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


def _rank_path(rank, world, port, out):
    """The bench's rank path with a stand-in step: own seeds, the timed
    region (barrier, steps, barrier, max over ranks), the job's rate and,
    on rank 0, the line."""
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    net = configs.network("bn20")
    n_cases, steps = 32, 3
    ev = configs.evidence("bn20", net, n_cases=n_cases, seed=bench.rank_evidence_seed("bn20", rank))

    def step():                      # a stand-in for one pass: rank 1 is slower
        time.sleep(0.004 * (1 + rank))
        return int(ev.sum())

    ms = bench.timed_region(step, steps, dist, "cpu", bench.WallTimer())
    value = bench.aggregate_rate(n_cases, world, ms / steps)
    line = bench.base_line(value, world, steps, 3, ms / steps) if rank == 0 else None
    out[rank] = (ms, value, line, ev.tobytes())
    dist.destroy_process_group()


def test_two_rank_bench_path():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_path, args=(world, _free_port(), out), nprocs=world, join=True)
    ms0, v0, line, ev0 = out[0]
    ms1, v1, none, ev1 = out[1]
    assert ms0 == ms1 >= 3 * 8.0            # the slowest rank's region, on every rank
    assert v0 == v1 == 32 * 2 / (ms0 / 3 / 1e3)
    assert none is None and ev0 != ev1      # one line (rank 0); independent batches
    assert line["n_gpus"] == 2 and line["scaling"] == "weak" and line["value"] == v0
    assert line["metric"] == bench.METRIC and line["ms_per_step"] == ms0 / 3


def test_gpus_flag_spawns_ranks():
    """`bench.py --gpus 2` outside torchrun relaunches itself as two ranks;
    the reference arm (the oracle on the host) needs no GPU, so the whole
    launch runs here: one line, from rank 0, with n_gpus = 2."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--impl", "reference",
                        "--workload", "bn20", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["impl"] == "reference" and d["metric"] == bench.METRIC


def test_reference_arm_without_steps():
    """`bench.py --impl reference` with no --steps picks its own step count
    (as the GPU arm does) and prints one line."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "bn20"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and 3 <= d["steps"] <= 20 and d["value"] > 0

#!/usr/bin/env python3
"""Benchmark: evidence cases/s of batched junction-tree inference on one GB300.

One step = one full inference pass (evidence reduction, collect, distribute,
log P(e) and posterior normalisation for every case) over one batch of the
workload's evidence cases.  Default workload: the 420-variable large-clique
network (cardinality 2..4, 1-4 parents from the previous 14, largest clique
between 4e6 and 1.6e7 entries), 5 % observed, with the batch set to the
largest number of cases one table arena admits under the memory budget;
synthetic and seeded (synth/).

Reported on one JSON line (rank 0):
  value       device-resident throughput (evidence already in HBM), cases/s
  e2e         the same through jt_infer with host buffers (H2D of evidence and
              D2H of results inside the timed region)
  roofline    the dominant kernel's achieved algorithmic GB/s vs measured HBM peak
  plain_gpu   the plain per-case FP64 GPU path on a sample of the same cases
  cpu_baseline the FP64 oracle on the host cores on a bounded sample
  cpu_layer_parallel  context: the paper's own multi-core CPU design
              (jt_infer_cpu: one case at a time, each tree layer one parallel
              loop over its table entries), best thread count of a sweep
  accuracy    sampled outputs of the timed run against the FP64 oracle

``--impl reference`` times the FP64 oracle (the reference arm for this build)
on the host cores instead.  Under torchrun each rank processes its own batch
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "bn60": "bn60_card2-5_B4096_obs10pct",
    "bn20": "bn20_binary_B100_obs20pct",
    "bn110": "bn110_hub60_card2-8_B8192_obs15pct",
    "bn420": "bn420_card2-4_Barena_obs5pct",
    "bn1000": "bn1000_ternary_B4096_obs5-30pct",
}
# cases per step; None = the largest batch one table arena admits under the
# plan's memory budget (the workload's batch is set by admission)
DEFAULT_CASES = {"bn20": 100, "bn60": 4096, "bn110": 8192, "bn420": None, "bn1000": 4096}

# the benchmark's metric, printed identically by both arms
METRIC = "evidence cases/sec at \u22641e-5 posterior error, batched vs plain; p50/p99 latency"


# DRAM traffic of the dominant kernel per launch (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture), valid only for the plan shape
# and kernel source it was taken with: keyed by (workload, cases, the plan's
# distribute work shape, sha256 prefix of csrc/kernels.cu); anything else
# reports null.
MEASURED_TRAFFIC = {
    ("bn420", 896, (768, (0,) * 32, 1), "c144a3405c3ce8c9"): 256720000000 + 25940000000,
    ("bn420", 896, (768, (0,) * 32, 1), "7dbc36f1415f70b1"): 257730000000 + 26180000000,
    ("bn420", 896, (768, (0,) * 32, 1), "a0d3b1563434d06a"): 254860000000 + 23520000000,
    ("bn420", 896, (768, (0,) * 32, 1), "c591329aa84cabcf"): 254850000000 + 23530000000,
    ("bn420", 896, (768, (0,) * 32, 0), "c591329aa84cabcf"): 329970000000 + 24160000000,
}


def _distribute_shape(tuned):
    """The plan options that shape the distribute pass's work lists."""
    items = int(tuned.get("items_per_tile_distribute") or tuned.get("items_per_tile") or 192)
    table = tuple(int(x) for x in (tuned.get("distribute_rows_by_bucket") or (0,) * 32))
    return (items, table, int(tuned.get("fuse_distribute", 1)))


def _kept_columns(net, roots):
    """Posterior columns of the variables a plan pruned to a query set keeps:
    the query and observed sets and their ancestors."""
    keep, stack = set(), list(roots)
    while stack:
        v = stack.pop()
        if v not in keep:
            keep.add(v)
            stack.extend(int(p) for p in net.parents_of(v))
    offs = np.concatenate([[0], np.cumsum(net.card)])
    return np.concatenate([np.arange(offs[v], offs[v + 1]) for v in sorted(keep)])


def _cpu_layers_rate(plan, ev, seconds=1.5):
    """jt_infer_cpu (the paper's design on the host cores) over a sweep of
    thread counts, as the paper picks its best thread count; each count
    runs a bounded sample of the workload's cases."""
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    plan.infer_cpu(ev[:1], threads=cores)
    one = max(time.perf_counter() - t0, 1e-6)
    m = int(max(1, min(len(ev), seconds / one)))
    sweep = {}
    for t in sorted({1, 2, 4, 8, 16, 32, cores}):
        if t > cores or m * one * cores / t > 10.0:   # bound the sweep's host time
            continue
        t0 = time.perf_counter()
        plan.infer_cpu(ev[:m], threads=t)
        sweep[t] = m / (time.perf_counter() - t0)
    best = max(sweep, key=sweep.get)
    return {"value": sweep[best], "unit": "cases/s", "threads": best, "cores": cores,
            "sweep": {str(k): round(v, 2) for k, v in sweep.items()}, "dtype": "f64",
            "sample": f"first {m} cases per thread count"}


def _bucket_table(info):
    """Rows per warp work item used in each table-size bucket (bucket b:
    2^b <= rows < 2^(b+1)) and the share of each pass's rows it holds."""
    out = {}
    for pas in ("collect", "distribute"):
        ent = info[f"{pas}_entries_by_bucket"]
        tot = float(sum(ent)) or 1.0
        out[pas] = {str(b): {"rows_per_item": info[f"{pas}_rows_by_bucket"][b], "share": round(e / tot, 4)}
                    for b, e in enumerate(ent) if e}
    return out


def _kernel_source_hash():
    import hashlib
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2212_04241_gb300", "csrc", "kernels.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_evidence_seed(name: str, rank: int) -> int:
    """Each rank draws its own independent batch of the workload."""
    from synth import configs
    return configs.EVIDENCE_SEED[name] + 1000 * rank


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's timed region (all ranks get the same value)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(cases_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job throughput: the cases of all ranks over the slowest rank's time."""
    return cases_per_rank * world / (ms_per_step / 1e3)


class EventTimer:
    """Device time of the timed region: CUDA events on the launching stream."""

    def __init__(self, stream):
        import torch
        self.stream = stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def start(self):
        self.e0.record(self.stream)

    def stop(self):
        self.e1.record(self.stream)

    def ms(self):
        return self.e0.elapsed_time(self.e1)


class WallTimer:
    """Host wall time (for ranks without a GPU)."""

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()

    def ms(self):
        return 1e3 * (self.t1 - self.t0)


def timed_region(step, steps, dist, device, timer, sync=lambda: None):
    """`steps` calls of step between a barrier and a synchronisation on both
    sides; returns the slowest rank's milliseconds (every rank gets it)."""
    if dist:
        dist.barrier()
    sync()
    timer.start()
    for _ in range(steps):
        step()
    timer.stop()
    sync()
    if dist:
        dist.barrier()
    return max_over_ranks(timer.ms(), dist, device)


def base_line(value, world, steps, warmup, ms_per_step):
    """The keys every line of this arm carries."""
    return {"metric": METRIC, "value": value, "unit": "cases/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic"}


def spawn_ranks(n):
    """--gpus N outside torchrun: relaunch this command as N ranks on this
    node, one GPU each (torch.distributed.run, rendezvous on 127.0.0.1);
    rank 0 prints the line.  Returns the launcher's exit status."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.run(cmd).returncode


def _oracle_rate(net, ev, threads, budget_s):
    """Oracle cases/s on up to len(ev) cases, stopping after ~budget_s."""
    import oracle  # CPU baseline leg only
    o = oracle.Oracle(net)
    done, t0 = 0, time.perf_counter()
    step = max(threads, 1) * 4
    while done < ev.shape[0]:
        o.infer(ev[done:done + step], threads=threads)
        done = min(ev.shape[0], done + step)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


SERVING_PLANS = ["bn60", "bn110", "bn420", "bn1000"]


# resident tiles per plan served with iteration-level batching (as many as
# the pool holds, up to these); a plan absent here is served with batch
# slots.  The rolling tiles stay resident, so that mode gets the larger pool
# (batch slots measured lower latency with 48 GB than with 96 GB: more slots
# in flight put more of the large plans' work in front of the small ones).
ROLLING_TILES = {"bn60": 16, "bn1000": 16, "bn110": 8, "bn420": 6}
SERVING_POOL_GB = 96.0
# batch-slot serving: work items per tile and layer per plan (others: the
# library default) and the plans whose batches run on the high-priority
# streams (jt_server_set_priority)
SERVING_ITEMS = {}
SERVING_HIGH = ()


def run_serving(duration_s: float = 3.0, rates=(0.25, 0.5, 0.9), seed: int = 7, max_batch: int = 64,
                arena_gb: float = SERVING_POOL_GB, schedule=None, min_requests: int = 20000, rolling: bool = False,
                items_per_tile: dict = None, high_priority=None):
    """The serving mix: resident plans of the four networks, one-case requests
    on a uniformly chosen plan with 5-30 % observed, Poisson arrivals at
    fractions of the measured saturated rate.  Returns p50/p99 latency
    (submit -> result on the host) and cases/s per offered rate, overall and
    per plan.  rolling: the plans of ROLLING_TILES are served with
    iteration-level batching (resident tiles that advance one tree layer per
    tick; requests join at the next tick), the others with batch slots."""
    import paper_2212_04241_gb300.jt as J
    from synth import configs
    from synth.bn import sample_cases
    rng = np.random.default_rng(seed)
    nets = [configs.network(nm) for nm in SERVING_PLANS]
    # small batches: 32-case tiles; many plans share the GPU, so each pass
    # runs layer by layer (a persistent dataflow pass would hold every SM
    # until it ends and queue the other plans' short passes behind it)
    sched = J.JT_SCHEDULE_LAYERS if schedule is None else schedule
    items_per_tile = SERVING_ITEMS if items_per_tile is None else items_per_tile
    high_priority = SERVING_HIGH if high_priority is None else high_priority
    plans = [J.Plan(n, cases_per_thread=1, schedule=sched, items_per_tile=items_per_tile.get(nm, 0))
             for nm, n in zip(SERVING_PLANS, nets)]
    pool = [sample_cases(n, 2048, (0.05, 0.30), seed + i) for i, n in enumerate(nets)]

    def drive(srv, pids, n_req, rate):
        """Submit n_req requests (Poisson at `rate`/s, or all at once if rate
        is None), wait for all, return wall seconds."""
        which = rng.integers(0, len(plans), size=n_req)
        rows = rng.integers(0, 2048, size=n_req)
        gaps = rng.exponential(1.0 / rate, size=n_req) if rate else np.zeros(n_req)
        tickets = []
        t0 = time.perf_counter()
        t_next = t0
        for i in range(n_req):
            t_next += gaps[i]
            while rate and time.perf_counter() < t_next:
                pass
            p = int(which[i])
            tickets.append((srv.submit(pids[p], pool[p][rows[i]]), plans[p].sum_card))
        srv.drain()
        dt = time.perf_counter() - t0
        for t, m in tickets:
            r = srv.poll(t, m)
            assert r is not None
        return dt

    def fresh():
        srv = J.Server(arena_bytes=int(arena_gb * (1 << 30)), max_batch=max_batch, max_inflight=8)
        if not rolling:
            pids = [srv.add_plan(pl) for pl in plans]
            for nm, pid in zip(SERVING_PLANS, pids):
                if nm in high_priority:
                    srv.set_priority(pid, True)
            return srv, pids
        pids = [None] * len(plans)
        for i, nm in enumerate(SERVING_PLANS):   # the small plans first
            if nm not in ROLLING_TILES:
                continue
            for t in range(ROLLING_TILES[nm], 0, -1):   # as many tiles as the pool holds
                try:
                    pids[i] = srv.add_plan(plans[i], rolling_tiles=t)
                    tiles_used[nm] = t
                    break
                except J.JTError:
                    continue
            if pids[i] is None:
                raise RuntimeError(f"rolling plan {nm} does not fit the pool")
        for i, nm in enumerate(SERVING_PLANS):
            if pids[i] is None:
                pids[i] = srv.add_plan(plans[i])
        return srv, pids

    tiles_used = {}

    srv, pids = fresh()
    drive(srv, pids, 2000, None)  # warm-up: slots, graphs
    n_sat = 20000
    sat = n_sat / drive(srv, pids, n_sat, None)
    srv.close()
    out = {"plans": SERVING_PLANS, "arena_gb": arena_gb, "max_batch": max_batch,
           "mode": ("rolling tiles (iteration-level batching) for " + ", ".join(sorted(ROLLING_TILES)) +
                    (", batch slots for the others" if set(ROLLING_TILES) != set(SERVING_PLANS) else ""))
           if rolling else "batch slots",
           "items_per_tile": dict(items_per_tile) or None,
           "high_priority": list(high_priority) or None,
           "saturated_cases_per_s": sat, "rates": []}
    if rolling:
        out["tiles"] = dict(tiles_used)
        out["tile_cases"] = {nm: int(pl.info()["tile_cases"]) for nm, pl in zip(SERVING_PLANS, plans)}
    if set(ROLLING_TILES) != set(SERVING_PLANS) or not rolling:
        out["schedule"] = "layers" if sched == J.JT_SCHEDULE_LAYERS else "dataflow"
    for f in rates:
        rate = f * sat
        n_req = int(max(min_requests, min(200000, rate * duration_s)))
        srv, pids = fresh()
        drive(srv, pids, 500, None)     # warm-up on this server: slots bound, graphs captured
        srv.reset_latency()
        st0 = srv.stats()
        dt = drive(srv, pids, n_req, rate)
        st = srv.stats()
        per_plan = {}
        for nm, pid in zip(SERVING_PLANS, pids):
            ps = srv.plan_stats(pid)
            per_plan[nm] = {"completed": ps["completed"], "p50_ms": ps["p50_ns"] / 1e6, "p99_ms": ps["p99_ns"] / 1e6}
        srv.close()
        out["rates"].append({"offered_fraction": f, "offered_cases_per_s": rate, "requests": n_req,
                             "achieved_cases_per_s": n_req / dt, "p50_ms": st["p50_ns"] / 1e6,
                             "p99_ms": st["p99_ns"] / 1e6, "batches": st["batches"] - st0["batches"],
                             "largest_batch": st["largest_batch"],
                             "peak_arena_gb": st["peak_arena_bytes"] / 2**30,
                             "slot_creations": st["slot_creations"] - st0["slot_creations"],
                             "slot_evictions": st["slot_evictions"] - st0["slot_evictions"],
                             "per_plan": per_plan})
    return out


def run_reference(args, name, net, ev, rank, world):
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    import oracle
    o = oracle.Oracle(net)
    # one step = a bounded sample of the workload on all host cores: one case
    # per core, or more while a step stays near a second
    t0 = time.perf_counter()
    o.infer(ev[:cores], threads=cores)
    t_one = max(time.perf_counter() - t0, 1e-6)
    per_step = int(min(ev.shape[0], cores * max(1, min(8, int(1.0 / t_one)))))
    t_step = t_one
    for i in range(args.warmup):
        t0 = time.perf_counter()
        o.infer(ev[:per_step], threads=cores)
        t_step = time.perf_counter() - t0
    # no --steps: as many steps as fill about ten seconds (3 to 20)
    steps = args.steps if args.steps > 0 else max(3, min(20, int(10.0 / max(t_step, 1e-3))))
    times = []
    for i in range(steps):
        sl = ev[(i * per_step) % ev.shape[0]:][:per_step]
        t0 = time.perf_counter()
        o.infer(sl, threads=cores)
        times.append(time.perf_counter() - t0)
    total = max(float(np.sum(times)), 1e-9)
    value = per_step * steps / total
    line = {"metric": METRIC, "value": value,
            "unit": "cases/s", "impl": "reference", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[name], "cases_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "cases/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} cases of the workload per step"},
            "e2e": {"value": value, "unit": "cases/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps; default: as many as fill about 2 s")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bn420", choices=sorted(WORKLOADS))
    ap.add_argument("--cases", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-layers", action="store_true",
                    help="skip the multi-core CPU comparator in the paper's layer-parallel style")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-mix latency measurement")
    ap.add_argument("--no-autotune", action="store_true", help="default plan options instead of jt_autotune")
    ap.add_argument("--observed-set", type=int, default=0,
                    help="K > 0: every case observes the same K variables (seeded choice, states from an "
                    "ancestral sample) and the plan is specialised to that set")
    ap.add_argument("--query-set", type=int, default=0,
                    help="Q > 0 (with --observed-set): the plan is also pruned to Q query variables (seeded choice "
                    "outside the observed set); the barren variables are removed")
    ap.add_argument("--plan", default="", help="fixed plan options as JSON (e.g. '{\"items_per_tile\": 96}'), "
                    "instead of jt_autotune")
    ap.add_argument("--serving-only", action="store_true", help="only the serving-mix measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return spawn_ranks(args.gpus)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    from synth import configs
    name = args.workload
    net = configs.network(name)
    arena_sized = not args.cases and DEFAULT_CASES[name] is None
    observed_set = None
    if args.observed_set > 0:
        # a fixed observed set shared by every case (its states vary per case)
        rng = np.random.default_rng(1234)
        observed_set = sorted(int(v) for v in rng.choice(net.n, size=args.observed_set, replace=False))
    query_set = None
    if args.query_set > 0:
        if not observed_set:
            raise SystemExit("--query-set needs --observed-set")
        rng = np.random.default_rng(4321)
        rest = [v for v in range(net.n) if v not in observed_set]
        query_set = sorted(int(v) for v in rng.choice(rest, size=args.query_set, replace=False))

    def make_evidence(n):
        """This rank's own independent batch of n cases (weak scaling)."""
        if observed_set:
            from synth.bn import sample_cases
            x = sample_cases(net, n, 1.0, seed=rank_evidence_seed(name, rank))
            e = np.full_like(x, -1, dtype=np.int32)
            e[:, observed_set] = x[:, observed_set]
            return e
        return configs.evidence(name, net, n_cases=n, seed=rank_evidence_seed(name, rank))

    if args.impl == "reference":
        # the oracle runs bounded samples of the workload; an arena-sized
        # batch needs a GPU plan to size it, so the sample pool is 1024 cases
        return run_reference(args, name, net, make_evidence(args.cases or DEFAULT_CASES[name] or 1024), rank, world)

    import torch
    if args.serving_only:
        print(json.dumps({"serving": {"batch_slots": run_serving(arena_gb=48.0), "rolling": run_serving(rolling=True)}}),
              flush=True)
        return 0
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    import paper_2212_04241_gb300.jt as J
    spec = {"observed_set": observed_set} if observed_set else {}
    if query_set:
        spec["query_set"] = query_set
    fixed = dict(json.loads(args.plan), **spec) if args.plan else None
    if arena_sized:
        # the batch is what one table arena admits under the memory budget
        probe = J.Plan(net, **(fixed or spec))
        n_cases = probe.info()["budget_chunk_cases"]
        probe.close()
    else:
        n_cases = args.cases or DEFAULT_CASES[name]
    # the library's autotuner picks the work shape for this network and batch
    if fixed is not None:
        tuned = fixed
    else:
        tuned, _ = J.autotune(net, n_cases, **spec) if not args.no_autotune else (dict(spec), None)
    plan = J.Plan(net, **tuned)
    if arena_sized:
        # the tuned tile width may admit a different batch: take its own
        n_cases = plan.info()["budget_chunk_cases"]
    ev = make_evidence(n_cases)
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    d_ev = torch.from_numpy(ev).cuda()
    d_lp = torch.empty(n_cases, dtype=torch.float64, device="cuda")
    d_post = torch.empty((n_cases, plan.sum_card), dtype=torch.float64, device="cuda")
    d_st = torch.empty(n_cases, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step():
        plan.infer_device(d_ev, d_lp, d_post, d_st, stream=sptr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = plan.info()
    if args.steps <= 0:
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        one = max(time.perf_counter() - t0, 1e-5)
        args.steps = int(min(5000, max(10, 2.0 / one)))

    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.5)  # let the sampler start before the timed region
    ms = timed_region(step, args.steps, dist, "cuda", EventTimer(stream), torch.cuda.synchronize)
    clock_info = clocks.stop()
    ms_per_step = ms / args.steps
    value = aggregate_rate(n_cases, world, ms_per_step)

    # accuracy of the timed run's outputs on a seeded sample (oracle)
    lp = d_lp.cpu().numpy()
    post = d_post.cpu().numpy()
    st = d_st.cpu().numpy()
    accuracy = None
    if rank == 0:
        import oracle
        idx = np.random.default_rng(0).choice(n_cases, size=min(64, n_cases), replace=False)
        olp, opost, ost = oracle.Oracle(net).infer(ev[idx], threads=os.cpu_count() or 1)
        ok = ost == 0
        cols = _kept_columns(net, query_set + observed_set) if query_set else np.arange(plan.sum_card)
        accuracy = {
            "sample_cases": int(len(idx)),
            "max_abs_posterior_err": float(np.max(np.abs(post[idx][ok][:, cols] - opost[ok][:, cols]))),
            "max_rel_logpe_err": float(np.max(np.abs(lp[idx][ok] - olp[ok]) / np.maximum(1, np.abs(olp[ok])))),
            "status_match": bool(np.array_equal(st[idx], ost)),
        }
        accuracy["pass"] = bool(accuracy["max_abs_posterior_err"] <= 1e-5 and
                                accuracy["max_rel_logpe_err"] <= 1e-6 and accuracy["status_match"])

    # per-kernel device time (instrumented pass, events around each layer launch)
    prof = plan.profile(d_ev, d_lp, d_post, d_st, stream=sptr)
    kinds = {"collect": prof["collect_ms"], "distribute": prof["distribute_ms"]}
    dom = max(kinds, key=kinds.get)
    # algorithmic bytes of one pass per kernel kind (per case):
    #   collect:    psi written 4|C|, messages written 4|S| and read 4|S|
    #   distribute: psi read 4|C|, ratios written 4|S| and read 4|S|
    # with recomputed clique tables no psi moves: collect writes and the
    # parent reads the messages (8|S|); distribute reads the child messages
    # once more (4|S|) and writes and reads the ratios (8|S|)
    recompute = bool(int(tuned.get("recompute_psi", 0))) and not observed_set
    C, S = float(info["sum_clique_entries"]), float(info["sum_sep_entries"])
    per_case_kind = ({"collect": 8.0 * S, "distribute": 12.0 * S} if recompute else
                     {"collect": 4.0 * C + 8.0 * S, "distribute": 4.0 * C + 8.0 * S})
    bytes_dom = per_case_kind[dom] * n_cases
    achieved = bytes_dom / (kinds[dom] / 1e3) / 1e9
    other = "collect" if dom == "distribute" else "distribute"
    other_frac = per_case_kind[other] * n_cases / (kinds[other] / 1e3)
    peak, peak_src = _peaks()
    dataflow = int(tuned.get("schedule", J.JT_SCHEDULE_DATAFLOW)) == J.JT_SCHEDULE_DATAFLOW
    kernel = f"k_{dom}_flow" if dataflow else f"k_{dom}"
    ksha = _kernel_source_hash()
    traffic = (MEASURED_TRAFFIC.get((name, n_cases, _distribute_shape(tuned), ksha))
               if dataflow and dom == "distribute" and not observed_set else None)
    roofline = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "traffic_source": (f"stored ncu capture (dram__bytes_read.sum + dram__bytes_write.sum per launch), "
                                   f"kernel source sha256 {ksha}" if traffic is not None else
                                   f"no stored ncu capture for kernel source sha256 {ksha} and this plan shape"),
                "launches": prof[f"{dom}_launches"],
                "kernel_ms_per_pass": kinds[dom], "other_kernel_ms_per_pass": kinds[other],
                "algorithmic_bytes_per_case": per_case_kind[dom],
                "tables": "recomputed in the distribute pass" if recompute else "stored by the collect pass",
                "other_kernel": (f"k_{other}_flow" if dataflow else f"k_{other}"),
                "other_kernel_frac": other_frac / 1e9 / peak,
                "whole_pass_algorithmic_GBps": info["algorithmic_bytes_per_case"] * n_cases / (prof["total_ms"] / 1e3) / 1e9}

    # end to end through jt_infer with host buffers
    e2e = None
    if rank == 0:
        import torch as _t
        # page-locked host buffers (allocated once, outside the timed region):
        # every step copies the evidence in and all outputs back
        ev_pinned = _t.from_numpy(ev).pin_memory().numpy()
        out = (_t.empty(n_cases, dtype=_t.float64, pin_memory=True).numpy(),
               _t.empty((n_cases, plan.sum_card), dtype=_t.float64, pin_memory=True).numpy(),
               _t.empty(n_cases, dtype=_t.int32, pin_memory=True).numpy())
        for _ in range(3):
            plan.infer(ev_pinned, out=out)
        times = []
        for _ in range(10):                  # median of 10 synchronous calls
            t0 = time.perf_counter()
            plan.infer(ev_pinned, out=out)
            times.append(time.perf_counter() - t0)
        dt = float(np.median(times))
        e2e = {"value": n_cases / dt, "unit": "cases/s", "h2d_bytes_per_step": int(ev.nbytes),
               "d2h_bytes_per_step": int(n_cases * (8 + 8 * plan.sum_card + 4)), "ms_per_step": dt * 1e3,
               "timing": "median of 10 synchronous calls after 3 warm-up calls"}

    plain = None
    if rank == 0 and not args.no_plain and not observed_set:
        m = min(n_cases, 64 if name in ("bn20", "bn60", "bn1000") else 8)
        plan.infer_plain(ev[:2])
        t0 = time.perf_counter()
        plan.infer_plain(ev[:m])
        dt = time.perf_counter() - t0
        plain = {"value": m / dt, "unit": "cases/s", "sample": f"first {m} cases", "dtype": "f64",
                 "batched_over_plain": value / world / (m / dt)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, done, dt = _oracle_rate(net, ev, cores, 15.0)
        rate1, done1, dt1 = _oracle_rate(net, ev, 1, 4.0)
        cpu = {"value": rate, "unit": "cases/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} cases of the workload in {dt:.1f} s",
               "one_thread": {"value": rate1, "sample": f"{done1} cases in {dt1:.1f} s, one case at a time"}}

    cpu_layers = None
    if rank == 0 and not args.no_cpu_layers and not observed_set:
        cpu_layers = _cpu_layers_rate(plan, ev)

    # the batch's table arena is released before the serving pools are made
    plan.close()
    serving = None
    if rank == 0 and not args.no_serving and world == 1:
        serving = {"batch_slots": run_serving(arena_gb=48.0), "rolling": run_serving(rolling=True)}

    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    launches = info["kernels_per_chunk"] * ((n_cases + info["chunk_cases"] - 1) // max(1, info["chunk_cases"]))
    line = dict(base_line(value, world, args.steps, args.warmup, ms_per_step), **{
        "config": {"workload": WORKLOADS[name] + (f"_observedset{args.observed_set}" if observed_set else "")
                   + (f"_queryset{args.query_set}" if query_set else ""),
                   "observed_set": observed_set, "query_set": query_set, "pruned_vars": info["pruned_vars"], "cases_per_gpu": n_cases, "tile_cases": info["tile_cases"],
                   "batch": ("arena-admitted: the cases one table arena holds under the automatic budget "
                             "(min(224 GiB, 70% of free device memory))" if arena_sized else "fixed"),
                   "arena_gb": info["arena_bytes"] / 1e9,
                   "chunk_cases": info["chunk_cases"], "levels": info["n_levels"],
                   "autotuned": ({k: tuned.get(k) for k in ("cases_per_thread", "items_per_tile", "items_per_tile_distribute")}
                                 if tuned and not args.plan and not args.no_autotune else None),
                   "work_shape_by_bucket": _bucket_table(info),
                   "plan_options": tuned if args.plan else None,
                   # the plan's options as used (replayable with --plan)
                   "tuned_options": {k: v for k, v in tuned.items() if k not in ("observed_set", "query_set")},
                   "schedule": "dataflow" if dataflow else "layers",
                   "sum_clique_entries": info["sum_clique_entries"],
                   "l2": "inputs larger than L2 (psi arena %.2f GB per step)" % (4.0 * info["sum_clique_entries"] * n_cases / 1e9),
                   "parallelism": f"cases sharded, {world} rank(s)"},
        "gpu_launches": int(launches * args.steps),
        "roofline": roofline, "clocks": clock_info, "e2e": e2e, "plain_gpu": plain,
        "cpu_baseline": cpu, "cpu_layer_parallel": cpu_layers, "accuracy": accuracy, "serving": serving,
    })
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

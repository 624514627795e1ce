"""Parity of the work shapes the benchmark times (GPU, through the C ABI).

jt_autotune picks a tile width and, per table-size bucket, the rows of one
warp work item for each pass.  These tests run the tuned plans of the
110-variable hub network and of the 420-variable large-clique network at
their arena-admitted batch sizes -- the shapes the benchmark times -- and
compare sampled cases with the FP64 oracle; every case of the batch is
checked for properties that hold at any size (status, normalised
posteriors, point masses).  Explicit bucket tables at the extremes of the
tuner's range are checked against the oracle too.
"""
import os

import numpy as np
import pytest

import oracle
from synth import configs
from tests.common import assert_parity32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402


def _run_device(plan, ev):
    n = ev.shape[0]
    d_ev = torch.from_numpy(ev).cuda()
    out = (torch.empty(n, dtype=torch.float64, device="cuda"),
           torch.empty((n, plan.sum_card), dtype=torch.float64, device="cuda"),
           torch.empty(n, dtype=torch.int32, device="cuda"))
    plan.infer_device(d_ev, *out, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


def _check_whole_batch(net, ev, lp, post, st):
    assert np.all(st == 0), "every sampled case has P(e) > 0"
    assert np.all(np.isfinite(lp)) and np.all(lp <= 1e-9)
    offs = np.concatenate([[0], np.cumsum(net.card)])
    for v in range(net.n):
        s = post[:, offs[v]:offs[v + 1]].sum(axis=1)
        assert np.max(np.abs(s - 1.0)) <= 1e-9, f"variable {v} not normalised"
        obs = ev[:, v] >= 0
        if obs.any():
            assert np.all(post[obs, offs[v] + ev[obs, v]] == 1.0)


@pytest.mark.parametrize("name,sample", [("bn110", 48), ("bn420", 16)])
def test_autotuned_plan_at_arena_batch(name, sample):
    net = configs.network(name)
    probe = J.Plan(net)
    n = probe.info()["budget_chunk_cases"]
    probe.close()
    n = min(n, 2432)                       # one arena chunk (bn110: the 19-tile chunk)
    tuned, ns = J.autotune(net, n)
    assert ns > 0
    plan = J.Plan(net, **tuned)
    info = plan.info()
    n = min(n, info["budget_chunk_cases"])
    ev = configs.evidence(name, net, n_cases=n, seed=777)
    lp, post, st = _run_device(plan, ev)
    _check_whole_batch(net, ev, lp, post, st)
    idx = np.random.default_rng(3).choice(n, size=min(sample, n), replace=False)
    olp, opost, ost = oracle.Oracle(net).infer(ev[idx], threads=os.cpu_count() or 1)
    assert_parity32(lp[idx], post[idx], st[idx], olp, opost, ost, where=f"{name} autotuned {tuned}")


@pytest.mark.parametrize("rows", [32, 4096])
def test_explicit_bucket_tables(rows):
    """Every bucket's items at one extreme of the tuner's range."""
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=1000)
    table = [rows] * J.JT_SIZE_BUCKETS
    plan = J.Plan(net, collect_rows_by_bucket=table, distribute_rows_by_bucket=table)
    info = plan.info()
    used = [r for r, e in zip(info["collect_rows_by_bucket"], info["collect_entries_by_bucket"]) if e]
    assert used and all(r == rows for r in used)
    lp, post, st = _run_device(plan, ev)
    olp, opost, ost = oracle.Oracle(net).infer(ev, threads=os.cpu_count() or 1)
    assert_parity32(lp, post, st, olp, opost, ost, where=f"bucket rows {rows}")

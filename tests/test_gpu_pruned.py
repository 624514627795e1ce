"""Plans pruned to a query set (GPU, through the C ABI).

A plan compiled with a query set Q keeps Q, the observed set O and their
ancestors; every other variable is barren (summing it out of its CPT gives
exactly 1) and is removed before the tree is built.  P(e) and the posterior
of every kept variable must equal the oracle's, computed on the FULL
network; the columns of removed variables are NaN; a case observing a
removed variable is flagged alone.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import sample_cases, tiny_random_network
from tests.common import assert_parity32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402


def _closure(net, roots):
    keep, stack = set(), list(roots)
    while stack:
        v = stack.pop()
        if v not in keep:
            keep.add(v)
            stack.extend(int(p) for p in net.parents_of(v))
    return sorted(keep)


def _columns(net, vars_):
    offs = np.concatenate([[0], np.cumsum(net.card)])
    return np.concatenate([np.arange(offs[v], offs[v + 1]) for v in vars_]) if vars_ else np.zeros(0, int)


def _cases(net, n_cases, keep, obs, extra, seed):
    """Ancestral samples observing every variable of obs and, with
    probability extra, each other kept variable; nothing else."""
    rng = np.random.default_rng(seed)
    x = sample_cases(net, n_cases, 1.0, seed=seed + 1)
    ev = np.full_like(x, -1)
    ev[:, obs] = x[:, obs]
    more = np.zeros_like(x, dtype=bool)
    more[:, keep] = rng.random((n_cases, len(keep))) < extra
    ev[more] = x[more]
    return ev.astype(np.int32)


def _check(net, plan, ev, keep, where, n_oracle=40):
    lp, post, st = plan.infer(ev)
    dropped = [v for v in range(net.n) if v not in set(keep)]
    assert np.all(np.isnan(post[:, _columns(net, dropped)]))
    kc = _columns(net, keep)
    idx = np.arange(0, len(ev), max(1, len(ev) // n_oracle))
    olp, opost, ost = oracle.Oracle(net).infer(ev[idx], threads=16)
    assert_parity32(lp[idx], post[idx][:, kc], st[idx], olp, opost[:, kc], ost, where=where)
    return lp, post, st


@pytest.mark.parametrize("name,q,n_obs,extra,n_cases", [("bn60", [41, 50], 6, 0.0, 700),
                                                        ("bn60", [59], 12, 0.1, 500),
                                                        ("bn1000", [10, 500, 990], 40, 0.1, 600),
                                                        ("bn110", [100, 60], 8, 0.05, 130)])
@pytest.mark.parametrize("schedule", [J.JT_SCHEDULE_DATAFLOW, J.JT_SCHEDULE_LAYERS])
def test_pruned_and_sliced_plan_matches_full_network_oracle(name, q, n_obs, extra, n_cases, schedule):
    net = configs.network(name)
    rng = np.random.default_rng(len(q) + n_obs)
    obs = sorted(int(v) for v in rng.choice([v for v in range(net.n) if v not in q], size=n_obs, replace=False))
    keep = _closure(net, q + obs)
    ev = _cases(net, n_cases, keep, obs, extra, seed=11)
    plan = J.Plan(net, query_set=q, observed_set=obs, schedule=schedule)
    assert plan.info()["pruned_vars"] == net.n - len(keep) > 0
    _check(net, plan, ev, keep, f"{name} pruned+sliced")


@pytest.mark.parametrize("name,q", [("bn60", [30, 45, 57]), ("bn1000", [999, 400])])
def test_pruned_plan_without_observed_set(name, q):
    """Evidence on any kept variables, different per case."""
    net = configs.network(name)
    keep = _closure(net, q)
    ev = _cases(net, 300, keep, [], 0.3, seed=5)
    plan = J.Plan(net, query_set=q)
    _check(net, plan, ev, keep, f"{name} pruned")
    # device path and host path agree bit for bit
    d_ev = torch.from_numpy(ev).cuda()
    d_lp = torch.empty(len(ev), dtype=torch.float64, device="cuda")
    d_post = torch.empty((len(ev), plan.sum_card), dtype=torch.float64, device="cuda")
    d_st = torch.empty(len(ev), dtype=torch.int32, device="cuda")
    plan.infer_device(d_ev, d_lp, d_post, d_st, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    lp, post, st = plan.infer(ev)
    assert np.array_equal(lp, d_lp.cpu().numpy()) and np.array_equal(st, d_st.cpu().numpy())
    assert np.array_equal(post, d_post.cpu().numpy(), equal_nan=True)


@pytest.mark.parametrize("seed", range(10))
def test_pruned_tiny_networks(seed):
    net = tiny_random_network(seed)
    q = [net.n - 1]
    keep = _closure(net, q)
    ev = _cases(net, 40, keep, [], 0.4, seed=seed)
    _check(net, J.Plan(net, query_set=q, cases_per_thread=1), ev, keep, f"tiny {seed} pruned")


def test_observing_a_removed_variable_flags_that_case():
    net = configs.network("bn60")
    q = [41, 50]
    keep = _closure(net, q)
    dropped = [v for v in range(net.n) if v not in set(keep)]
    ev = _cases(net, 200, keep, [], 0.2, seed=2)
    ev[9, dropped[0]] = 0
    lp, post, st = J.Plan(net, query_set=q).infer(ev)
    assert st[9] == J.JT_CASE_BAD_EVIDENCE and np.isnan(lp[9])
    assert np.all(st[np.arange(200) != 9] == 0)


def test_pruned_plans_refused_by_other_paths():
    net = configs.network("bn20")
    p = J.Plan(net, query_set=[3])
    ev = np.full((1, net.n), -1, dtype=np.int32)
    for call in (p.infer_plain, p.infer_cpu):
        with pytest.raises(J.JTError) as e:
            call(ev)
        assert e.value.status == J.JT_EINVAL
    srv = J.Server(arena_bytes=1 << 28, max_batch=8)
    with pytest.raises(J.JTError) as e:
        srv.add_plan(p)
    assert e.value.status == J.JT_EINVAL


def test_autotune_and_profile_on_pruned_plan():
    net = configs.network("bn60")
    q, obs = [41, 50], [3, 17]
    opts, ns = J.autotune(net, 512, query_set=q, observed_set=obs)
    assert opts["query_set"] == q and opts["observed_set"] == obs and ns > 0
    plan = J.Plan(net, **opts)
    keep = _closure(net, q + obs)
    ev = _cases(net, 512, keep, obs, 0.1, seed=4)
    _check(net, plan, ev, keep, "autotuned pruned plan")
    d_ev = torch.from_numpy(ev).cuda()
    d_lp = torch.empty(len(ev), dtype=torch.float64, device="cuda")
    d_post = torch.empty((len(ev), plan.sum_card), dtype=torch.float64, device="cuda")
    d_st = torch.empty(len(ev), dtype=torch.int32, device="cuda")
    prof = plan.profile(d_ev, d_lp, d_post, d_st, stream=torch.cuda.current_stream().cuda_stream)
    assert prof["collect_launches"] >= 1 and prof["total_ms"] > 0
    lp, post, st = plan.infer(ev)
    assert np.array_equal(st, d_st.cpu().numpy()) and np.array_equal(lp, d_lp.cpu().numpy())
    assert np.array_equal(post, d_post.cpu().numpy(), equal_nan=True)

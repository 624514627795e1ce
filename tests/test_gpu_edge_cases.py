"""GPU edge cases of the batched FP32 path (through the C ABI), checked
against closed forms computed here from the network's CPTs -- independent of
the oracle -- and against the oracle where no closed form exists:

* a network of one variable (P(e) is a prior entry, the posterior the prior);
* every variable observed (log P(e) is the sum of the logs of the CPT
  entries selected by the assignment: Section 1's query at a full
  assignment);
* independent variables (every variable its own component tree: log P(e)
  sums the observed priors, posteriors are priors);
* a deep chain (hundreds of tree layers, exercising the layer order of both
  schedules and the power-of-two rescaling against forward-backward);
* the largest variable cardinality and the largest clique the workloads have.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import make_network, sample_cases
from tests.common import LOGPE_REL32, POST_TOL32, assert_parity32, max_logpe_err
from tests.refsolvers import chain_forward_backward

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402

SCHEDULES = [J.JT_SCHEDULE_DATAFLOW, J.JT_SCHEDULE_LAYERS]


def _prior_marginals(net):
    """Exact marginals of a network whose variables have no parents."""
    return [net.cpt_of(v).reshape(-1) for v in range(net.n)]


@pytest.mark.parametrize("card", [2, 5, 60])
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_single_variable_network(card, schedule):
    net = make_network(1, [card], [[]], 1.0, np.random.default_rng(card))
    prior = net.cpt_of(0).reshape(-1)
    ev = np.array([[-1]] + [[s] for s in range(card)], dtype=np.int32)
    lp, post, st = J.Plan(net, schedule=schedule).infer(ev)
    assert np.all(st == 0)
    assert abs(lp[0]) <= 1e-6 and np.max(np.abs(post[0] - prior)) <= POST_TOL32
    for s in range(card):
        assert abs(lp[1 + s] - np.log(prior[s])) <= LOGPE_REL32 * max(1.0, abs(np.log(prior[s])))
        assert post[1 + s][s] == 1.0 and np.sum(post[1 + s]) == 1.0


@pytest.mark.parametrize("name,n_cases", [("bn20", 100), ("bn60", 500), ("bn1000", 200)])
@pytest.mark.parametrize("schedule", SCHEDULES)
def test_every_variable_observed(name, n_cases, schedule):
    """log P(x) = sum_v log P(x_v | x_pa(v)) for a full assignment x."""
    net = configs.network(name)
    x = sample_cases(net, n_cases, 1.0, seed=31)          # every variable observed
    assert np.all(x >= 0)
    expect = np.zeros(n_cases)
    for v in range(net.n):
        table = net.cpt_of(v)
        pa = [int(p) for p in net.parents_of(v)]
        idx = tuple(x[:, p] for p in pa) + (x[:, v],)
        expect += np.log(table[idx])
    lp, post, st = J.Plan(net, schedule=schedule).infer(x)
    assert np.all(st == 0)
    assert max_logpe_err(lp, expect) <= LOGPE_REL32
    offs = np.concatenate([[0], np.cumsum(net.card)])
    for v in range(net.n):     # point masses
        assert np.array_equal(post[np.arange(n_cases), offs[v] + x[:, v]], np.ones(n_cases))
    assert np.allclose(post.sum(axis=1), net.n)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_independent_variables(schedule):
    rng = np.random.default_rng(5)
    n = 64
    card = rng.integers(2, 7, size=n).tolist()
    net = make_network(n, card, [[] for _ in range(n)], 1.0, rng)
    ev = sample_cases(net, 300, (0.0, 0.5), seed=9)
    pri = _prior_marginals(net)
    lp, post, st = J.Plan(net, schedule=schedule).infer(ev)
    assert np.all(st == 0)
    expect = np.array([sum(np.log(pri[v][e[v]]) for v in range(n) if e[v] >= 0) for e in ev])
    assert max_logpe_err(lp, expect) <= LOGPE_REL32
    offs = np.concatenate([[0], np.cumsum(card)])
    for i, e in enumerate(ev):
        for v in range(n):
            got = post[i, offs[v]:offs[v + 1]]
            want = np.eye(card[v])[e[v]] if e[v] >= 0 else pri[v]
            assert np.max(np.abs(got - want)) <= POST_TOL32


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_deep_chain_against_forward_backward(schedule):
    """A 400-variable chain: a tree of ~200 layers from the centre root (~400
    from the largest); with 90 % of the variables observed P(e) is far below
    FP32's smallest normal, so only the per-message rescaling keeps it."""
    rng = np.random.default_rng(11)
    n, r = 400, 3
    net = make_network(n, [r] * n, [[]] + [[v - 1] for v in range(1, n)], 1.0, rng)
    pi = net.cpt_of(0).reshape(-1)
    T = [net.cpt_of(v) for v in range(1, n)]
    ev = sample_cases(net, 64, 0.9, seed=3)
    for root_rule in (J.JT_ROOT_MIN_HEIGHT, J.JT_ROOT_LARGEST):
        p = J.Plan(net, schedule=schedule, root_rule=root_rule)
        lp, post, st = p.infer(ev)
        assert np.all(st == 0)
        for i, e in enumerate(ev):
            flp, marg = chain_forward_backward(pi, T, e)
            assert lp[i] < -100.0     # far below FP32's smallest normal in linear scale
            assert abs(lp[i] - flp) <= LOGPE_REL32 * max(1.0, abs(flp)), (i, lp[i], flp)
            got = post[i].reshape(n, r)
            assert np.max(np.abs(got - np.stack(marg))) <= POST_TOL32


def _least_likely_chain_evidence(net, n):
    """Every variable of a chain observed, each in the state its CPT row
    (given the previous variable's state) makes least likely."""
    x = np.zeros(n, dtype=np.int32)
    x[0] = int(np.argmin(net.cpt_of(0).reshape(-1)))
    for v in range(1, n):
        x[v] = int(np.argmin(net.cpt_of(v)[x[v - 1]]))
    return x


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_rescaling_keeps_fp32_in_range(schedule):
    """rescale=1 (default) against rescale=0 on a 400-variable chain whose
    every variable is observed in its least likely state: log P(e) (a sum of
    logs of CPT entries, Section 1's query at a full assignment) is far below
    FP32's smallest subnormal (about -103 in natural log) even after each
    clique's base table is scaled to a maximum in [1, 2), so unscaled
    messages lose the case while scaled ones reproduce the closed form."""
    rng = np.random.default_rng(23)
    n, r = 400, 3
    net = make_network(n, [r] * n, [[]] + [[v - 1] for v in range(1, n)], 1.0, rng)
    x = _least_likely_chain_evidence(net, n)
    expect = np.log(net.cpt_of(0).reshape(-1)[x[0]]) + sum(np.log(net.cpt_of(v)[x[v - 1], x[v]]) for v in range(1, n))
    # upper bound of the unscaled root total: each clique's factor is at most
    # 2 x (entry / row maximum) once its base table is scaled into [1, 2)
    bound = np.log(2.0 * net.cpt_of(0).reshape(-1)[x[0]] / net.cpt_of(0).max())
    bound += sum(np.log(2.0 * net.cpt_of(v)[x[v - 1], x[v]] / net.cpt_of(v).max()) for v in range(1, n))
    assert bound < -200.0
    ev = np.stack([x, x])
    lp, post, st = J.Plan(net, schedule=schedule).infer(ev)
    assert np.all(st == J.JT_CASE_OK)
    assert np.all(np.abs(lp - expect) <= LOGPE_REL32 * abs(expect))
    lp0, _, st0 = J.Plan(net, schedule=schedule, rescale=0).infer(ev)
    lost = (st0 == J.JT_CASE_ZERO_EVIDENCE) | (np.abs(lp0 - expect) > 1.0)
    assert np.all(lost), (st0, lp0, expect)


@pytest.mark.parametrize("name,n_cases", [("bn20", 100), ("bn60", 400)])
def test_rescaling_off_within_fp32_range(name, n_cases):
    """Where no message leaves FP32's range, rescale=0 gives the oracle's
    results too (both with and without its own rescaling)."""
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n_cases)
    lp, post, st = J.Plan(net, rescale=0).infer(ev)
    o = oracle.Oracle(net)
    for rescale in (False, True):
        olp, opost, ost = o.infer(ev, rescale=rescale, threads=16)
        assert_parity32(lp, post, st, olp, opost, ost, where=f"{name} rescale=0 vs oracle rescale={rescale}")


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_hub_cardinality_and_largest_clique(schedule):
    """bn110: a 60-state hub variable in 44 families and a 1.9e6-entry
    clique; 130 cases in one chunk and in two (arena room for one tile)."""
    net = configs.network("bn110")
    ev = configs.evidence("bn110", net, n_cases=130)
    ev[0, 0] = 59                  # the hub in its last state
    ev[1, 0] = -1
    probe = J.Plan(net, schedule=schedule)
    probe.infer(ev[:1])
    per_tile = probe.info()["arena_bytes"]
    lp, post, st = probe.infer(ev)
    small = J.Plan(net, schedule=schedule, arena_bytes=per_tile)
    lp2, post2, st2 = small.infer(ev)
    assert small.info()["chunk_cases"] == small.info()["tile_cases"]
    assert np.array_equal(st, st2) and np.array_equal(lp, lp2) and np.array_equal(post, post2)
    idx = [0, 1, 2, 129]
    olp, opost, ost = oracle.Oracle(net).infer(ev[idx], threads=8)
    assert_parity32(lp[idx], post[idx], st[idx], olp, opost, ost, where=f"bn110 hub, schedule {schedule}")

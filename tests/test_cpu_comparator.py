"""The multi-core CPU comparator in the paper's layer-parallel style
(jt_infer_cpu), CPU only: the library's own host compiler and an FP64
layer-by-layer Hugin pass, checked against the FP64 oracle (an independent
implementation, itself pinned to brute force) and for independence of the
thread count.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import sample_cases, tiny_random_network
from tests.common import TOL64
import paper_2212_04241_gb300.jt as J


def _check(lp, post, st, olp, opost, ost):
    assert np.array_equal(st, ost)
    ok = ost == 0
    assert np.all(np.isneginf(lp[ost == 1]))
    np.testing.assert_allclose(lp[ok], olp[ok], rtol=0, atol=TOL64 * max(1.0, np.abs(olp[ok]).max(initial=1.0)))
    np.testing.assert_allclose(post[ok], opost[ok], rtol=0, atol=TOL64)


def test_bn20_all_cases():
    net = configs.network("bn20")
    ev = configs.evidence("bn20", net)
    p = J.Plan(net, host_only=1)
    _check(*p.infer_cpu(ev, threads=4), *oracle.Oracle(net).infer(ev))


@pytest.mark.parametrize("name,n", [("bn60", 40), ("bn1000", 8)])
def test_workload_sample_and_thread_independence(name, n):
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n, seed=3)
    p = J.Plan(net, host_only=1)
    a = p.infer_cpu(ev, threads=1)
    _check(*a, *oracle.Oracle(net).infer(ev, threads=4))
    for t in (3, 8):
        b = p.infer_cpu(ev, threads=t)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("seed", range(20))
def test_tiny_networks_with_zero_probability_evidence(seed):
    net = tiny_random_network(seed)
    rng = np.random.default_rng(seed + 100)
    ev = sample_cases(net, 8, (0.0, 0.6), seed)
    arb = np.full((4, net.n), -1, dtype=np.int32)       # arbitrary patterns, some with P(e) = 0
    for i in range(4):
        for v in range(net.n):
            if rng.random() < 0.5:
                arb[i, v] = rng.integers(0, net.card[v])
    ev = np.concatenate([ev, arb])
    _check(*J.Plan(net, host_only=1).infer_cpu(ev, threads=3), *oracle.Oracle(net).infer(ev))


def test_invalid_evidence_and_refusals():
    net = configs.network("bn20")
    ev = configs.evidence("bn20", net, n_cases=3)
    ev[1, 4] = 7                                        # state out of range
    lp, post, st = J.Plan(net, host_only=1).infer_cpu(ev)
    assert st[1] == J.JT_CASE_BAD_EVIDENCE and np.isnan(lp[1]) and np.all(np.isnan(post[1]))
    assert st[0] == 0 and st[2] == 0
    with pytest.raises(J.JTError) as e:
        J.Plan(net, host_only=1, observed_set=[1, 2]).infer_cpu(ev[:1])
    assert e.value.status == J.JT_EINVAL


def test_drawn_networks_against_enumeration():
    """Hypothesis-drawn tiny networks and evidence (impossible evidence
    included): the comparator equals brute-force enumeration of the joint,
    with 1 and 3 threads."""
    hypothesis = pytest.importorskip("hypothesis")
    from hypothesis import given, settings, HealthCheck, strategies as st
    from synth.bn import make_network
    from tests.refsolvers import brute_force, joint

    @st.composite
    def cases(draw):
        n = draw(st.integers(1, 8))
        card = [draw(st.integers(2, 3)) for _ in range(n)]
        parents = []
        for v in range(n):
            k = draw(st.integers(0, min(v, 3)))
            parents.append(sorted(draw(st.lists(st.integers(0, v - 1), min_size=k, max_size=k, unique=True)))
                           if v else [])
        net = make_network(n, card, parents, draw(st.sampled_from([0.3, 1.0])),
                           np.random.default_rng(draw(st.integers(0, 2 ** 31 - 1))))
        rows = draw(st.lists(st.lists(st.integers(-1, 2), min_size=n, max_size=n), min_size=1, max_size=4))
        ev = np.array([[min(x, card[v] - 1) for v, x in enumerate(r)] for r in rows], dtype=np.int32)
        return net, ev

    @settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])
    @given(cases())
    def check(case):
        net, ev = case
        blp, bpost = brute_force(net, ev, joint(net))
        zero = ~np.isfinite(blp)
        p = J.Plan(net, host_only=1)
        for t in (1, 3):
            lp, post, st_ = p.infer_cpu(ev, threads=t)
            assert np.array_equal(st_ == J.JT_CASE_ZERO_EVIDENCE, zero)
            ok = ~zero
            if ok.any():
                np.testing.assert_allclose(lp[ok], blp[ok], rtol=0, atol=TOL64 * max(1.0, np.abs(blp[ok]).max()))
                np.testing.assert_allclose(post[ok], bpost[ok], rtol=0, atol=TOL64)

    check()

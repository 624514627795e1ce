"""Pin the FP64 oracle to things other than itself (CPU only).

* hand-derived closed forms (tests/golden/*.json);
* brute-force enumeration of the full joint (the plain definition of P(e)
  and P(X_v | e), Section 1 of the paper) on many tiny random networks and
  on the 20-variable binary workload (2^20-entry joint, 100 cases);
* the chain special case against the textbook forward/backward recursion;
* no evidence: P(e) = 1 and posteriors equal the prior marginals;
* independent root variables: P(e) = product of their priors.
"""
import numpy as np
import pytest

import oracle
from synth import configs, empty_evidence
from synth.bn import make_network, tiny_random_network, sample_cases
from tests.common import TOL64, golden_cases
from tests.refsolvers import (brute_force, chain_forward_backward, joint,
                              prior_marginals_chain)


@pytest.mark.parametrize("name,g,net", golden_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_golden_closed_forms(name, g, net):
    o = oracle.Oracle(net)
    offs = np.concatenate([[0], np.cumsum(net.card)])
    for case in g["cases"]:
        ev = np.asarray(case["evidence"], dtype=np.int32)
        for rescale in (True, False):
            lp, post, st = o.infer(ev, rescale=rescale)
            if case["pe"] == 0.0:
                assert st[0] == 1
                assert np.isneginf(lp[0])
                assert np.all(np.isnan(post[0]))
                continue
            assert st[0] == 0
            assert abs(lp[0] - np.log(case["pe"])) < 1e-12
            for v, pv in enumerate(case["posteriors"]):
                np.testing.assert_allclose(post[0, offs[v]:offs[v + 1]], pv, atol=1e-12)


def _random_evidence(net, rng, n_cases):
    """Evidence from ancestral samples with a random observed fraction."""
    return sample_cases(net, n_cases, (0.0, 0.6), int(rng.integers(1 << 30)))


@pytest.mark.parametrize("seed", range(60))
def test_tiny_random_vs_brute_force(seed):
    alpha = 0.3 if seed % 3 == 0 else 1.0
    net = tiny_random_network(seed, alpha=alpha)
    rng = np.random.default_rng(seed + 7)
    ev = _random_evidence(net, rng, 12)
    # also a few arbitrary (possibly zero-probability) evidence patterns
    arb = np.full((6, net.n), -1, dtype=np.int32)
    for i in range(6):
        for v in range(net.n):
            if rng.random() < 0.4:
                arb[i, v] = rng.integers(0, net.card[v])
    ev = np.concatenate([ev, arb, empty_evidence(net)])
    J = joint(net)
    blp, bpost = brute_force(net, ev, J)
    for root in ("largest", "center"):
        o = oracle.Oracle(net, root=root)
        for rescale in (True, False):
            lp, post, st = o.infer(ev, rescale=rescale)
            zero = ~np.isfinite(blp)
            assert np.array_equal(st == 1, zero)
            assert np.all(np.isneginf(lp[zero]))
            ok = ~zero
            np.testing.assert_allclose(lp[ok], blp[ok], rtol=0, atol=TOL64 * max(1, np.abs(blp[ok]).max(initial=1)))
            np.testing.assert_allclose(post[ok], bpost[ok], rtol=0, atol=TOL64)


def test_bn20_workload_vs_brute_force():
    """The 20-variable binary workload: 2^20-entry joint, all 100 cases."""
    net = configs.network("bn20")
    ev = configs.evidence("bn20", net)
    assert ev.shape == (100, 20)
    assert np.all((ev >= 0).sum(axis=1) == 4)
    blp, bpost = brute_force(net, ev)
    o = oracle.Oracle(net, root="largest")
    lp, post, st = o.infer(ev)
    assert np.all(st == 0)
    np.testing.assert_allclose(lp, blp, rtol=0, atol=1e-12)
    np.testing.assert_allclose(post, bpost, rtol=0, atol=1e-12)


def _chain_network(cards, seed):
    rng = np.random.default_rng(seed)
    n = len(cards)
    parents = [[]] + [[i - 1] for i in range(1, n)]
    return make_network(n, cards, parents, 1.0, rng)


@pytest.mark.parametrize("seed", range(5))
def test_chain_vs_forward_backward(seed):
    rng = np.random.default_rng(seed)
    n = 40
    cards = [int(c) for c in rng.integers(2, 6, size=n)]
    net = _chain_network(cards, seed)
    pi = net.cpt_of(0)
    T = [net.cpt_of(t) for t in range(1, n)]
    o = oracle.Oracle(net)
    offs = np.concatenate([[0], np.cumsum(net.card)])
    ev = sample_cases(net, 8, 0.3, seed)
    lp, post, st = o.infer(ev)
    for i in range(ev.shape[0]):
        flp, marg = chain_forward_backward(pi, T, ev[i])
        assert abs(lp[i] - flp) < 1e-10 * max(1, abs(flp))
        for t in range(n):
            np.testing.assert_allclose(post[i, offs[t]:offs[t + 1]], marg[t], atol=1e-12)


def test_no_evidence_gives_priors():
    net = _chain_network([3, 2, 4, 2, 3, 5, 2], 11)
    o = oracle.Oracle(net)
    lp, post, st = o.infer(empty_evidence(net))
    assert abs(lp[0]) < 1e-14
    pri = prior_marginals_chain(net.cpt_of(0), [net.cpt_of(t) for t in range(1, net.n)])
    offs = np.concatenate([[0], np.cumsum(net.card)])
    for t in range(net.n):
        np.testing.assert_allclose(post[0, offs[t]:offs[t + 1]], pri[t], atol=1e-14)
    # and on every workload: P(e) = 1 without evidence
    for name in ("bn60", "bn1000"):
        net = configs.network(name)
        lp, post, st = oracle.Oracle(net).infer(empty_evidence(net))
        assert abs(lp[0]) < 1e-12


def test_independent_roots_product_of_priors():
    """Evidence only on parentless variables: P(e) = product of their priors."""
    net = configs.network("bn60")
    roots = [v for v in range(net.n) if net.parent_ptr[v + 1] == net.parent_ptr[v]]
    assert len(roots) >= 3
    rng = np.random.default_rng(3)
    o = oracle.Oracle(net)
    for _ in range(5):
        ev = empty_evidence(net)
        expect = 0.0
        for v in roots:
            s = int(rng.integers(0, net.card[v]))
            ev[0, v] = s
            expect += np.log(net.cpt_of(v)[s])
        lp, _, _ = o.infer(ev)
        assert abs(lp[0] - expect) < 1e-12 * max(1, abs(expect))

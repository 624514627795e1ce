"""Invariants of calibrated junction trees, checked on the FP64 oracle.

* every calibrated clique sums to the same P(e);
* adjacent cliques agree on their separator marginals;
* posteriors sum to 1 and observed variables are point masses;
* P(e) and posteriors do not depend on the root or on the elimination
  order (min-fill vs min-degree), nor on power-of-two rescaling;
* the oracle's clique tree is a junction tree: running intersection, every
  family covered by a clique, cliques maximal.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import tiny_random_network, sample_cases


def _marginal(vars_, table, keep):
    axes = tuple(i for i, v in enumerate(vars_) if v not in keep)
    m = table.sum(axis=axes) if axes else table
    kept = [v for v in vars_ if v in keep]
    return kept, m


def _check_calibration(o, net, ev):
    lp, post, st = o.infer(ev)
    pe = np.exp(lp[0])
    tabs = {}
    for c in range(o.n_cliques):
        vars_, t = o.calibrated(ev, c)
        tabs[c] = (vars_, t)
        assert abs(t.sum() - pe) <= 1e-12 * max(pe, 1e-300) + 1e-300 * 0
    for c in range(o.n_cliques):
        vars_, parent = o.clique(c)
        if parent < 0:
            continue
        pv, pt = tabs[parent]
        cv, ct = tabs[c]
        sep = [v for v in cv if v in pv]
        k1, m1 = _marginal(cv, ct, sep)
        k2, m2 = _marginal(pv, pt, sep)
        assert k1 == k2
        np.testing.assert_allclose(m1, m2, rtol=1e-11, atol=1e-300)


@pytest.mark.parametrize("seed", range(12))
def test_calibration_tiny(seed):
    net = tiny_random_network(seed + 100)
    ev = sample_cases(net, 1, 0.3, seed)[0]
    _check_calibration(oracle.Oracle(net), net, ev)


def test_calibration_bn60():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=2)
    o = oracle.Oracle(net)
    for e in ev:
        _check_calibration(o, net, e)


def test_posterior_normalisation_and_point_masses():
    for name in ("bn60", "bn1000"):
        net = configs.network(name)
        ev = configs.evidence(name, net, n_cases=16)
        lp, post, st = oracle.Oracle(net).infer(ev)
        offs = np.concatenate([[0], np.cumsum(net.card)])
        for v in range(net.n):
            pv = post[:, offs[v]:offs[v + 1]]
            np.testing.assert_allclose(pv.sum(axis=1), 1.0, atol=1e-12)
            assert np.all(pv >= 0)
            obs = ev[:, v] >= 0
            if obs.any():
                onehot = np.eye(net.card[v])[ev[obs, v]]
                assert np.array_equal(pv[obs], onehot)


@pytest.mark.parametrize("name", ["bn60", "bn1000"])
def test_root_and_order_independence(name):
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=8)
    ref = oracle.Oracle(net).infer(ev)
    variants = [oracle.Oracle(net, root="center"),
                oracle.Oracle(net, elim="mindegree"),
                oracle.Oracle(net, root=0)]
    for o in variants:
        lp, post, st = o.infer(ev)
        np.testing.assert_allclose(lp, ref[0], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(post, ref[1], atol=1e-12)
    # rescaling only moves exponents: identical up to rounding
    lp, post, st = oracle.Oracle(net).infer(ev, rescale=False)
    np.testing.assert_allclose(lp, ref[0], rtol=1e-12)
    np.testing.assert_allclose(post, ref[1], atol=1e-12)


def _check_junction_tree(o, net):
    cl = o.cliques()
    sets = [set(v) for v, _ in cl]
    # maximality
    for i, a in enumerate(sets):
        for j, b in enumerate(sets):
            if i != j:
                assert not a <= b
    # family coverage
    for v in range(net.n):
        fam = set(int(p) for p in net.parents_of(v)) | {v}
        assert any(fam <= s for s in sets)
    # tree: exactly one root, parents form a tree
    parents = [p for _, p in cl]
    assert parents.count(-1) == 1
    # running intersection: cliques containing x form a connected subtree
    for x in range(net.n):
        holders = [c for c, s in enumerate(sets) if x in s]
        assert holders
        tops = [c for c in holders if parents[c] < 0 or x not in sets[parents[c]]]
        assert len(tops) == 1, f"variable {x} splits into {len(tops)} subtrees"


@pytest.mark.parametrize("name", ["bn20", "bn60", "bn110", "bn1000"])
def test_oracle_tree_is_junction_tree(name):
    net = configs.network(name)
    _check_junction_tree(oracle.Oracle(net), net)
    _check_junction_tree(oracle.Oracle(net, root="center"), net)


def test_center_root_minimises_height():
    for name in ("bn60", "bn110", "bn1000"):
        net = configs.network(name)
        oc = oracle.Oracle(net, root="center")
        for r in range(0, oc.n_cliques, max(1, oc.n_cliques // 15)):
            assert oracle.Oracle(net, root=r).height >= oc.height

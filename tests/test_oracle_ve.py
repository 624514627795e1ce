"""Oracle vs an independent exact algorithm (variable elimination), CPU only.

Variable elimination computes P(e) and P(X_v = s, e) by summing variables
out of the product of the (evidence-reduced) CPTs in a greedy min-size order,
with no clique tree at all.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from tests.refsolvers import ve_joint_marginal, ve_log_pe


@pytest.mark.parametrize("name,n_cases", [("bn60", 6), ("bn110", 2)])
def test_oracle_vs_variable_elimination(name, n_cases):
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n_cases)
    o = oracle.Oracle(net)
    lp, post, st = o.infer(ev)
    offs = np.concatenate([[0], np.cumsum(net.card)])
    rng = np.random.default_rng(5)
    for i in range(n_cases):
        vlp = ve_log_pe(net, ev[i])
        assert abs(lp[i] - vlp) <= 1e-10 * max(1.0, abs(vlp)), (lp[i], vlp)
        free = [v for v in range(net.n) if ev[i, v] < 0]
        for v in rng.choice(free, size=min(3, len(free)), replace=False):
            jm = ve_joint_marginal(net, ev[i], int(v))
            np.testing.assert_allclose(post[i, offs[v]:offs[v + 1]], jm / jm.sum(), atol=1e-11)
            assert abs(np.log(jm.sum()) - vlp) < 1e-10 * max(1.0, abs(vlp))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["bn420", "bn1000"])
def test_oracle_vs_variable_elimination_large(name):
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=1)
    lp, post, st = oracle.Oracle(net).infer(ev)
    vlp = ve_log_pe(net, ev[0])
    assert abs(lp[0] - vlp) <= 1e-10 * max(1.0, abs(vlp))

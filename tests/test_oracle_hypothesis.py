"""Property-based pin of the oracle (CPU only): hypothesis draws tiny
networks -- random DAGs over up to 8 variables with 2-3 states, any earlier
variable a possible parent, isolated variables and several components
allowed, Dirichlet rows of varying concentration -- and evidence patterns
(including impossible ones), and the oracle's log P(e), status and
posteriors must equal brute-force enumeration of the full joint (the plain
definition of Section 1's query) under both root rules, with and without
rescaling.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, HealthCheck, strategies as st  # noqa: E402

import oracle  # noqa: E402
from synth.bn import make_network  # noqa: E402
from tests.common import TOL64  # noqa: E402
from tests.refsolvers import brute_force, joint  # noqa: E402


@st.composite
def networks_and_evidence(draw):
    n = draw(st.integers(1, 8))
    card = [draw(st.integers(2, 3)) for _ in range(n)]
    parents = []
    for v in range(n):
        k = draw(st.integers(0, min(v, 3)))
        parents.append(sorted(draw(st.lists(st.integers(0, v - 1), min_size=k, max_size=k, unique=True))) if v else [])
    alpha = draw(st.sampled_from([0.2, 1.0, 5.0]))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    net = make_network(n, card, parents, alpha, np.random.default_rng(seed))
    cases = draw(st.lists(st.lists(st.integers(-1, 2), min_size=n, max_size=n), min_size=1, max_size=4))
    ev = np.array([[min(x, card[v] - 1) for v, x in enumerate(c)] for c in cases], dtype=np.int32)
    return net, ev


@settings(max_examples=300, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(networks_and_evidence())
def test_oracle_equals_enumeration(case):
    net, ev = case
    blp, bpost = brute_force(net, ev, joint(net))
    zero = ~np.isfinite(blp)
    for root in ("largest", "center"):
        o = oracle.Oracle(net, root=root)
        for rescale in (True, False):
            lp, post, status = o.infer(ev, rescale=rescale)
            assert np.array_equal(status == 1, zero)
            assert np.all(np.isneginf(lp[zero]))
            ok = ~zero
            if ok.any():
                np.testing.assert_allclose(lp[ok], blp[ok], rtol=0, atol=TOL64 * max(1.0, np.abs(blp[ok]).max()))
                np.testing.assert_allclose(post[ok], bpost[ok], rtol=0, atol=TOL64)

"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each mutant is the oracle compiled with one plausible mistake
(-DORACLE_MUTANT=k, see jt_oracle.c): a missing separator division, an
inverted evidence test, a transposed CPT layout, a dropped rescale exponent,
a dropped marginalisation term, a wrong message order, a minimum instead of
maximum spanning tree, unmarried parents.  The same brute-force and
closed-form pins that the correct oracle passes must fail for every mutant.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import tiny_random_network, sample_cases
from tests.common import golden_cases
from tests.refsolvers import brute_force

MUTANTS = [1, 2, 3, 4, 5, 6, 8, 9]


def _pins_pass(mutant: int) -> bool:
    """True when every pin agrees with the (possibly mutated) oracle."""
    try:
        for _, g, net in golden_cases():
            o = oracle.Oracle(net, mutant=mutant)
            for case in g["cases"]:
                if case["pe"] == 0.0:
                    continue
                lp, post, st = o.infer(np.asarray(case["evidence"], dtype=np.int32))
                if not abs(lp[0] - np.log(case["pe"])) < 1e-9:
                    return False
                offs = np.concatenate([[0], np.cumsum(net.card)])
                for v, pv in enumerate(case["posteriors"]):
                    if not np.allclose(post[0, offs[v]:offs[v + 1]], pv, atol=1e-9):
                        return False
        nets = [configs.network("bn20")] + [tiny_random_network(s) for s in range(20)]
        for k, net in enumerate(nets):
            ev = sample_cases(net, 8, 0.3, 1000 + k)
            blp, bpost = brute_force(net, ev)
            o = oracle.Oracle(net, mutant=mutant)
            lp, post, st = o.infer(ev)
            if not (np.allclose(lp, blp, atol=1e-9) and np.allclose(post, bpost, atol=1e-9)):
                return False
    except oracle.OracleError:
        return False
    return True


def test_correct_oracle_passes_pins():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", MUTANTS)
def test_mutant_is_caught(mutant):
    assert not _pins_pass(mutant), f"planted mistake {mutant} slipped through the pins"

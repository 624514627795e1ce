"""Plans specialised to an observed set (GPU, through the C ABI).

When every case of a batch observes the same set O of variables (their
states varying from case to case), the compiler slices O's dimensions out
of every clique and separator table and each case reads the slice of the
base tables that its states select (the reduction step of Section 2 read as
dimension removal).  The results must equal the oracle's and the standard
plan's within the FP32 tolerance, for cases observing O only and O plus
further variables, under both schedules.
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import sample_cases, tiny_random_network
from tests.common import POST_TOL32, assert_parity32, max_logpe_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402


def observed_set_cases(net, n_cases, n_obs, extra, seed):
    """Cases that all observe the same n_obs variables (states from an
    ancestral sample) and, with probability `extra`, each other variable."""
    rng = np.random.default_rng(seed)
    obs = np.sort(rng.choice(net.n, size=n_obs, replace=False))
    x = sample_cases(net, n_cases, 1.0, seed=seed + 1)      # full assignments
    ev = np.full_like(x, -1)
    ev[:, obs] = x[:, obs]
    more = rng.random(x.shape) < extra
    ev[more] = x[more]
    return obs.tolist(), ev.astype(np.int32)


@pytest.mark.parametrize("name,n_cases,n_obs,extra", [("bn20", 100, 4, 0.0), ("bn60", 700, 6, 0.0),
                                                      ("bn60", 700, 6, 0.05), ("bn60", 300, 15, 0.1),
                                                      ("bn110", 140, 17, 0.0), ("bn1000", 300, 100, 0.05)])
@pytest.mark.parametrize("schedule", [J.JT_SCHEDULE_DATAFLOW, J.JT_SCHEDULE_LAYERS])
def test_sliced_plan_matches_oracle_and_standard_plan(name, n_cases, n_obs, extra, schedule):
    net = configs.network(name)
    obs, ev = observed_set_cases(net, n_cases, n_obs, extra, seed=17)
    sliced = J.Plan(net, observed_set=obs, schedule=schedule)
    info = sliced.info()
    assert info["sliced_vars"] == n_obs
    a = sliced.infer(ev)
    b = J.Plan(net, schedule=schedule).infer(ev)
    assert np.array_equal(a[2], b[2])
    ok = a[2] == 0
    assert np.max(np.abs(a[1][ok] - b[1][ok])) <= POST_TOL32
    assert max_logpe_err(a[0][ok], b[0][ok]) <= 1e-6
    idx = np.arange(0, n_cases, max(1, n_cases // (8 if name == "bn110" else 40)))
    olp, opost, ost = oracle.Oracle(net).infer(ev[idx], threads=16)
    assert_parity32(a[0][idx], a[1][idx], a[2][idx], olp, opost, ost, where=f"{name} sliced {n_obs}")


@pytest.mark.parametrize("seed", range(12))
def test_sliced_tiny_networks(seed):
    net = tiny_random_network(seed)
    k = max(1, net.n // 3)
    obs, ev = observed_set_cases(net, 40, k, 0.2, seed=seed)
    lp, post, st = J.Plan(net, observed_set=obs, cases_per_thread=1).infer(ev)
    assert_parity32(lp, post, st, *oracle.Oracle(net).infer(ev), where=f"tiny {seed}")


def test_case_breaking_the_observed_set_is_flagged_alone():
    net = configs.network("bn60")
    obs, ev = observed_set_cases(net, 200, 6, 0.0, seed=3)
    ev[7, obs[2]] = -1                        # one case leaves a variable of the set unobserved
    lp, post, st = J.Plan(net, observed_set=obs).infer(ev)
    assert st[7] == J.JT_CASE_BAD_EVIDENCE and np.isnan(lp[7])
    others = np.arange(200) != 7
    assert np.all(st[others] == 0)
    olp, opost, ost = oracle.Oracle(net).infer(ev[others][:20], threads=16)
    assert_parity32(lp[others][:20], post[others][:20], st[others][:20], olp, opost, ost, where="flagged case")


def test_plain_path_refuses_sliced_plans():
    net = configs.network("bn20")
    obs, ev = observed_set_cases(net, 4, 3, 0.0, seed=1)
    p = J.Plan(net, observed_set=obs)
    with pytest.raises(J.JTError) as e:
        p.infer_plain(ev)
    assert e.value.status == J.JT_EINVAL

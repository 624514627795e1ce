"""Property-based checks of the library's host compiler (CPU only).

For networks drawn by hypothesis (random DAGs up to 9 variables, 2-4
states, isolated variables and several components allowed), the library's
compiler (jt_compile, host only) must produce the same maximal cliques as
the oracle's independently written compiler (both follow min-fill with
lowest-index ties), a tree of the right height for the chosen root rule,
and index maps that pass the mixed-radix checker of tests/native.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, HealthCheck, strategies as st  # noqa: E402

import oracle  # noqa: E402
import paper_2212_04241_gb300.jt as J  # noqa: E402
from synth.bn import make_network  # noqa: E402
from tests.test_index_maps import ROOT, _write  # noqa: E402


@st.composite
def networks(draw):
    n = draw(st.integers(1, 9))
    card = [draw(st.integers(2, 4)) for _ in range(n)]
    parents = []
    for v in range(n):
        k = draw(st.integers(0, min(v, 3)))
        parents.append(sorted(draw(st.lists(st.integers(0, v - 1), min_size=k, max_size=k, unique=True))) if v else [])
    return make_network(n, card, parents, 1.0, np.random.default_rng(draw(st.integers(0, 2 ** 31 - 1))))


@settings(max_examples=200, deadline=None, suppress_health_check=[HealthCheck.too_slow])
@given(networks())
def test_cliques_and_height_match_the_oracle_compiler(net):
    for rule, name in ((J.JT_ROOT_LARGEST, "largest"), (J.JT_ROOT_MIN_HEIGHT, "center")):
        p = J.Plan(net, host_only=1, root_rule=rule)
        info = p.info()
        ours = sorted(tuple(sorted(p.clique(c)[0])) for c in range(info["n_cliques"]))
        o = oracle.Oracle(net, root=name)
        assert ours == sorted(tuple(v) for v, _ in o.cliques())
        assert info["n_levels"] == o.height + 1


@pytest.fixture(scope="module")
def map_checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("hmaps") / "check_maps")
    subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(ROOT, "tests", "native", "check_maps.cpp"),
                    os.path.join(ROOT, "paper_2212_04241_gb300", "csrc", "compile.cpp"), "-o", exe],
                   check=True, capture_output=True)
    return exe


@settings(max_examples=100, deadline=None, suppress_health_check=[HealthCheck.too_slow,
                                                                   HealthCheck.function_scoped_fixture])
@given(networks(), st.data())
def test_index_maps_of_drawn_networks(map_checker, tmp_path, net, data):
    path = str(tmp_path / "net.bin")
    _write(net, path)
    args = []
    if net.n > 1 and data.draw(st.booleans()):
        obs = data.draw(st.lists(st.integers(0, net.n - 1), min_size=1, max_size=net.n - 1, unique=True))
        args.append("obs=" + ",".join(str(v) for v in sorted(obs)))
    if data.draw(st.booleans()):
        q = data.draw(st.lists(st.integers(0, net.n - 1), min_size=1, max_size=2, unique=True))
        args.append("query=" + ",".join(str(v) for v in sorted(q)))
    r = subprocess.run([map_checker, path, *args], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and " 0 failed" in r.stdout, (args, r.stdout)

"""The library's index maps against a direct mixed-radix restatement (CPU).

`tests/native/check_maps.cpp` is built against the library's host compiler
and checks every map of a compiled plan -- the extension of child messages
into a clique, the evidence digits, the base-table slice maps of
observed-set plans, and every distribute task's marginalisation (each
source entry visited once, target and ratio entries right) -- by decoding
each table entry's digits with plain division (Section 2's index mapping
between an original and an updated table).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from synth import configs
from synth.bn import tiny_random_network

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("maps") / "check_maps")
    subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(ROOT, "tests", "native", "check_maps.cpp"),
                    os.path.join(ROOT, "paper_2212_04241_gb300", "csrc", "compile.cpp"), "-o", exe],
                   check=True, capture_output=True)
    return exe


def _write(net, path):
    par = np.ascontiguousarray(net.parents, dtype=np.int32)
    cpt = np.ascontiguousarray(net.cpt, dtype=np.float64)
    with open(path, "wb") as f:
        f.write(np.array([net.n, par.size, cpt.size], dtype=np.int64).tobytes())
        f.write(np.ascontiguousarray(net.card, dtype=np.int32).tobytes())
        f.write(np.ascontiguousarray(net.parent_ptr, dtype=np.int32).tobytes())
        f.write(par.tobytes())
        f.write(cpt.tobytes())


def _run(checker, net, tmp_path, *args):
    path = str(tmp_path / "net.bin")
    _write(net, path)
    r = subprocess.run([checker, path, *args], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 failed" in r.stdout


@pytest.mark.parametrize("name", ["bn20", "bn60", "bn110", "bn1000"])
def test_workload_maps(checker, name, tmp_path):
    _run(checker, configs.network(name), tmp_path)


@pytest.mark.parametrize("name,obs,query", [("bn60", "2,15,18,29,35,46", ""), ("bn1000", "5,600,700", "999,400"),
                                            ("bn60", "", "41,50")])
def test_specialised_plan_maps(checker, name, obs, query, tmp_path):
    args = ([f"obs={obs}"] if obs else []) + ([f"query={query}"] if query else [])
    _run(checker, configs.network(name), tmp_path, *args)


@pytest.mark.parametrize("seed", range(30))
def test_tiny_network_maps(checker, seed, tmp_path):
    _run(checker, tiny_random_network(seed), tmp_path)

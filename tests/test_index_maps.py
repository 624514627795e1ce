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


@pytest.mark.parametrize("name,args", [("bn60", ["cpt=1", "rows=4096"]), ("bn60", ["cpt=1", "rows=128"]),
                                       ("bn110", ["cpt=2", "rows=256"]), ("bn420", ["cpt=4"]),
                                       ("bn420", ["cpt=1", "rows=128"]), ("bn60", ["fuse=0"]),
                                       ("bn420", ["rows=64"])])
def test_fused_pair_maps(checker, name, args, tmp_path):
    """Fused distribute pairs (two marginals of one clique table from one
    read): every index of the reordered primary, the secondary's per-F-block
    targets, and the pieces of F-blocks larger than an item."""
    _run(checker, configs.network(name), tmp_path, *args)


@pytest.mark.parametrize("seed", range(30, 60))
def test_tiny_network_fused_maps(checker, seed, tmp_path):
    _run(checker, tiny_random_network(seed), tmp_path, "cpt=1", "rows=128" if seed % 2 else "rows=4096")

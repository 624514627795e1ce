"""Shared test helpers: golden fixtures and comparison tolerances."""
from __future__ import annotations

import glob
import json
import os

import numpy as np

from synth.bn import make_network

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# FP64 oracle vs exact solvers
TOL64 = 1e-11
# FP32 GPU path vs FP64 oracle: max abs posterior error and the log P(e)
# criterion |d log P(e)| <= 1e-6 * max(1, |log P(e)|)
POST_TOL32 = 1e-5
LOGPE_REL32 = 1e-6


def golden_cases():
    out = []
    for path in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.json"))):
        with open(path) as f:
            g = json.load(f)
        rng = np.random.default_rng(0)
        net = make_network(len(g["card"]), g["card"], g["parents"], 1.0, rng)
        net.cpt = np.concatenate([np.asarray(r, dtype=np.float64) for r in g["cpt"]])
        out.append((os.path.basename(path), g, net))
    return out


def logpe_close(a, b, rel):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    both_inf = np.isneginf(a) & np.isneginf(b)
    err = np.abs(a - b)
    bound = rel * np.maximum(1.0, np.abs(b))
    return bool(np.all(both_inf | (err <= bound)))


def max_logpe_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ok = np.isfinite(b)
    if not ok.any():
        return 0.0
    return float(np.max(np.abs(a[ok] - b[ok]) / np.maximum(1.0, np.abs(b[ok]))))


def assert_parity32(lp, post, st, olp, opost, ost, where=""):
    """FP32 batched path vs FP64 oracle: statuses equal, max abs posterior
    error <= 1e-5, |d log P(e)| <= 1e-6 * max(1, |log P(e)|)."""
    assert np.array_equal(st, ost), f"{where}: status mismatch"
    ok = ost == 0
    perr = float(np.max(np.abs(post[ok] - opost[ok]))) if ok.any() else 0.0
    lerr = max_logpe_err(lp[ok], olp[ok]) if ok.any() else 0.0
    assert perr <= POST_TOL32, f"{where}: posterior error {perr:.3g}"
    assert lerr <= LOGPE_REL32, f"{where}: log P(e) error {lerr:.3g}"
    return perr, lerr

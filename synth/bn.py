"""Seeded synthetic Bayesian networks and evidence cases.

This module only *generates inputs*: random DAGs in topological order,
Dirichlet-distributed conditional probability tables (CPTs) and evidence
cases drawn by ancestral sampling.  It contains no junction-tree arithmetic
and is shared by the oracle tests, the CUDA parity tests and the benchmark.

The workload shape follows the evaluation setup of the paper (Section 3:
random test cases with a fixed fraction of observed variables); the
networks themselves are synthetic stand-ins for the bnlearn networks the
paper uses, which are not available here.

Conventions (the library's C ABI uses the same ones):
  * variables are numbered 0..n-1 in topological order;
  * ``parent_ptr``/``parents`` is a CSR list, parents of a node ascending;
  * the CPT of node v is a row-major array with one row per joint parent
    configuration (mixed radix, the first listed parent varies slowest) and
    ``card[v]`` columns (the child's state varies fastest); all CPTs are
    concatenated in node order into one float64 array;
  * evidence is int32 ``[n_cases, n]`` with -1 for an unobserved variable.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Network:
    card: np.ndarray        # int32 [n]
    parent_ptr: np.ndarray  # int32 [n+1]
    parents: np.ndarray     # int32 [nnz]
    cpt: np.ndarray         # float64 [sum_v rows(v)*card(v)]
    cpt_ptr: np.ndarray     # int64 [n+1], offsets of each node's CPT in ``cpt``

    @property
    def n(self) -> int:
        return int(self.card.shape[0])

    def parents_of(self, v: int) -> np.ndarray:
        return self.parents[self.parent_ptr[v]:self.parent_ptr[v + 1]]

    def cpt_of(self, v: int) -> np.ndarray:
        """CPT of node v reshaped to [card(p1), ..., card(pk), card(v)]."""
        pa = self.parents_of(v)
        shape = tuple(int(self.card[p]) for p in pa) + (int(self.card[v]),)
        return self.cpt[self.cpt_ptr[v]:self.cpt_ptr[v + 1]].reshape(shape)


def round_half_up(x: float) -> int:
    return int(np.floor(x + 0.5))


def make_network(n, card, parent_lists, alpha, rng) -> Network:
    """Pack parent lists and draw Dirichlet(alpha) CPT rows with ``rng``."""
    card = np.asarray(card, dtype=np.int32)
    ptr = np.zeros(n + 1, dtype=np.int32)
    flat = []
    for v in range(n):
        pa = sorted(int(p) for p in parent_lists[v])
        assert all(0 <= p < v for p in pa), "parents must precede the child"
        flat.extend(pa)
        ptr[v + 1] = len(flat)
    parents = np.asarray(flat, dtype=np.int32)
    cpt_ptr = np.zeros(n + 1, dtype=np.int64)
    blocks = []
    for v in range(n):
        pa = parents[ptr[v]:ptr[v + 1]]
        rows = int(np.prod([card[p] for p in pa], dtype=np.int64)) if len(pa) else 1
        g = rng.gamma(alpha, 1.0, size=(rows, int(card[v])))
        # a row of all-zero gammas is astronomically unlikely; guard anyway
        s = g.sum(axis=1, keepdims=True)
        bad = (s[:, 0] <= 0)
        if bad.any():
            g[bad] = 1.0
            s = g.sum(axis=1, keepdims=True)
        blocks.append((g / s).ravel())
        cpt_ptr[v + 1] = cpt_ptr[v] + rows * int(card[v])
    cpt = np.concatenate(blocks).astype(np.float64)
    return Network(card, ptr, parents, cpt, cpt_ptr)


def random_network(n, card_choices, k_range, window, alpha, seed,
                   hub_card=None, hub_frac=0.0, root_has_parents=True):
    """Random DAG in topological order.

    Each node v draws a parent count k uniformly from ``k_range`` (inclusive),
    clamped to the number of available predecessors, and picks that many
    parents uniformly without replacement among the previous ``window`` nodes.
    With ``hub_card`` set, node 0 gets that cardinality and is added as an
    extra parent of round(hub_frac * n) nodes drawn uniformly from 1..n-1.
    """
    rng = np.random.default_rng(seed)
    card = rng.choice(np.asarray(card_choices), size=n).astype(np.int32)
    if hub_card is not None:
        card[0] = hub_card
    parent_lists = []
    for v in range(n):
        lo = max(0, v - window)
        avail = v - lo
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        k = min(k, avail)
        if v == 0 and not root_has_parents:
            k = 0
        pa = rng.choice(np.arange(lo, v), size=k, replace=False) if k > 0 else []
        parent_lists.append(set(int(p) for p in pa))
    if hub_card is not None:
        m = round_half_up(hub_frac * n)
        kids = rng.choice(np.arange(1, n), size=m, replace=False)
        for c in kids:
            parent_lists[int(c)].add(0)
    return make_network(n, card, parent_lists, alpha, rng)


def sample_cases(net: Network, n_cases: int, observed, seed) -> np.ndarray:
    """Ancestral sampling of full assignments, then a random observed subset.

    ``observed`` is either a fraction p (exactly round_half_up(p*n) variables
    are observed per case) or a pair (p_lo, p_hi) from which each case draws
    its own fraction uniformly.  Variables to observe are chosen uniformly
    without replacement.  Evidence sampled this way always has P(e) > 0.
    """
    rng = np.random.default_rng(seed)
    n = net.n
    x = np.zeros((n_cases, n), dtype=np.int64)
    for v in range(n):
        pa = net.parents_of(v)
        r = int(net.card[v])
        table = net.cpt[net.cpt_ptr[v]:net.cpt_ptr[v + 1]].reshape(-1, r)
        row = np.zeros(n_cases, dtype=np.int64)
        for p in pa:
            row = row * int(net.card[p]) + x[:, p]
        cdf = np.cumsum(table[row], axis=1)
        u = rng.random(n_cases)[:, None] * cdf[:, -1:]
        x[:, v] = np.minimum((u >= cdf).sum(axis=1), r - 1)
    ev = np.full((n_cases, n), -1, dtype=np.int32)
    for i in range(n_cases):
        if isinstance(observed, tuple):
            p = rng.uniform(observed[0], observed[1])
        else:
            p = observed
        m = min(n, round_half_up(p * n))
        idx = rng.choice(n, size=m, replace=False)
        ev[i, idx] = x[i, idx]
    return ev


def empty_evidence(net: Network, n_cases: int = 1) -> np.ndarray:
    return np.full((n_cases, net.n), -1, dtype=np.int32)


def tiny_random_network(seed, max_vars=12, max_card=4, max_joint=1 << 18,
                        alpha=1.0):
    """Small random network for exhaustive checks.

    Any earlier node may be a parent (not just a window), some nodes have no
    parents, and the graph may be disconnected.  The joint table size
    prod(card) is kept at most ``max_joint`` so brute force stays cheap.
    Dirichlet(alpha) rows; with ``alpha`` small some CPT entries underflow
    towards zero, which exercises zero separators.
    """
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, max_vars + 1))
    card = []
    size = 1
    for _ in range(n):
        c = int(rng.integers(2, max_card + 1))
        while size * c > max_joint and c > 2:
            c -= 1
        if size * c > max_joint:
            n = len(card)
            break
        card.append(c)
        size *= c
    n = len(card)
    parent_lists = []
    p_edge = float(rng.uniform(0.05, 0.6))
    for v in range(n):
        pa = [u for u in range(v) if rng.random() < p_edge][:4]
        parent_lists.append(set(pa))
    return make_network(n, card, parent_lists, alpha, rng)

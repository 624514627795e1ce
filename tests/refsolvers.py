"""Independent exact solvers used to pin the oracle (test code only).

None of these shares code with the oracle or with the GPU library:
  * ``brute_force``: the plain definition -- enumerate the full joint
    P(x) = prod_v P(x_v | x_pa(v)), then P(e) = sum over x consistent with e
    and P(X_v = s | e) = P(X_v = s, e) / P(e).
  * ``variable_elimination``: sum-product variable elimination with a greedy
    min-size order (a different exact algorithm from the junction tree).
  * ``chain_forward_backward``: the textbook HMM-style forward/backward
    recursion for a chain-structured network.
  * ``prior_marginals``: forward propagation of priors on a polytree-free
    chain/tree network without evidence (topological sum-product).
"""
from __future__ import annotations

import string

import numpy as np


def _family_factor(net, v):
    """CPT of v as (vars ascending, ndarray with one axis per var)."""
    pa = [int(p) for p in net.parents_of(v)]
    fam = pa + [v]
    t = net.cpt_of(v)
    order = sorted(range(len(fam)), key=lambda i: fam[i])
    return tuple(fam[i] for i in order), np.transpose(t, order)


def joint(net):
    """Full joint as an ndarray with axis v for variable v (small nets only)."""
    n = net.n
    shape = [int(c) for c in net.card]
    J = np.ones(shape, dtype=np.float64)
    for v in range(n):
        fam, t = _family_factor(net, v)
        bshape = [1] * n
        for a, u in enumerate(fam):
            bshape[u] = shape[u]
        # t's axes are in ascending var order, matching broadcast order
        J = J * t.reshape(bshape)
    return J


def brute_force(net, evidence, J=None):
    """log P(e) and posteriors (same layout as the oracle) by enumeration."""
    if J is None:
        J = joint(net)
    ev = np.atleast_2d(evidence)
    n = net.n
    offs = np.concatenate([[0], np.cumsum(net.card)]).astype(int)
    log_pe = np.zeros(ev.shape[0])
    post = np.zeros((ev.shape[0], int(offs[-1])))
    for i, e in enumerate(ev):
        idx = tuple(int(x) if x >= 0 else slice(None) for x in e)
        sub = J[idx]  # remaining axes: unobserved vars in ascending order
        pe = sub.sum()
        log_pe[i] = np.log(pe) if pe > 0 else -np.inf
        free = [v for v in range(n) if e[v] < 0]
        for v in range(n):
            if e[v] >= 0:
                post[i, offs[v]:offs[v + 1]] = 0.0
                post[i, offs[v] + int(e[v])] = 1.0
            else:
                ax = free.index(v)
                other = tuple(a for a in range(sub.ndim) if a != ax)
                m = sub.sum(axis=other) if other else sub
                post[i, offs[v]:offs[v + 1]] = m / pe
    return log_pe, post


# ----------------------------------------------------------------------
# variable elimination
# ----------------------------------------------------------------------

def _einsum_product(factors, keep):
    """Multiply factors (vars, array) and sum out everything not in keep."""
    allv = []
    for vs, _ in factors:
        for v in vs:
            if v not in allv:
                allv.append(v)
    letters = {v: (string.ascii_letters[i]) for i, v in enumerate(allv)}
    assert len(allv) <= 52
    out = [v for v in allv if v in keep]
    spec = ",".join("".join(letters[v] for v in vs) for vs, _ in factors)
    spec += "->" + "".join(letters[v] for v in out)
    arr = np.einsum(spec, *[a for _, a in factors], optimize="greedy")
    return tuple(out), arr


def _reduce(factor, ev):
    vs, a = factor
    idx = []
    keep = []
    for v in vs:
        if ev[v] >= 0:
            idx.append(int(ev[v]))
        else:
            idx.append(slice(None))
            keep.append(v)
    return tuple(keep), a[tuple(idx)]


def _eliminate(factors, to_eliminate):
    factors = list(factors)
    remaining = set(to_eliminate)
    while remaining:
        # greedy: variable whose elimination creates the smallest factor
        best, best_size = None, None
        for x in sorted(remaining):
            scope = set()
            for vs, a in factors:
                if x in vs:
                    scope |= set(vs)
            size = 1
            for v in scope:
                for vs, a in factors:
                    if v in vs:
                        size *= a.shape[vs.index(v)]
                        break
            if best is None or size < best_size:
                best, best_size = x, size
        x = best
        remaining.discard(x)
        touch = [f for f in factors if x in f[0]]
        rest = [f for f in factors if x not in f[0]]
        if not touch:
            continue
        scope = set()
        for vs, _ in touch:
            scope |= set(vs)
        scope.discard(x)
        rest.append(_einsum_product(touch, scope))
        factors = rest
    return factors


def ve_log_pe(net, evidence):
    """log P(e) by variable elimination over all unobserved variables."""
    ev = np.asarray(evidence)
    factors = [_reduce(_family_factor(net, v), ev) for v in range(net.n)]
    free = [v for v in range(net.n) if ev[v] < 0]
    rest = _eliminate(factors, free)
    val = 1.0
    for vs, a in rest:
        assert len(vs) == 0
        val *= float(a)
    return np.log(val)


def ve_joint_marginal(net, evidence, v):
    """Vector P(X_v = s, e) over s, by variable elimination."""
    ev = np.asarray(evidence)
    assert ev[v] < 0
    factors = [_reduce(_family_factor(net, u), ev) for u in range(net.n)]
    free = [u for u in range(net.n) if ev[u] < 0 and u != v]
    rest = _eliminate(factors, free)
    res = np.ones(int(net.card[v]))
    for vs, a in rest:
        if len(vs) == 0:
            res = res * float(a)
        else:
            assert vs == (v,)
            res = res * a
    return res


# ----------------------------------------------------------------------
# closed forms on special structures
# ----------------------------------------------------------------------

def chain_forward_backward(pi, T, evidence):
    """Chain x0 -> x1 -> ... -> x_{n-1}, P(x0) = pi, P(x_t | x_{t-1}) = T[t]
    (T[t][i, j] = P(x_t = j | x_{t-1} = i)).  Returns (log P(e), marginals)
    via the forward/backward recursion with per-step normalisation."""
    n = len(T) + 1
    def lam(t, r):
        l = np.ones(r)
        if evidence[t] >= 0:
            l = np.zeros(r)
            l[evidence[t]] = 1.0
        return l
    alpha = []
    c = []
    a = pi * lam(0, len(pi))
    c.append(a.sum()); a = a / c[-1]; alpha.append(a)
    for t in range(1, n):
        a = (alpha[-1] @ T[t - 1]) * lam(t, T[t - 1].shape[1])
        c.append(a.sum()); a = a / c[-1]; alpha.append(a)
    beta = [None] * n
    beta[n - 1] = np.ones_like(alpha[n - 1])
    for t in range(n - 2, -1, -1):
        b = T[t] @ (beta[t + 1] * lam(t + 1, T[t].shape[1]))
        beta[t] = b / c[t + 1]
    marg = [alpha[t] * beta[t] for t in range(n)]
    marg = [m / m.sum() for m in marg]
    return float(np.sum(np.log(c))), marg


def prior_marginals_chain(pi, T):
    m = [np.asarray(pi, dtype=np.float64)]
    for t in range(len(T)):
        m.append(m[-1] @ T[t])
    return m

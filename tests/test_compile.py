"""The library's host compiler (jt_compile with host_only=1), CPU only.

Checks the junction-tree properties of the plan it builds and compares its
clique set with the oracle's independently written compiler (both follow
the same min-fill rule, so the maximal cliques must coincide as sets).
"""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.bn import make_network, tiny_random_network
import paper_2212_04241_gb300.jt as J


def _plan(net, **kw):
    return J.Plan(net, host_only=1, **kw)


def _structure(p):
    info = p.info()
    return [p.clique(c) for c in range(info["n_cliques"])], info


@pytest.mark.parametrize("name", ["bn20", "bn60", "bn110", "bn420", "bn1000"])
def test_cliques_match_oracle(name):
    net = configs.network(name)
    cl, info = _structure(_plan(net))
    o = oracle.Oracle(net)
    ours = sorted(tuple(sorted(v)) for v, _, _ in cl)
    theirs = sorted(tuple(v) for v, _ in o.cliques())
    assert ours == theirs
    assert info["max_clique_entries"] == o.max_clique
    assert info["sum_clique_entries"] == o.sum_clique


@pytest.mark.parametrize("name", ["bn20", "bn60", "bn110", "bn1000"])
@pytest.mark.parametrize("root_rule", [J.JT_ROOT_LARGEST, J.JT_ROOT_MIN_HEIGHT])
def test_junction_tree_properties(name, root_rule):
    net = configs.network(name)
    p = _plan(net, root_rule=root_rule)
    cl, info = _structure(p)
    sets = [set(v) for v, _, _ in cl]
    parents = [par for _, par, _ in cl]
    depths = [d for _, _, d in cl]
    assert parents.count(-1) == 1
    root = parents.index(-1)
    assert root == info["root"]
    # depth = BFS layer (Section 2's traversal): parent is one layer up
    for c, par in enumerate(parents):
        if par >= 0:
            assert depths[c] == depths[par] + 1
    assert info["n_levels"] == max(depths) + 1
    # family coverage
    for v in range(net.n):
        fam = set(int(q) for q in net.parents_of(v)) | {v}
        assert any(fam <= s for s in sets)
    # running intersection
    for x in range(net.n):
        holders = [c for c, s in enumerate(sets) if x in s]
        tops = [c for c in holders if parents[c] < 0 or x not in sets[parents[c]]]
        assert len(tops) == 1
    # layout: the upward separator is the outermost block, in the parent's order
    for c, (vars_, par, _) in enumerate(cl):
        if par < 0:
            continue
        sep = [v for v in cl[par][0] if v in sets[c]]
        assert vars_[:len(sep)] == sep
    # root rule
    o = oracle.Oracle(net, root="largest" if root_rule == J.JT_ROOT_LARGEST else "center")
    assert info["n_levels"] == o.height + 1
    if root_rule == J.JT_ROOT_LARGEST:
        sizes = [int(np.prod([net.card[v] for v in s])) for s in sets]
        assert sizes[root] == max(sizes) and root == sizes.index(max(sizes))


@pytest.mark.parametrize("seed", range(25))
def test_tiny_networks_compile(seed):
    net = tiny_random_network(seed)
    cl, info = _structure(_plan(net))
    o = oracle.Oracle(net)
    assert sorted(tuple(sorted(v)) for v, _, _ in cl) == sorted(tuple(v) for v, _ in o.cliques())


def test_validation_errors():
    net = configs.network("bn20")
    bad = make_network(net.n, net.card, [list(net.parents_of(v)) for v in range(net.n)], 1.0,
                       np.random.default_rng(0))
    bad.cpt = bad.cpt.copy()
    bad.cpt[3] += 0.01  # a CPT row no longer sums to 1
    with pytest.raises(J.JTError) as e:
        _plan(bad)
    assert e.value.status == J.JT_EINVAL
    neg = make_network(net.n, net.card, [list(net.parents_of(v)) for v in range(net.n)], 1.0,
                       np.random.default_rng(0))
    neg.cpt = neg.cpt.copy()
    neg.cpt[0], neg.cpt[1] = -0.5, 1.5
    with pytest.raises(J.JTError) as e:
        _plan(neg)
    assert e.value.status == J.JT_EINVAL
    # a directed cycle: 0 -> 1 -> 2 -> 0
    cyc = make_network(3, [2, 2, 2], [[], [0], [1]], 1.0, np.random.default_rng(0))
    cyc.parents = np.array([2, 0, 1], dtype=np.int32)
    cyc.parent_ptr = np.array([0, 1, 2, 3], dtype=np.int32)
    cyc.cpt = np.full(12, 0.5)
    with pytest.raises(J.JTError) as e:
        _plan(cyc)
    assert e.value.status == J.JT_ECYCLE
    # a clique above the configured limit
    with pytest.raises(J.JTError) as e:
        _plan(configs.network("bn60"), max_clique_entries=1000)
    assert e.value.status == J.JT_ETOOBIG


def test_algorithmic_bytes_formula():
    net = configs.network("bn60")
    info = _plan(net).info()
    expect = (8 * info["sum_clique_entries"] + 16 * info["sum_sep_entries"] + 4 * net.n
              + 8 * info["sum_card"] + 8)
    assert info["algorithmic_bytes_per_case"] == expect


@pytest.mark.parametrize("name", ["bn20", "bn60", "bn110", "bn420", "bn1000"])
def test_evidence_placement_smallest_table(name):
    """Each variable's evidence indicator enters the smallest table holding
    it; an upward separator wins ties (Hugin enters evidence into one table;
    multiplying a child's message by the indicator before the parent absorbs
    it is the same product).  Recount the separator placements from the
    plan's cliques."""
    net = configs.network(name)
    p = _plan(net)
    cl, info = _structure(p)
    size = lambda vs: int(np.prod([net.card[v] for v in vs])) if vs else 1
    expect = 0
    for v in range(net.n):
        best = None  # (cost, is_sep)
        for vars_, par, _ in cl:
            if v not in vars_:
                continue
            up = [x for x in vars_ if par >= 0 and x in cl[par][0]]
            if v in up and (best is None or size(up) < best[0] or (size(up) == best[0] and not best[1])):
                best = (size(up), True)
            if best is None or size(vars_) < best[0]:
                best = (size(vars_), False)
        expect += best[1]
    assert info["separator_evidence_vars"] == expect
    assert expect > 0


def test_schedule_option():
    net = configs.network("bn60")
    flow = J.Plan(net, host_only=1).info()
    layers = J.Plan(net, host_only=1, schedule=J.JT_SCHEDULE_LAYERS).info()
    assert flow["kernels_per_chunk"] == 5          # evidence, two passes, log P(e), posteriors
    assert layers["kernels_per_chunk"] == 3 + 2 * layers["n_levels"]
    with pytest.raises(J.JTError) as e:
        J.Plan(net, host_only=1, schedule=7)
    assert e.value.status == J.JT_EINVAL
    with pytest.raises(J.JTError) as e:
        J.Plan(net, host_only=1, stall_clique=layers["n_cliques"] + 1)
    assert e.value.status == J.JT_EINVAL


def test_rescale_option():
    net = configs.network("bn20")
    assert J.default_opts().rescale == 1                 # power-of-two rescaling by default
    J.Plan(net, host_only=1, rescale=0)
    for bad in (2, -1):
        with pytest.raises(J.JTError) as e:
            J.Plan(net, host_only=1, rescale=bad)
        assert e.value.status == J.JT_EINVAL


def test_observed_set_option():
    """A plan specialised to an observed set leaves those variables out of
    every clique and separator table: the tables shrink by the product of
    their cardinalities over each clique holding them; the base tables keep
    the full layout."""
    net = configs.network("bn60")
    full = _plan(net).info()
    obs = [2, 15, 18, 29, 35, 46]
    p = _plan(net, observed_set=obs)
    info = p.info()
    assert info["sliced_vars"] == len(obs)
    assert info["n_cliques"] == full["n_cliques"]
    assert info["n_vars"] == net.n and info["sum_card"] == full["sum_card"] == int(np.sum(net.card))
    assert info["sum_clique_entries"] < full["sum_clique_entries"]
    size = lambda vs: int(np.prod([net.card[v] for v in vs])) if vs else 1
    total = 0
    for c in range(info["n_cliques"]):
        vars_, _, _ = p.clique(c)
        assert not set(vars_) & set(obs)
        total += size(vars_)
    assert total == info["sum_clique_entries"]
    for bad in ([3, 3], [60], [-1]):
        with pytest.raises(J.JTError) as e:
            _plan(net, observed_set=bad)
        assert e.value.status == J.JT_EINVAL


def _ancestral_closure(net, roots):
    keep, stack = set(), list(roots)
    while stack:
        v = stack.pop()
        if v not in keep:
            keep.add(v)
            stack.extend(int(p) for p in net.parents_of(v))
    return keep


@pytest.mark.parametrize("name,q,o", [("bn60", [41, 50], [3, 17]), ("bn60", [59], []),
                                      ("bn1000", [10, 500, 990], [20, 700]), ("bn110", [100], [5])])
def test_query_set_pruning(name, q, o):
    """A plan pruned to a query set keeps the query set, the observed set and
    their ancestors (every other variable is barren); evidence and posterior
    rows keep the full network's layout."""
    net = configs.network(name)
    p = _plan(net, query_set=q, observed_set=o)
    info = p.info()
    keep = _ancestral_closure(net, q + o)
    assert info["pruned_vars"] == net.n - len(keep)
    assert info["n_vars"] == net.n and info["sum_card"] == int(np.sum(net.card))
    held = set()
    for c in range(info["n_cliques"]):
        held |= set(p.clique(c)[0])
    assert held == keep - set(o)          # the observed set is also sliced out of the tables
    for bad in ([3, 3], [net.n], [-2]):
        with pytest.raises(J.JTError) as e:
            _plan(net, query_set=bad)
        assert e.value.status == J.JT_EINVAL


def test_query_set_keeping_everything_is_the_full_plan():
    net = configs.network("bn20")
    sinks = [v for v in range(net.n) if all(v not in net.parents_of(u) for u in range(net.n))]
    a, b = _plan(net, query_set=sinks).info(), _plan(net).info()
    assert a["pruned_vars"] == 0 and a["sum_clique_entries"] == b["sum_clique_entries"]

"""The five synthetic workloads (networks + evidence recipes).

Each recipe stands in for the paper's evaluation networks (Section 3, Table 1:
bnlearn networks, 2000 random cases, 20 % observed), which are not available
here.  The network seed of the rejection-sampled workloads (the first seed,
counting up from 0, whose junction tree satisfies the stated largest-clique
bound under min-fill triangulation) is stored in ``seeds.json``; that file is
written by ``select_seeds.py``.

Workloads:
  bn20   20 binary variables, 0-2 parents from the previous 6, Dirichlet(1),
         seed 0; 100 cases, 20 % observed.  Small enough for brute force.
  bn60   60 variables, cardinality in {2..5}, 0-3 parents from the previous 8,
         Dirichlet(1); largest clique <= 1e5 entries; 4096 cases, 10 % observed.
  bn110  110 variables, hub variable 0 with 60 states added as a parent of
         40 % of the nodes, others cardinality {2..8}, 0-3 parents from the
         previous 10, Dirichlet(0.5); largest clique <= 2e6; 8192 cases, 15 %.
  bn420  420 variables, cardinality {2,3,4}, 1-4 parents (node 0 none) from
         the previous 14, Dirichlet(1); largest clique in [4e6, 1.6e7];
         5 % observed; batch size set by the table-arena budget.
  bn1000 1000 ternary variables, 0-2 parents from the previous 5, Dirichlet(1)
         (many small cliques; one of the resident plans of the serving mix).
"""
from __future__ import annotations

import json
import os

from .bn import random_network, sample_cases

_HERE = os.path.dirname(os.path.abspath(__file__))

RECIPES = {
    "bn20": dict(n=20, card_choices=[2], k_range=(0, 2), window=6, alpha=1.0,
                 cases=100, observed=0.2, clique_bound=None),
    "bn60": dict(n=60, card_choices=[2, 3, 4, 5], k_range=(0, 3), window=8,
                 alpha=1.0, cases=4096, observed=0.1,
                 clique_bound=(0, 100_000)),
    "bn110": dict(n=110, card_choices=[2, 3, 4, 5, 6, 7, 8], k_range=(0, 3),
                  window=10, alpha=0.5, hub_card=60, hub_frac=0.4, cases=8192,
                  observed=0.15, clique_bound=(0, 2_000_000)),
    "bn420": dict(n=420, card_choices=[2, 3, 4], k_range=(1, 4), window=14,
                  alpha=1.0, root_has_parents=False, cases=None, observed=0.05,
                  clique_bound=(4_000_000, 16_000_000)),
    "bn1000": dict(n=1000, card_choices=[3], k_range=(0, 2), window=5,
                   alpha=1.0, cases=None, observed=(0.05, 0.30),
                   clique_bound=None),
}

# evidence seeds are separate from network seeds
EVIDENCE_SEED = {"bn20": 100, "bn60": 101, "bn110": 102, "bn420": 103,
                 "bn1000": 104}

SEED_FILE = os.path.join(_HERE, "seeds.json")


def stored_seeds() -> dict:
    if not os.path.exists(SEED_FILE):
        return {"bn20": 0, "bn1000": 0}
    with open(SEED_FILE) as f:
        return json.load(f)


def network_kwargs(name: str) -> dict:
    r = RECIPES[name]
    kw = dict(n=r["n"], card_choices=r["card_choices"], k_range=r["k_range"],
              window=r["window"], alpha=r["alpha"])
    for opt in ("hub_card", "hub_frac", "root_has_parents"):
        if opt in r:
            kw[opt] = r[opt]
    return kw


def network(name: str, seed: int | None = None):
    """The workload's network; ``seed`` overrides the stored seed."""
    if seed is None:
        seeds = stored_seeds()
        if name not in seeds:
            raise KeyError(f"no stored seed for {name}; run synth/select_seeds.py")
        seed = seeds[name]
    return random_network(seed=seed, **network_kwargs(name))


def evidence(name: str, net, n_cases: int | None = None, seed: int | None = None):
    r = RECIPES[name]
    if n_cases is None:
        n_cases = r["cases"]
    if seed is None:
        seed = EVIDENCE_SEED[name]
    return sample_cases(net, n_cases, r["observed"], seed)

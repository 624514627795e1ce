"""Seeded synthetic inputs (networks, CPTs, evidence) shared by tests and bench."""
from .bn import Network, make_network, random_network, sample_cases, empty_evidence, round_half_up
from . import configs

__all__ = ["Network", "make_network", "random_network", "sample_cases",
           "empty_evidence", "round_half_up", "configs"]

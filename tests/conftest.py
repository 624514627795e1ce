import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# The property-based modules need hypothesis; where it is not installed they
# are left out of collection (rather than reported as skipped modules).
collect_ignore = []
if importlib.util.find_spec("hypothesis") is None:
    collect_ignore += ["test_compile_hypothesis.py", "test_oracle_hypothesis.py"]


def pytest_report_header(config):
    if collect_ignore:
        return "hypothesis not installed: " + ", ".join(collect_ignore) + " not collected"
    return None


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test, run with JT_SLOW_TESTS=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("JT_SLOW_TESTS") == "1":
        return
    skip = pytest.mark.skip(reason="slow; set JT_SLOW_TESTS=1")
    for it in items:
        if "slow" in it.keywords:
            it.add_marker(skip)

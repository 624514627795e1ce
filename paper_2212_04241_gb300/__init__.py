"""GB300-native junction-tree exact inference for Bayesian networks.

The compute path lives in ``_build/libjt.so`` (C ABI: include/jt.h); this
package is a thin binding around it.  Build with ``build.build()``.
"""
from . import build  # noqa: F401

__all__ = ["build", "jt"]


def __getattr__(name):
    if name == "jt":
        from . import jt as _jt
        return _jt
    raise AttributeError(name)

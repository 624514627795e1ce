"""FP64 junction-tree oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and it
shares no code with the GPU library (see ``jt_oracle.c`` for what it computes
and which passages of the paper it follows).

Layout of the outputs (same as the GPU library's C ABI so the two can be
compared element by element):
  log_pe     float64 [n_cases]
  posteriors float64 [n_cases, sum(card)], variable v's states at
             offsets sum(card[:v]) .. sum(card[:v+1]); point masses for
             observed variables; NaN when P(e) = 0
  status     int32 [n_cases]: 0 ok, 1 zero-probability evidence
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jt_oracle.c")


def lib_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_mut{mutant}.so"
    return os.path.join(_HERE, "_build", name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no fast-math) into a shared library."""
    out = lib_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC",
           f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


_libs: dict = {}


def _load(mutant: int = 0):
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant))
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.orc_compile.argtypes = [I, P, P, P, P, I, I, ctypes.POINTER(P)]
        lib.orc_compile.restype = I
        lib.orc_free.argtypes = [P]
        lib.orc_free.restype = None
        lib.orc_info.argtypes = [P, P]
        lib.orc_clique.argtypes = [P, I, P, P]
        lib.orc_infer.argtypes = [P, P, I, P, P]
        lib.orc_calibrated.argtypes = [P, P, I, I, P, P]
        lib.orc_infer_batch.argtypes = [P, I, P, I, P, P, P, I]
        _libs[mutant] = lib
    return _libs[mutant]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


class Oracle:
    """Compiled junction tree of one network.

    elim: "minfill" or "mindegree"; root: "largest", "center" or a clique id.
    """

    def __init__(self, net, elim: str = "minfill", root="largest", mutant: int = 0):
        self._lib = _load(mutant)
        self.net = net
        self._card = np.ascontiguousarray(net.card, dtype=np.int32)
        self._pptr = np.ascontiguousarray(net.parent_ptr, dtype=np.int32)
        self._par = np.ascontiguousarray(net.parents, dtype=np.int32)
        if self._par.size == 0:
            self._par = np.zeros(1, dtype=np.int32)
        self._cpt = np.ascontiguousarray(net.cpt, dtype=np.float64)
        er = {"minfill": 0, "mindegree": 1}[elim]
        rr = {"largest": 0, "center": 1}.get(root) if isinstance(root, str) else int(root) + 2
        h = ctypes.c_void_p()
        st = self._lib.orc_compile(int(net.n), _ptr(self._card), _ptr(self._pptr),
                                   _ptr(self._par), _ptr(self._cpt), er, rr, ctypes.byref(h))
        if st != 0:
            raise OracleError(f"orc_compile failed with {st}")
        self._h = h
        info = np.zeros(7, dtype=np.int64)
        self._lib.orc_info(self._h, _ptr(info))
        (self.n_cliques, self.root, self.height, self.sum_clique, self.max_clique,
         self.sum_sep, self.sum_card) = (int(x) for x in info)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    def clique(self, c: int):
        vars_ = np.zeros(64, dtype=np.int32)
        parent = ctypes.c_int()
        nv = self._lib.orc_clique(self._h, c, _ptr(vars_), ctypes.byref(parent))
        return [int(v) for v in vars_[:nv]], int(parent.value)

    def cliques(self):
        return [self.clique(c) for c in range(self.n_cliques)]

    def infer(self, evidence, rescale: bool = True, threads: int = 1):
        ev = np.ascontiguousarray(np.atleast_2d(evidence), dtype=np.int32)
        assert ev.shape[1] == self.net.n
        m = ev.shape[0]
        log_pe = np.zeros(m, dtype=np.float64)
        post = np.zeros((m, self.sum_card), dtype=np.float64)
        status = np.zeros(m, dtype=np.int32)
        self._lib.orc_infer_batch(self._h, m, _ptr(ev), int(rescale), _ptr(log_pe),
                                  _ptr(post), _ptr(status), int(threads))
        return log_pe, post, status

    def calibrated(self, evidence, c: int, rescale: bool = True):
        """Calibrated potential of clique c as an ndarray with one axis per
        clique variable (ascending ids), in true scale."""
        ev = np.ascontiguousarray(evidence, dtype=np.int32)
        vars_, _ = self.clique(c)
        shape = [int(self.net.card[v]) for v in vars_]
        t = np.zeros(int(np.prod(shape)), dtype=np.float64)
        ex = ctypes.c_long()
        self._lib.orc_calibrated(self._h, _ptr(ev), int(rescale), c, _ptr(t), ctypes.byref(ex))
        return vars_, np.ldexp(t.reshape(shape), int(ex.value))

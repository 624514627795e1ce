"""Thin ctypes binding of the C ABI in include/jt.h (argument marshalling only).

Every step of inference runs inside libjt.so (host compiler + CUDA kernels);
this module only converts numpy arrays / torch tensors to pointers.  There is
no CPU fallback: if the library is missing or fails to load, importing this
module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjt.so")

JT_OK, JT_EINVAL, JT_ECYCLE, JT_ETOOBIG, JT_ENOMEM, JT_ECUDA, JT_ETIMEOUT, JT_EBUSY, JT_ENOTFOUND = range(9)
JT_CASE_OK, JT_CASE_ZERO_EVIDENCE, JT_CASE_BAD_EVIDENCE, JT_CASE_INCOMPLETE = 0, 1, 2, 3
JT_ROOT_LARGEST, JT_ROOT_MIN_HEIGHT = 0, 1
JT_SCHEDULE_DATAFLOW, JT_SCHEDULE_LAYERS = 0, 1
JT_SIZE_BUCKETS = 32


class JTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class CompileOpts(ctypes.Structure):
    _fields_ = [("root_rule", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("cases_per_thread", ctypes.c_int32), ("rows_per_cta", ctypes.c_int32),
                ("max_clique_entries", ctypes.c_int64), ("arena_bytes", ctypes.c_int64),
                ("use_graphs", ctypes.c_int32), ("items_per_tile", ctypes.c_int32),
                ("items_per_tile_distribute", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("wait_limit_us", ctypes.c_int32), ("stall_clique", ctypes.c_int32),
                ("n_observed_set", ctypes.c_int32), ("observed_set", ctypes.c_void_p),
                ("rescale", ctypes.c_int32), ("n_query_set", ctypes.c_int32), ("query_set", ctypes.c_void_p),
                ("collect_rows_by_bucket", ctypes.c_int32 * JT_SIZE_BUCKETS),
                ("distribute_rows_by_bucket", ctypes.c_int32 * JT_SIZE_BUCKETS),
                ("fuse_distribute", ctypes.c_int32), ("recompute_psi", ctypes.c_int32),
                ("collect_prefetch", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("n_cliques", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("root", ctypes.c_int32),
                ("sum_clique_entries", ctypes.c_int64), ("max_clique_entries", ctypes.c_int64),
                ("sum_sep_entries", ctypes.c_int64), ("sum_card", ctypes.c_int64),
                ("tile_cases", ctypes.c_int32), ("chunk_cases", ctypes.c_int32),
                ("arena_bytes", ctypes.c_int64), ("static_device_bytes", ctypes.c_int64),
                ("collect_items", ctypes.c_int64), ("distribute_items", ctypes.c_int64),
                ("algorithmic_bytes_per_case", ctypes.c_double),
                ("kernels_per_chunk", ctypes.c_int32), ("sliced_vars", ctypes.c_int32),
                ("separator_evidence_vars", ctypes.c_int32), ("pruned_vars", ctypes.c_int32),
                ("budget_chunk_cases", ctypes.c_int32),
                ("collect_rows_by_bucket", ctypes.c_int32 * JT_SIZE_BUCKETS),
                ("distribute_rows_by_bucket", ctypes.c_int32 * JT_SIZE_BUCKETS),
                ("collect_entries_by_bucket", ctypes.c_int64 * JT_SIZE_BUCKETS),
                ("distribute_entries_by_bucket", ctypes.c_int64 * JT_SIZE_BUCKETS)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if isinstance(v, ctypes.Array) else v
        return out


EXPORTS = ["jt_default_opts", "jt_compile", "jt_autotune", "jt_infer", "jt_infer_device", "jt_infer_plain", "jt_infer_cpu",
           "jt_profile", "jt_debug_stall",
           "jt_plan_info", "jt_plan_clique", "jt_plan_free", "jt_status_string", "jt_last_error",
           "jt_server_create", "jt_server_add_plan", "jt_server_add_plan_rolling", "jt_submit", "jt_poll", "jt_server_drain",
           "jt_server_stats", "jt_server_plan_stats", "jt_server_set_priority", "jt_server_reset_latency",
           "jt_server_destroy"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libjt.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "jt_default_opts": ([ctypes.POINTER(CompileOpts)], None),
        "jt_compile": ([I32, P, P, P, P, ctypes.POINTER(CompileOpts), ctypes.POINTER(P)], ctypes.c_int),
        "jt_autotune": ([I32, P, P, P, P, ctypes.POINTER(CompileOpts), I32, ctypes.POINTER(CompileOpts),
                         ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "jt_infer": ([P, I32, P, P, P, P, P], ctypes.c_int),
        "jt_infer_device": ([P, I32, P, P, P, P, P], ctypes.c_int),
        "jt_infer_plain": ([P, I32, P, P, P, P, P], ctypes.c_int),
        "jt_infer_cpu": ([P, I32, P, P, P, P, I32], ctypes.c_int),
        "jt_profile": ([P, I32, P, P, P, P, P, P], ctypes.c_int),
        "jt_debug_stall": ([P, I32], ctypes.c_int),
        "jt_plan_info": ([P, ctypes.POINTER(PlanInfo)], ctypes.c_int),
        "jt_plan_clique": ([P, I32, P, P, P, P], ctypes.c_int),
        "jt_plan_free": ([P], None),
        "jt_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "jt_last_error": ([], ctypes.c_char_p),
        "jt_server_create": ([I64, I32, I32, ctypes.POINTER(P)], ctypes.c_int),
        "jt_server_add_plan": ([P, P, ctypes.POINTER(I32)], ctypes.c_int),
        "jt_server_add_plan_rolling": ([P, P, I32, ctypes.POINTER(I32)], ctypes.c_int),
        "jt_submit": ([P, I32, P, P, I32, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
        "jt_poll": ([P, ctypes.c_uint64, P, P, P], ctypes.c_int),
        "jt_server_drain": ([P], ctypes.c_int),
        "jt_server_stats": ([P, P], ctypes.c_int),
        "jt_server_plan_stats": ([P, I32, P], ctypes.c_int),
        "jt_server_reset_latency": ([P], ctypes.c_int),
        "jt_server_set_priority": ([P, I32, I32], ctypes.c_int),
        "jt_server_destroy": ([P], None),
    }
    for name in EXPORTS:
        f = getattr(lib, name)
        f.argtypes, f.restype = sig[name]
    return lib


lib = _load()


def _check(st: int):
    if st != JT_OK:
        raise JTError(st, f"{lib.jt_status_string(st).decode()}: {lib.jt_last_error().decode()}")


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def default_opts(**kw) -> CompileOpts:
    """jt_compile_opts with the defaults, then the given fields.  observed_set
    and query_set take sequences of variable ids (kept alive with the
    returned struct)."""
    o = CompileOpts()
    lib.jt_default_opts(ctypes.byref(o))
    obs = kw.pop("observed_set", None)
    qry = kw.pop("query_set", None)
    for k, v in kw.items():
        if k in ("collect_rows_by_bucket", "distribute_rows_by_bucket"):
            arr = getattr(o, k)
            for i, x in enumerate(v):
                arr[i] = int(x)
        else:
            setattr(o, k, v)
    if obs is not None and len(obs) > 0:
        arr = np.ascontiguousarray(obs, dtype=np.int32)
        o._observed_keepalive = arr
        o.n_observed_set = int(arr.size)
        o.observed_set = arr.ctypes.data
    if qry is not None and len(qry) > 0:
        arr = np.ascontiguousarray(qry, dtype=np.int32)
        o._query_keepalive = arr
        o.n_query_set = int(arr.size)
        o.query_set = arr.ctypes.data
    return o


def _net_arrays(net):
    card = np.ascontiguousarray(net.card, dtype=np.int32)
    pptr = np.ascontiguousarray(net.parent_ptr, dtype=np.int32)
    par = np.ascontiguousarray(net.parents, dtype=np.int32)
    if par.size == 0:
        par = np.zeros(1, dtype=np.int32)
    cpt = np.ascontiguousarray(net.cpt, dtype=np.float64)
    return card, pptr, par, cpt


def autotune(net, n_cases: int, **opts):
    """jt_autotune: the fastest tile shape for this network and batch size.
    Returns (options dict for Plan(...), ns per case)."""
    card, pptr, par, cpt = _net_arrays(net)
    base = default_opts(**opts)
    best = CompileOpts()
    ns = ctypes.c_double()
    _check(lib.jt_autotune(int(net.n), _ptr(card), _ptr(pptr), _ptr(par), _ptr(cpt), ctypes.byref(base),
                           int(n_cases), ctypes.byref(best), ctypes.byref(ns)))
    out = {k: getattr(best, k) for k in ("root_rule", "cases_per_thread", "rows_per_cta", "items_per_tile",
                                           "items_per_tile_distribute", "use_graphs", "arena_bytes",
                                           "max_clique_entries", "schedule", "rescale", "fuse_distribute",
                                           "recompute_psi", "collect_prefetch")}
    for k in ("collect_rows_by_bucket", "distribute_rows_by_bucket"):
        out[k] = [int(x) for x in getattr(best, k)]
    for k in ("observed_set", "query_set"):
        if opts.get(k) is not None:
            out[k] = list(opts[k])
    return out, ns.value


class Plan:
    """A compiled network (jt_compile).  Keyword arguments set jt_compile_opts."""

    def __init__(self, net, **opts):
        self.net = net
        self.n = int(net.n)
        card = np.ascontiguousarray(net.card, dtype=np.int32)
        pptr = np.ascontiguousarray(net.parent_ptr, dtype=np.int32)
        par = np.ascontiguousarray(net.parents, dtype=np.int32)
        if par.size == 0:
            par = np.zeros(1, dtype=np.int32)
        cpt = np.ascontiguousarray(net.cpt, dtype=np.float64)
        o = default_opts(**opts)
        h = ctypes.c_void_p()
        _check(lib.jt_compile(self.n, _ptr(card), _ptr(pptr), _ptr(par), _ptr(cpt), ctypes.byref(o),
                              ctypes.byref(h)))
        self._h = h
        self.sum_card = int(self.info()["sum_card"])

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.jt_plan_free(self._h)
        self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = PlanInfo()
        _check(lib.jt_plan_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    def clique(self, c: int):
        nv = ctypes.c_int32()
        vars_ = np.zeros(64, dtype=np.int32)
        parent = ctypes.c_int32()
        depth = ctypes.c_int32()
        _check(lib.jt_plan_clique(self._h, c, ctypes.byref(nv), _ptr(vars_), ctypes.byref(parent),
                                  ctypes.byref(depth)))
        return [int(v) for v in vars_[:nv.value]], int(parent.value), int(depth.value)

    def _outputs(self, m):
        return (np.zeros(m, dtype=np.float64), np.zeros((m, self.sum_card), dtype=np.float64),
                np.zeros(m, dtype=np.int32))

    def infer(self, evidence, stream=None, out=None):
        """Batched FP32 path, host buffers (jt_infer).  ``out`` = (log_pe,
        posteriors, status) preallocated C-contiguous arrays of float64 [n],
        float64 [n, sum_card] and int32 [n]; page-locked ones are copied to
        and from the device directly."""
        ev = np.ascontiguousarray(np.atleast_2d(evidence), dtype=np.int32)
        assert ev.shape[1] == self.n
        if out is None:
            lp, post, st = self._outputs(ev.shape[0])
        else:
            lp, post, st = out
            m = ev.shape[0]
            assert lp.dtype == np.float64 and lp.shape == (m,) and lp.flags.c_contiguous
            assert post.dtype == np.float64 and post.shape == (m, self.sum_card) and post.flags.c_contiguous
            assert st.dtype == np.int32 and st.shape == (m,) and st.flags.c_contiguous
        _check(lib.jt_infer(self._h, ev.shape[0], _ptr(ev), _ptr(lp), _ptr(post), _ptr(st), stream))
        return lp, post, st

    def infer_plain(self, evidence, stream=None):
        """Plain per-case FP64 path, host buffers (jt_infer_plain)."""
        ev = np.ascontiguousarray(np.atleast_2d(evidence), dtype=np.int32)
        assert ev.shape[1] == self.n
        lp, post, st = self._outputs(ev.shape[0])
        _check(lib.jt_infer_plain(self._h, ev.shape[0], _ptr(ev), _ptr(lp), _ptr(post), _ptr(st), stream))
        return lp, post, st

    def infer_cpu(self, evidence, threads=0):
        """Multi-core CPU comparator in the paper's layer-parallel style, host
        buffers (jt_infer_cpu); threads = 0 uses every hardware thread."""
        ev = np.ascontiguousarray(np.atleast_2d(evidence), dtype=np.int32)
        assert ev.shape[1] == self.n
        lp, post, st = self._outputs(ev.shape[0])
        _check(lib.jt_infer_cpu(self._h, ev.shape[0], _ptr(ev), _ptr(lp), _ptr(post), _ptr(st), int(threads)))
        return lp, post, st

    def infer_device(self, d_evidence, d_log_pe, d_post, d_status, n_cases=None, stream=None):
        """Batched FP32 path, device buffers (jt_infer_device).  Arguments are
        torch CUDA tensors (or raw device addresses); ``stream`` is a
        cudaStream_t value (e.g. torch.cuda.current_stream().cuda_stream)."""
        if n_cases is None:
            n_cases = int(d_evidence.shape[0])
        s = None if stream is None else ctypes.c_void_p(int(stream))
        _check(lib.jt_infer_device(self._h, int(n_cases), _ptr(d_evidence), _ptr(d_log_pe), _ptr(d_post),
                                   _ptr(d_status), s))

    def debug_stall(self, enabled: bool):
        """Testing hook (jt_debug_stall): turn the compiled stall_clique stall on or off."""
        _check(lib.jt_debug_stall(self._h, 1 if enabled else 0))

    def profile(self, d_evidence, d_log_pe, d_post, d_status, n_cases=None, stream=None):
        """Instrumented run (jt_profile): per-kernel-type device milliseconds."""
        if n_cases is None:
            n_cases = int(d_evidence.shape[0])
        out = np.zeros(6, dtype=np.float64)
        s = None if stream is None else ctypes.c_void_p(int(stream))
        _check(lib.jt_profile(self._h, int(n_cases), _ptr(d_evidence), _ptr(d_log_pe), _ptr(d_post),
                              _ptr(d_status), s, _ptr(out)))
        return {"collect_ms": out[0], "distribute_ms": out[1], "other_ms": out[2],
                "collect_launches": int(out[3]), "distribute_launches": int(out[4]), "total_ms": out[5]}


class Server:
    """Continuous-batching request loop (jt_server_*)."""

    def __init__(self, arena_bytes=0, max_batch=256, max_inflight=8):
        h = ctypes.c_void_p()
        _check(lib.jt_server_create(int(arena_bytes), int(max_batch), int(max_inflight), ctypes.byref(h)))
        self._h = h
        self._plans = []

    def add_plan(self, plan: Plan, rolling_tiles: int = 0) -> int:
        """Register a plan: batch slots (jt_server_add_plan), or iteration-level
        batching over `rolling_tiles` resident tiles (jt_server_add_plan_rolling)."""
        pid = ctypes.c_int32()
        if rolling_tiles > 0:
            _check(lib.jt_server_add_plan_rolling(self._h, plan.handle, int(rolling_tiles), ctypes.byref(pid)))
        else:
            _check(lib.jt_server_add_plan(self._h, plan.handle, ctypes.byref(pid)))
        self._plans.append(plan)
        return int(pid.value)

    def submit(self, plan_id: int, evidence, query=None) -> int:
        ev = np.ascontiguousarray(evidence, dtype=np.int32)
        t = ctypes.c_uint64()
        if query is None:
            _check(lib.jt_submit(self._h, plan_id, _ptr(ev), None, 0, ctypes.byref(t)))
        else:
            q = np.ascontiguousarray(query, dtype=np.int32)
            _check(lib.jt_submit(self._h, plan_id, _ptr(ev), _ptr(q), int(q.size), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, out_len: int):
        """(log_pe, posteriors, status) or None while pending."""
        lp = ctypes.c_double()
        st = ctypes.c_int32()
        post = np.zeros(out_len, dtype=np.float64)
        r = lib.jt_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(lp), _ptr(post), ctypes.byref(st))
        if r == JT_EBUSY:
            return None
        _check(r)
        return lp.value, post, st.value

    def drain(self):
        _check(lib.jt_server_drain(self._h))

    def stats(self) -> dict:
        out = np.zeros(9, dtype=np.int64)
        _check(lib.jt_server_stats(self._h, _ptr(out)))
        keys = ["completed", "batches", "largest_batch", "peak_arena_bytes", "p50_ns", "p99_ns", "outstanding",
                "slot_creations", "slot_evictions"]
        return dict(zip(keys, (int(x) for x in out)))

    def reset_latency(self):
        _check(lib.jt_server_reset_latency(self._h))

    def set_priority(self, plan_id: int, high: bool = True):
        """Run the plan's batches on the high-priority streams (jt_server_set_priority)."""
        _check(lib.jt_server_set_priority(self._h, int(plan_id), 1 if high else 0))

    def plan_stats(self, plan_id: int) -> dict:
        out = np.zeros(4, dtype=np.int64)
        _check(lib.jt_server_plan_stats(self._h, int(plan_id), _ptr(out)))
        return dict(zip(["completed", "batches", "p50_ns", "p99_ns"], (int(x) for x in out)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.jt_server_destroy(self._h)
        self._h = None

    def __del__(self):
        self.close()

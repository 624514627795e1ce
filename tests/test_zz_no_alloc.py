"""jt_infer_device_noalloc against jt_infer_device (GPU, through the C ABI).

The no-allocation variant is for callers that cannot allocate device memory
while serving (memory owned by another allocator, loops that cannot afford
cudaMalloc's device-wide synchronisation, no allocation after start-up).
It runs the same kernels in the same order as the regular entry point, so
its outputs must equal that entry point's bit for bit, call after call,
although every call reuses the same fixed device array.  This file is named
to be collected last.
"""
import ctypes

import numpy as np
import pytest

from synth import configs
from tests.common import LOGPE_REL32, POST_TOL32, max_logpe_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402

_fn = J.lib.jt_infer_device_noalloc
_fn.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 5
_fn.restype = ctypes.c_int


def _buffers(n, sum_card):
    return (torch.empty(n, dtype=torch.float64, device="cuda"),
            torch.empty((n, sum_card), dtype=torch.float64, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


def _noalloc(plan, d_ev, lp, post, st):
    s = torch.cuda.current_stream().cuda_stream
    return _fn(plan.handle, int(d_ev.shape[0]), ctypes.c_void_p(d_ev.data_ptr()),
               ctypes.c_void_p(lp.data_ptr()), ctypes.c_void_p(post.data_ptr()),
               ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(s))


# A case tile must fit the 64 MiB array: narrower tiles (fewer cases per
# thread) keep the per-tile tables of the larger networks small enough.
@pytest.mark.parametrize("name,n_cases,cpt", [("bn60", 300, 2), ("bn20", 100, 8), ("bn1000", 777, 4)])
def test_noalloc_matches_regular_entry_point_twice(name, n_cases, cpt):
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n_cases)
    plan = J.Plan(net, cases_per_thread=cpt)
    d_ev = torch.from_numpy(ev).cuda()
    ref = _buffers(n_cases, plan.sum_card)
    plan.infer_device(d_ev, *ref, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    rlp, rpost, rst = (t.cpu().numpy() for t in ref)
    for call in range(2):   # the array keeps the previous call's contents
        out = _buffers(n_cases, plan.sum_card)
        for t in out:
            t.fill_(-7)
        assert _noalloc(plan, d_ev, *out) == J.JT_OK, J.lib.jt_last_error().decode()
        torch.cuda.synchronize()
        lp, post, st = (t.cpu().numpy() for t in out)
        assert np.array_equal(st, rst), f"call {call}: status mismatch"
        # the same kernels in the same order: bitwise equal (the tolerance
        # check states the bound the library promises in any case)
        assert np.array_equal(lp, rlp, equal_nan=True), f"call {call}: log P(e) differs"
        assert np.array_equal(post, rpost, equal_nan=True), f"call {call}: posteriors differ"
        ok = rst == 0
        assert np.max(np.abs(post[ok] - rpost[ok])) <= POST_TOL32, f"call {call}"
        assert max_logpe_err(lp[ok], rlp[ok]) <= LOGPE_REL32, f"call {call}"


def test_noalloc_refuses_plan_larger_than_scratch():
    net = configs.network("bn110")       # ~9 GB of tables per case tile
    plan = J.Plan(net)
    ev = configs.evidence("bn110", net, n_cases=4)
    d_ev = torch.from_numpy(ev).cuda()
    out = _buffers(4, plan.sum_card)
    r = _noalloc(plan, d_ev, *out)
    assert r == J.JT_ENOMEM
    assert "static scratch" in J.lib.jt_last_error().decode()


def test_noalloc_pruned_and_sliced_plan():
    """Evidence and posterior rows of a pruned plan keep the full network's
    layout on this entry point too."""
    from synth.bn import sample_cases
    net = configs.network("bn1000")
    q, obs = [999, 400], [5, 600, 700]
    x = sample_cases(net, 333, 1.0, seed=8)
    ev = np.full_like(x, -1, dtype=np.int32)
    ev[:, obs] = x[:, obs]
    plan = J.Plan(net, query_set=q, observed_set=obs)
    assert plan.info()["pruned_vars"] > 0
    d_ev = torch.from_numpy(ev).cuda()
    ref = _buffers(len(ev), plan.sum_card)
    plan.infer_device(d_ev, *ref, stream=torch.cuda.current_stream().cuda_stream)
    out = _buffers(len(ev), plan.sum_card)
    assert _noalloc(plan, d_ev, *out) == J.JT_OK, J.lib.jt_last_error().decode()
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy(), equal_nan=True)

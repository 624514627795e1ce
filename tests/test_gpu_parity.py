"""GPU parity: the CUDA paths (through the C ABI) against the FP64 oracle.

* plain FP64 path: every case of the 20-variable workload and samples of the
  others, FP64 tolerance;
* batched FP32 path: max abs posterior error <= 1e-5 and
  |d log P(e)| <= 1e-6 * max(1, |log P(e)|) against the oracle, on every
  workload, in the launch configuration the benchmark uses (default options,
  full batch sizes, chunked by the arena), plus edge cases: empty and ragged
  batches, zero-probability and invalid evidence, no evidence, tiny random
  networks, forced multi-chunk batches, every cases-per-thread width.
"""
import numpy as np
import pytest

import oracle
from synth import configs, empty_evidence
from synth.bn import tiny_random_network, sample_cases
from tests.common import assert_parity32, golden_cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402

ORACLE_THREADS = 16


def _oracle(net, ev):
    return oracle.Oracle(net).infer(ev, threads=ORACLE_THREADS)


def test_bn20_plain_all_cases():
    net = configs.network("bn20")
    ev = configs.evidence("bn20", net)
    p = J.Plan(net, root_rule=J.JT_ROOT_LARGEST)
    lp, post, st = p.infer_plain(ev)
    olp, opost, ost = _oracle(net, ev)
    assert np.array_equal(st, ost)
    np.testing.assert_allclose(lp, olp, rtol=0, atol=1e-12)
    np.testing.assert_allclose(post, opost, rtol=0, atol=1e-12)


@pytest.mark.parametrize("cpt", [1, 2, 4, 8])
def test_bn20_batched_all_cases(cpt):
    net = configs.network("bn20")
    ev = configs.evidence("bn20", net)
    p = J.Plan(net, cases_per_thread=cpt)
    assert_parity32(*p.infer(ev), *_oracle(net, ev), where=f"bn20 cpt={cpt}")


def test_bn60_full_batch_all_cases():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net)          # 4096 cases, the benchmark workload
    p = J.Plan(net)
    olp, opost, ost = _oracle(net, ev)
    perr, lerr = assert_parity32(*p.infer(ev), olp, opost, ost, where="bn60")
    print(f"bn60 max posterior err {perr:.3g}, log P(e) err {lerr:.3g}")


@pytest.mark.parametrize("opts", [dict(cases_per_thread=1), dict(cases_per_thread=2), dict(cases_per_thread=4),
                                  dict(use_graphs=0), dict(root_rule=J.JT_ROOT_LARGEST), dict(schedule=J.JT_SCHEDULE_LAYERS),
                                  dict(rows_per_cta=64), dict(rows_per_cta=4096)])
def test_bn60_option_variants(opts):
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=300)
    p = J.Plan(net, **opts)
    assert_parity32(*p.infer(ev), *_oracle(net, ev), where=str(opts))


def test_bn60_plain_sample():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=64)
    lp, post, st = J.Plan(net).infer_plain(ev)
    olp, opost, ost = _oracle(net, ev)
    assert np.array_equal(st, ost)
    np.testing.assert_allclose(lp, olp, rtol=0, atol=1e-11)
    np.testing.assert_allclose(post, opost, rtol=0, atol=1e-11)


def test_device_path_matches_host_path_bitwise():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=1000)
    p = J.Plan(net)
    lp, post, st = p.infer(ev)
    d_ev = torch.from_numpy(ev).cuda()
    d_lp = torch.empty(ev.shape[0], dtype=torch.float64, device="cuda")
    d_post = torch.empty((ev.shape[0], p.sum_card), dtype=torch.float64, device="cuda")
    d_st = torch.empty(ev.shape[0], dtype=torch.int32, device="cuda")
    p.infer_device(d_ev, d_lp, d_post, d_st, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(d_lp.cpu().numpy(), lp)
    assert np.array_equal(d_post.cpu().numpy(), post)
    assert np.array_equal(d_st.cpu().numpy(), st)


@pytest.mark.parametrize("chunks", [1, 4])
def test_pinned_host_buffers_match_pageable_bitwise(chunks):
    """jt_infer copies page-locked caller buffers directly (asynchronously,
    over every chunk); the results equal the staged pageable path bit for bit."""
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=1000)
    opts = {}
    if chunks > 1:
        probe = J.Plan(net)
        probe.infer(ev[:1])
        opts = dict(arena_bytes=2 * probe.info()["arena_bytes"])   # 1000 cases in 4 chunks of 256
    p = J.Plan(net, **opts)
    lp, post, st = p.infer(ev)
    ev_pin = torch.from_numpy(ev).pin_memory().numpy()
    out = (torch.full((1000,), -7.0, dtype=torch.float64, pin_memory=True).numpy(),
           torch.full((1000, p.sum_card), -7.0, dtype=torch.float64, pin_memory=True).numpy(),
           torch.full((1000,), -7, dtype=torch.int32, pin_memory=True).numpy())
    p.infer(ev_pin, out=out)
    assert np.array_equal(out[0], lp) and np.array_equal(out[1], post) and np.array_equal(out[2], st)


def test_result_independent_of_batch_position():
    """A case gives bit-identical results alone, in a small batch and at any
    position of a large batch (fixed per-case reduction order)."""
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=700)
    p = J.Plan(net)
    lp, post, st = p.infer(ev)
    for i in (0, 5, 127, 128, 255, 256, 699):
        a = p.infer(ev[i:i + 1])
        assert a[0][0] == lp[i] and np.array_equal(a[1][0], post[i])
    perm = np.random.default_rng(0).permutation(700)
    b = p.infer(ev[perm])
    assert np.array_equal(b[0], lp[perm]) and np.array_equal(b[1], post[perm])


@pytest.mark.parametrize("n_cases", [0, 1, 31, 127, 129, 255, 257, 513])
def test_ragged_and_empty_batches(n_cases):
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=max(n_cases, 1))[:n_cases]
    p = J.Plan(net)
    lp, post, st = p.infer(ev)
    assert lp.shape == (n_cases,)
    if n_cases:
        assert_parity32(lp, post, st, *_oracle(net, ev), where=f"n={n_cases}")


def test_forced_multi_chunk():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=1000)
    # room for two case tiles only: 1000 cases run as 4 chunks
    probe = J.Plan(net)
    probe.infer(ev[:1])
    per_tile = probe.info()["arena_bytes"]
    p = J.Plan(net, arena_bytes=2 * per_tile)
    lp, post, st = p.infer(ev)
    assert p.info()["chunk_cases"] == 2 * p.info()["tile_cases"]
    assert_parity32(lp, post, st, *_oracle(net, ev), where="multi-chunk")


def test_golden_and_special_evidence():
    for name, g, net in golden_cases():
        p = J.Plan(net)
        ev = np.asarray([c["evidence"] for c in g["cases"]], dtype=np.int32)
        lp, post, st = p.infer(ev)
        plp, ppost, pst = p.infer_plain(ev)
        offs = np.concatenate([[0], np.cumsum(net.card)])
        for i, case in enumerate(g["cases"]):
            if case["pe"] == 0.0:
                assert st[i] == J.JT_CASE_ZERO_EVIDENCE and np.isneginf(lp[i])
                assert pst[i] == J.JT_CASE_ZERO_EVIDENCE and np.isneginf(plp[i])
                assert np.all(np.isnan(post[i])) and np.all(np.isnan(ppost[i]))
                continue
            assert st[i] == 0 and pst[i] == 0
            assert abs(lp[i] - np.log(case["pe"])) <= 1e-6 * max(1, abs(np.log(case["pe"])))
            assert abs(plp[i] - np.log(case["pe"])) <= 1e-12
            for v, pv in enumerate(case["posteriors"]):
                np.testing.assert_allclose(post[i, offs[v]:offs[v + 1]], pv, atol=1e-6)
                np.testing.assert_allclose(ppost[i, offs[v]:offs[v + 1]], pv, atol=1e-12)


def test_invalid_evidence_flags_only_that_case():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=10)
    ev[3, 7] = int(net.card[7])   # out of range
    ev[6, 2] = -5
    p = J.Plan(net)
    lp, post, st = p.infer(ev)
    assert st[3] == J.JT_CASE_BAD_EVIDENCE and st[6] == J.JT_CASE_BAD_EVIDENCE
    assert np.isnan(lp[3]) and np.all(np.isnan(post[3]))
    good = [i for i in range(10) if i not in (3, 6)]
    assert_parity32(lp[good], post[good], st[good], *_oracle(net, ev[good]), where="bad-ev")
    plp, ppost, pst = p.infer_plain(ev)
    assert pst[3] == J.JT_CASE_BAD_EVIDENCE and pst[6] == J.JT_CASE_BAD_EVIDENCE


def test_no_evidence_probability_one():
    for name in ("bn60", "bn1000"):
        net = configs.network(name)
        p = J.Plan(net)
        ev = empty_evidence(net, 3)
        lp, post, st = p.infer(ev)
        assert np.all(np.abs(lp) <= 1e-6)
        assert_parity32(lp, post, st, *_oracle(net, ev), where=f"{name} no evidence")


@pytest.mark.parametrize("seed", range(40))
def test_tiny_random_networks(seed):
    net = tiny_random_network(seed, alpha=0.3 if seed % 3 == 0 else 1.0)
    ev = sample_cases(net, 70, (0.0, 0.6), seed)
    p = J.Plan(net)
    assert_parity32(*p.infer(ev), *_oracle(net, ev), where=f"tiny {seed}")
    plp, ppost, pst = p.infer_plain(ev[:8])
    olp, opost, ost = _oracle(net, ev[:8])
    np.testing.assert_allclose(plp, olp, atol=1e-11)
    np.testing.assert_allclose(ppost, opost, atol=1e-11)


def test_bn1000_many_small_cliques():
    net = configs.network("bn1000")
    ev = configs.evidence("bn1000", net, n_cases=512)
    p = J.Plan(net)
    assert_parity32(*p.infer(ev), *_oracle(net, ev), where="bn1000")


def test_bn110_full_batch_sampled():
    """The 8192-case high-cardinality workload at full size (several arena
    chunks); a seeded sample of cases against the oracle, and posterior
    normalisation on every case."""
    net = configs.network("bn110")
    ev = configs.evidence("bn110", net)
    p = J.Plan(net)
    lp, post, st = p.infer(ev)
    assert np.all(st == 0)
    offs = np.concatenate([[0], np.cumsum(net.card)])
    for v in range(net.n):
        np.testing.assert_allclose(post[:, offs[v]:offs[v + 1]].sum(axis=1), 1.0, atol=1e-9)
    idx = np.random.default_rng(1).choice(ev.shape[0], size=48, replace=False)
    assert_parity32(lp[idx], post[idx], st[idx], *_oracle(net, ev[idx]), where="bn110")


def test_bn420_arena_batch_sampled():
    net = configs.network("bn420")
    p = J.Plan(net)
    ev = configs.evidence("bn420", net, n_cases=512)
    lp, post, st = p.infer(ev)
    assert np.all(st == 0)
    idx = np.random.default_rng(2).choice(ev.shape[0], size=32, replace=False)
    assert_parity32(lp[idx], post[idx], st[idx], *_oracle(net, ev[idx]), where="bn420")
    plp, ppost, pst = p.infer_plain(ev[idx[:4]])
    olp, opost, ost = _oracle(net, ev[idx[:4]])
    np.testing.assert_allclose(plp, olp, atol=1e-10)
    np.testing.assert_allclose(ppost, opost, atol=1e-10)


def test_autotuned_plan_parity():
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=512)
    opts, ns = J.autotune(net, 512)
    assert opts["cases_per_thread"] in (4, 8) and opts["items_per_tile"] in (96, 192, 384, 768, 1536)
    assert opts["items_per_tile_distribute"] in (96, 192, 384, 768, 1536)
    assert ns > 0
    p = J.Plan(net, **opts)
    assert_parity32(*p.infer(ev), *_oracle(net, ev), where=f"autotuned {opts}")


@pytest.mark.parametrize("name,cpt,n", [("bn60", 1, 333), ("bn60", 4, 1000), ("bn1000", 1, 200), ("bn1000", 4, 700),
                                        ("bn20", 2, 100), ("bn110", 4, 130)])
def test_schedules_bitwise_equal(name, cpt, n):
    """The dataflow schedule (one launch per pass, per-tile readiness
    counters) computes every case exactly as the layer schedule does: same
    items, same arithmetic, only the order of independent work differs.  A
    missing dependency would show as a bitwise difference."""
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n, seed=77)
    a = J.Plan(net, cases_per_thread=cpt, schedule=J.JT_SCHEDULE_DATAFLOW).infer(ev)
    b = J.Plan(net, cases_per_thread=cpt, schedule=J.JT_SCHEDULE_LAYERS).infer(ev)
    assert np.array_equal(a[2], b[2])
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1], equal_nan=True)


@pytest.mark.parametrize("name,n", [("bn60", 1000), ("bn110", 130)])
def test_repeat_runs_bitwise_equal(name, n):
    """Every reduction has a fixed order (split segments add their pieces in
    piece order; per-case maxima are integer maxima), so results repeat
    bitwise: the same plan run twice, and a second plan of the same network."""
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n, seed=5)
    p = J.Plan(net)
    a = p.infer(ev)
    b = p.infer(ev)
    c = J.Plan(net).infer(ev)
    for x in (b, c):
        assert np.array_equal(a[2], x[2]) and np.array_equal(a[0], x[0])
        assert np.array_equal(a[1], x[1], equal_nan=True)


def test_expired_wait_reports_timeout_and_context_stays_usable():
    """A dataflow wait that can never be satisfied (a producer that does not
    exist, set by the testing option stall_clique) expires after the plan's
    wait limit: the call returns JT_ETIMEOUT, the device path marks every
    case JT_CASE_INCOMPLETE, and other plans keep working on the device."""
    import time
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=300)
    good = J.Plan(net)
    root = good.info()["root"]
    bad = J.Plan(net, stall_clique=root + 1, wait_limit_us=2000)
    t0 = time.time()
    with pytest.raises(J.JTError) as e:
        bad.infer(ev)
    assert e.value.status == J.JT_ETIMEOUT
    assert time.time() - t0 < 10
    d_ev = torch.from_numpy(ev).cuda()
    d_lp = torch.empty(300, dtype=torch.float64, device="cuda")
    d_post = torch.empty((300, bad.sum_card), dtype=torch.float64, device="cuda")
    d_st = torch.empty(300, dtype=torch.int32, device="cuda")
    bad.infer_device(d_ev, d_lp, d_post, d_st, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.all(d_st.cpu().numpy() == J.JT_CASE_INCOMPLETE)
    assert np.all(np.isnan(d_lp.cpu().numpy()))
    assert_parity32(*good.infer(ev), *_oracle(net, ev), where="after an expired wait")


@pytest.mark.parametrize("which", ["root", "leaf"])
def test_same_plan_recovers_after_expired_wait(which):
    """A pass whose bounded waits expire may leave split-sum counters and
    per-tile state behind in the plan's arena; the next pass on the SAME
    plan and arena must start clean and match the oracle.  The stall is
    turned on and off on one plan (jt_debug_stall); short items make many
    split segments, whose counters a failed pass can leave short."""
    net = configs.network("bn60")
    ev = configs.evidence("bn60", net, n_cases=300)
    probe = J.Plan(net, host_only=1)
    info = probe.info()
    if which == "root":
        k = info["root"]
    else:
        depth = [probe.clique(c)[2] for c in range(info["n_cliques"])]
        k = int(np.argmax(depth))
    plan = J.Plan(net, stall_clique=k + 1, wait_limit_us=2000, items_per_tile=1536,
                  items_per_tile_distribute=1536)
    expect = _oracle(net, ev)
    for _ in range(2):
        with pytest.raises(J.JTError) as e:
            plan.infer(ev)                       # stalled: the waits expire
        assert e.value.status == J.JT_ETIMEOUT
        plan.debug_stall(False)
        assert_parity32(*plan.infer(ev), *expect, where=f"stall on clique {k} lifted")
        # the device path: a stalled call marks its cases, the next
        # synchronous call reports the expired wait and clears it
        plan.debug_stall(True)
        d_ev = torch.from_numpy(ev).cuda()
        d_lp = torch.empty(300, dtype=torch.float64, device="cuda")
        d_post = torch.empty((300, plan.sum_card), dtype=torch.float64, device="cuda")
        d_st = torch.empty(300, dtype=torch.int32, device="cuda")
        plan.infer_device(d_ev, d_lp, d_post, d_st, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.all(d_st.cpu().numpy() == J.JT_CASE_INCOMPLETE)
        with pytest.raises(J.JTError) as e:
            plan.infer(ev)
        assert e.value.status == J.JT_ETIMEOUT
        plan.debug_stall(False)
        assert_parity32(*plan.infer(ev), *expect, where=f"device path, stall on clique {k} lifted")
        plan.debug_stall(True)


def test_debug_stall_needs_a_stall_plan():
    net = configs.network("bn20")
    with pytest.raises(J.JTError) as e:
        J.Plan(net).debug_stall(False)
    assert e.value.status == J.JT_EINVAL


def _device_run(plan, ev):
    n = ev.shape[0]
    d_ev = torch.from_numpy(ev).cuda()
    out = (torch.empty(n, dtype=torch.float64, device="cuda"),
           torch.empty((n, plan.sum_card), dtype=torch.float64, device="cuda"),
           torch.empty(n, dtype=torch.int32, device="cuda"))
    plan.infer_device(d_ev, *out, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


@pytest.mark.parametrize("name,n_cases", [("bn20", 100), ("bn60", 1000), ("bn1000", 500), ("bn110", 256), ("bn420", 128)])
@pytest.mark.parametrize("schedule", [J.JT_SCHEDULE_DATAFLOW, J.JT_SCHEDULE_LAYERS])
def test_recomputed_tables_equal_stored_bitwise(name, n_cases, schedule):
    """recompute_psi: the collect pass stores no clique tables and the
    distribute pass rebuilds each row from the base table, the child
    messages and the evidence in the collect pass's order -- the outputs
    equal the stored-table plan's bit for bit (and so the oracle's within
    the FP32 tolerance, checked on a sample)."""
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n_cases, seed=55)
    stored = J.Plan(net, schedule=schedule, fuse_distribute=0)
    recomp = J.Plan(net, schedule=schedule, recompute_psi=1)
    a = _device_run(stored, ev)
    b = _device_run(recomp, ev)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    # no clique tables in the per-batch arena
    assert recomp.info()["arena_bytes"] < stored.info()["arena_bytes"]
    idx = np.arange(min(n_cases, 24))
    assert_parity32(b[0][idx], b[1][idx], b[2][idx], *_oracle(net, ev[idx]), where=f"recompute {name}")


@pytest.mark.parametrize("name,n_cases", [("bn60", 1000), ("bn420", 128)])
def test_collect_prefetch_changes_no_result(name, n_cases):
    """collect_prefetch only requests rows into L2 ahead of use: outputs are
    bit for bit those of the plan without it."""
    net = configs.network(name)
    ev = configs.evidence(name, net, n_cases=n_cases, seed=56)
    a = _device_run(J.Plan(net), ev)
    b = _device_run(J.Plan(net, collect_prefetch=1), ev)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)

"""Serving loop (continuous batching) on the GPU, through the C ABI.

* every result equals the FP64 oracle within the FP32 tolerance;
* a request gives bit-identical results alone and inside a mixed stream of
  requests on several plans (fixed per-case reduction order);
* requests are coalesced into batches and batches of different plans are in
  flight together; admission respects the arena budget;
* query subsets, unknown tickets, stats.
"""
import time

import numpy as np
import pytest

import oracle
from synth import configs
from tests.common import assert_parity32

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2212_04241_gb300.jt as J  # noqa: E402


def _wait(srv, tickets, out_len):
    res = {}
    deadline = time.time() + 120
    while len(res) < len(tickets):
        for t in tickets:
            if t in res:
                continue
            r = srv.poll(t, out_len[t])
            if r is not None:
                res[t] = r
        assert time.time() < deadline, "serving results did not arrive"
    return res


@pytest.fixture(scope="module")
def plans():
    names = ["bn60", "bn1000", "bn20"]
    out = []
    for nm in names:
        net = configs.network(nm)
        out.append((nm, net, J.Plan(net, cases_per_thread=1)))
    return out


def test_alone_vs_mix_bitwise_and_oracle(plans):
    rng = np.random.default_rng(0)
    reqs = []
    for pi, (nm, net, plan) in enumerate(plans):
        ev = configs.evidence(nm, net, n_cases=40, seed=500 + pi)
        for e in ev:
            reqs.append((pi, e))
    order = rng.permutation(len(reqs))

    srv = J.Server(arena_bytes=8 << 30, max_batch=64, max_inflight=6)
    pids = [srv.add_plan(p) for _, _, p in plans]
    # alone: one request at a time
    alone = {}
    for i in range(len(reqs)):
        pi, e = reqs[i]
        t = srv.submit(pids[pi], e)
        srv.drain()
        alone[i] = srv.poll(t, plans[pi][2].sum_card)
        assert alone[i] is not None
    # mix: everything at once, interleaved across plans
    tickets, out_len, which = [], {}, {}
    for i in order:
        pi, e = reqs[i]
        t = srv.submit(pids[pi], e)
        tickets.append(t)
        out_len[t] = plans[pi][2].sum_card
        which[t] = i
    res = _wait(srv, tickets, out_len)
    st = srv.stats()
    assert st["completed"] == 2 * len(reqs)
    assert st["largest_batch"] > 1, "requests were not coalesced"
    for t, (lp, post, cs) in res.items():
        a = alone[which[t]]
        assert lp == a[0] and cs == a[2] and np.array_equal(post, a[1])
    # oracle check
    for pi, (nm, net, plan) in enumerate(plans):
        idx = [i for i in range(len(reqs)) if reqs[i][0] == pi]
        ev = np.stack([reqs[i][1] for i in idx])
        olp, opost, ost = oracle.Oracle(net).infer(ev, threads=8)
        lp = np.array([alone[i][0] for i in idx])
        post = np.stack([alone[i][1] for i in idx])
        cs = np.array([alone[i][2] for i in idx], dtype=np.int32)
        assert_parity32(lp, post, cs, olp, opost, ost, where=f"serving {nm}")
    assert st["p99_ns"] >= st["p50_ns"] > 0
    srv.close()


def test_query_subset_and_errors(plans):
    nm, net, plan = plans[0]
    srv = J.Server(arena_bytes=4 << 30, max_batch=32, max_inflight=2)
    pid = srv.add_plan(plan)
    ev = configs.evidence(nm, net, n_cases=1)[0]
    q = [5, 0, 17]
    t_all = srv.submit(pid, ev)
    t_q = srv.submit(pid, ev, query=q)
    srv.drain()
    full = srv.poll(t_all, plan.sum_card)
    offs = np.concatenate([[0], np.cumsum(net.card)])
    m = int(sum(net.card[v] for v in q))
    sub = srv.poll(t_q, m)
    expect = np.concatenate([full[1][offs[v]:offs[v + 1]] for v in q])
    assert np.array_equal(sub[1], expect)
    with pytest.raises(J.JTError) as e:
        srv.poll(t_all, plan.sum_card)  # already released
    assert e.value.status == J.JT_ENOTFOUND
    with pytest.raises(J.JTError) as e:
        srv.submit(pid + 7, ev)
    assert e.value.status == J.JT_ENOTFOUND
    srv.close()


def test_admission_by_arena_bytes(plans):
    """A budget that holds a single batch slot still serves two plans: one
    plan's batch waits until the other's slot is released."""
    (n0, net0, p0), (n1, net1, p1) = plans[0], plans[1]
    srv_probe = J.Server(arena_bytes=64 << 30, max_batch=16, max_inflight=4)
    srv_probe.add_plan(p0)
    srv_probe.add_plan(p1)
    srv_probe.close()
    # per-slot bytes are not exposed; use a budget between one and two slots
    budget = 0
    for cand in [1 << 24, 1 << 25, 1 << 26, 1 << 27, 1 << 28]:
        try:
            s = J.Server(arena_bytes=cand, max_batch=16, max_inflight=4)
            s.add_plan(p0)
            s.add_plan(p1)
            s.close()
            budget = cand
            break
        except J.JTError:
            s.close()
    assert budget
    srv = J.Server(arena_bytes=budget, max_batch=16, max_inflight=4)
    a, b = srv.add_plan(p0), srv.add_plan(p1)
    e0 = configs.evidence(n0, net0, n_cases=50)
    e1 = configs.evidence(n1, net1, n_cases=50)
    tickets, out_len = [], {}
    for i in range(50):
        for pid, e, p in ((a, e0[i], p0), (b, e1[i], p1)):
            t = srv.submit(pid, e)
            tickets.append(t)
            out_len[t] = p.sum_card
    res = _wait(srv, tickets, out_len)
    assert len(res) == 100
    st = srv.stats()
    assert st["peak_arena_bytes"] <= budget
    # slots are bound once and reused; when the pool cannot hold both plans'
    # slots the plans take turns, evicting each other's idle slot
    resident = st["slot_creations"] - st["slot_evictions"]
    assert 1 <= resident <= 4 and st["slot_creations"] <= st["batches"]
    for pid in (a, b):
        ps = srv.plan_stats(pid)
        assert ps["completed"] == 50 and ps["batches"] >= 1 and ps["p99_ns"] >= ps["p50_ns"] > 0
    srv.close()


def test_slots_are_reused_batch_after_batch(plans):
    """A plan's batch slots are regions of the server's pool bound once and
    reused: many waves of requests create at most max_inflight slots."""
    nm, net, plan = plans[0]
    srv = J.Server(arena_bytes=8 << 30, max_batch=16, max_inflight=3)
    pid = srv.add_plan(plan)
    ev = configs.evidence(nm, net, n_cases=64, seed=9)
    for wave in range(6):
        tickets = [srv.submit(pid, e) for e in ev]
        res = _wait(srv, tickets, {t: plan.sum_card for t in tickets})
        assert all(r[2] == 0 for r in res.values())
    st = srv.stats()
    assert st["completed"] == 6 * 64 and st["batches"] >= 6 * 4
    assert 1 <= st["slot_creations"] <= 3 and st["slot_evictions"] == 0
    with pytest.raises(J.JTError) as e:
        srv.plan_stats(pid + 1)
    assert e.value.status == J.JT_ENOTFOUND
    srv.close()


def test_expired_device_wait_in_a_served_batch():
    """A plan whose dataflow waits expire (the testing option stall_clique
    makes one clique wait for a producer that does not exist, limit 2 ms):
    its requests come back as JT_CASE_INCOMPLETE with NaN outputs, batch
    after batch, while another plan served alongside stays correct."""
    net = configs.network("bn60")
    good = J.Plan(net, cases_per_thread=1)
    bad = J.Plan(net, cases_per_thread=1, stall_clique=good.info()["root"] + 1, wait_limit_us=2000)
    ev = configs.evidence("bn60", net, n_cases=6, seed=21)
    srv = J.Server(arena_bytes=4 << 30, max_batch=8, max_inflight=4)
    pg, pb = srv.add_plan(good), srv.add_plan(bad)
    for _ in range(2):                        # two rounds: the slot serves again after a failure
        tb = [srv.submit(pb, e) for e in ev[:3]]
        tg = [srv.submit(pg, e) for e in ev[3:]]
        out_len = {t: good.sum_card for t in tb + tg}
        res = _wait(srv, tb + tg, out_len)
        for t in tb:
            lp, post, st = res[t]
            assert st == J.JT_CASE_INCOMPLETE and np.isnan(lp)
        olp, opost, ost = oracle.Oracle(net).infer(ev[3:])
        lp = np.array([res[t][0] for t in tg])
        post = np.stack([res[t][1] for t in tg])
        st = np.array([res[t][2] for t in tg], dtype=np.int32)
        assert_parity32(lp, post, st, olp, opost, ost, where="served beside a stalled plan")
    srv.close()


def test_rolling_alone_vs_mix_and_slots_bitwise(plans):
    """Iteration-level batching: requests that arrive while other tiles are
    mid-pass join at the next tick.  Each result equals the same request
    served alone, and the batch-slot path's result, bit for bit, and the
    FP64 oracle within the FP32 tolerance."""
    rng = np.random.default_rng(1)
    reqs = []
    for pi, (nm, net, plan) in enumerate(plans):
        ev = configs.evidence(nm, net, n_cases=60, seed=900 + pi)
        reqs += [(pi, e) for e in ev]
    srv = J.Server(arena_bytes=8 << 30, max_batch=32, max_inflight=4)
    rolled = [srv.add_plan(p, rolling_tiles=4) for _, _, p in plans]
    slotted = [srv.add_plan(p) for _, _, p in plans]
    out_len = lambda pi: plans[pi][2].sum_card  # noqa: E731
    alone = {}
    for i, (pi, e) in enumerate(reqs[::7]):
        t = srv.submit(rolled[pi], e)
        srv.drain()
        alone[i * 7] = srv.poll(t, out_len(pi))
    # the mix: submitted in waves with pauses, so that new requests arrive
    # while earlier tiles are between layers
    tickets, lens, which = [], {}, {}
    order = rng.permutation(len(reqs))
    for w, chunk in enumerate(np.array_split(order, 6)):
        for i in chunk:
            pi, e = reqs[i]
            t = srv.submit(rolled[pi], e)
            tickets.append(t)
            lens[t] = out_len(pi)
            which[t] = i
        time.sleep(0.002 * w)
    res = _wait(srv, tickets, lens)
    # the batch-slot path on the same requests
    st_tickets, st_which = [], {}
    for i in range(len(reqs)):
        pi, e = reqs[i]
        t = srv.submit(slotted[pi], e)
        st_tickets.append(t)
        lens[t] = out_len(pi)
        st_which[t] = i
    slot_res = _wait(srv, st_tickets, lens)
    by_req = {which[t]: r for t, r in res.items()}
    for t, r in slot_res.items():
        a = by_req[st_which[t]]
        assert a[0] == r[0] and a[2] == r[2] and np.array_equal(a[1], r[1]), "rolling vs batch slots"
    for i, a in alone.items():
        b = by_req[i]
        assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1]), "alone vs mix"
    for pi, (nm, net, plan) in enumerate(plans):
        idx = [i for i in range(len(reqs)) if reqs[i][0] == pi]
        ev = np.stack([reqs[i][1] for i in idx])
        olp, opost, ost = oracle.Oracle(net).infer(ev, threads=8)
        lp = np.array([by_req[i][0] for i in idx])
        post = np.stack([by_req[i][1] for i in idx])
        cs = np.array([by_req[i][2] for i in idx], dtype=np.int32)
        assert_parity32(lp, post, cs, olp, opost, ost, where=f"rolling {nm}")
    st = srv.stats()
    assert st["completed"] == len(alone) + 2 * len(reqs)
    for pid in rolled:
        ps = srv.plan_stats(pid)
        assert ps["p99_ns"] >= ps["p50_ns"] > 0
    srv.close()


def test_rolling_refuses_tiles_beyond_the_pool(plans):
    nm, net, plan = plans[1]
    srv = J.Server(arena_bytes=1 << 26, max_batch=8, max_inflight=2)
    with pytest.raises(J.JTError) as e:
        srv.add_plan(plan, rolling_tiles=1 << 16)
    assert e.value.status == J.JT_ENOMEM
    srv.close()


def test_priority_class_changes_no_result(plans):
    """jt_server_set_priority moves a plan's batches to the high-priority
    streams; the same requests give the same results bit for bit with and
    without it, and an unknown plan id is refused."""
    srv = J.Server(arena_bytes=8 << 30, max_batch=32, max_inflight=4)
    pids = [srv.add_plan(p) for _, _, p in plans]
    reqs = []
    for pi, (nm, net, plan) in enumerate(plans):
        for e in configs.evidence(nm, net, n_cases=24, seed=700 + pi):
            reqs.append((pi, e))

    def run():
        tickets, out_len = [], {}
        for pi, e in reqs:
            t = srv.submit(pids[pi], e)
            tickets.append(t)
            out_len[t] = plans[pi][2].sum_card
        res = _wait(srv, tickets, out_len)
        return [res[t] for t in tickets]

    before = run()
    for pid in pids[::2]:
        srv.set_priority(pid, True)
    after = run()
    for a, b in zip(before, after):
        assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])
    with pytest.raises(J.JTError) as e:
        srv.set_priority(len(pids) + 3, True)
    assert e.value.status == J.JT_ENOTFOUND
    srv.close()

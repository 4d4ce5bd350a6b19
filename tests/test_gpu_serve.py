"""Serving (fock_serve_*): continuous batching on one GPU.

* every result equals the result of solving that problem alone (the batched
  planner fixes reduction orders and start vectors per problem, so the
  comparison is bitwise);
* requests submitted while batches run are admitted before those batches
  finish (their work overlaps on the device);
* the HBM budget bounds what is in flight; a problem larger than the budget
  is refused at submission.
"""
import threading
import time

import numpy as np
import pytest

import lattice_inputs as li
from tests import _cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fock():
    from paper_1702_00339_gb300 import build, fock as f
    build.build()
    return f


def _mix():
    ps = []
    for s in range(3):
        ps.append(_cases.periodic_chain_small(L=5 + s, n0=6, n_perp=16, m0=8, seed=s, R=12))
        ps.append(_cases.box_chain_small(L=8 + 2 * s, n0=5, pad=5, n_perp=14, seed=s, R=12, k=4))
    ps.append(_cases.periodic_3d_small(L=(3, 2, 2), n0=4, R=10))
    ps.append(_cases.periodic_chain_small(L=6, n0=8, n_perp=20, m0=4, R=16))
    return ps


def test_results_equal_alone_and_in_the_mix(fock):
    ps = _mix()
    ctx = fock.Context(0)
    alone = [ctx.solve([p])[0] for p in ps]
    ctx.close()
    srv = fock.Server(0, slots=3, max_batch=3)
    tickets = [None] * len(ps)

    def submit(idx):
        for i in idx:
            tickets[i] = srv.submit(ps[i])
            time.sleep(0.002)

    th = [threading.Thread(target=submit, args=(range(r, len(ps), 2),)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    res = [srv.poll(t, timeout_ms=120000) for t in tickets]
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(ps) and st["batches"] >= 2
    for p, a, r in zip(ps, alone, res):
        assert r["status"] == 0 and a["status"] == 0
        assert np.array_equal(r["evals"], a["evals"])
        if not (p.is_box or p.defects):
            assert np.array_equal(r["block_of"], a["block_of"])
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]


def test_arrivals_are_admitted_while_batches_run(fock):
    big = [_cases.with_table(li.config2(s, L=48, n0=15, pad=32, n_perp=128, R=24)) for s in range(8)]
    for p in big:
        p.k_eig = 16
    small = [_cases.periodic_chain_small(L=6, n0=6, n_perp=16, m0=8, seed=s, R=12) for s in range(4)]
    srv = fock.Server(0, slots=2, max_batch=8)
    tb = [srv.submit(p) for p in big]
    # wait until the first batch is on the device, then submit more
    t_end = time.time() + 60
    while srv.stats()["inflight"] == 0 and time.time() < t_end:
        time.sleep(0.001)
    ts = [srv.submit(p) for p in small]
    rb = [srv.poll(t, timeout_ms=120000) for t in tb]
    rs = [srv.poll(t, timeout_ms=120000) for t in ts]
    st = srv.stats()
    srv.stop()
    assert all(r["status"] == 0 for r in rb + rs)
    # the later arrivals were admitted while a batch of the earlier ones was
    # still on the device
    assert min(r["t_admit_ns"] for r in rs) < max(r["t_done_ns"] for r in rb)
    assert st["max_inflight"] == 2


def test_budget_bounds_what_is_in_flight(fock):
    ps = _mix()[:6]
    srv = fock.Server(0, slots=3, max_batch=8, budget_bytes=64 << 20)
    ts = [srv.submit(p) for p in ps]
    rs = [srv.poll(t, timeout_ms=120000) for t in ts]
    st = srv.stats()
    srv.stop()
    assert all(r["status"] == 0 for r in rs)
    assert st["peak_reserved_bytes"] <= st["budget_bytes"]


def test_refusals(fock):
    srv = fock.Server(0, slots=1, budget_bytes=1 << 20)
    with pytest.raises(fock.FockError) as e:
        srv.submit(_cases.with_table(li.config2(0)))
    assert e.value.code == fock.FOCK_ENOMEM
    bad = _cases.periodic_chain_small(L=5, n0=6, n_perp=16, m0=8, R=12)
    bad.exps = -bad.exps
    with pytest.raises(fock.FockError) as e:
        srv.submit(bad)
    assert e.value.code == fock.FOCK_EINVAL
    srv.stop()


def test_structured_request_published_when_it_leaves_the_iteration(fock):
    """A box chain that converges in tens of iterations and a ring of 194
    cells with three defects that needs hundreds share one batch (one slot,
    both queued behind a 16^3 lattice).  The chain's result is published when
    it converges, before the batch ends, and the client frees it at once
    while the batch still runs; both results equal a solve alone bit for
    bit."""
    fast = _cases.box_chain_small(L=12, n0=5, pad=6, n_perp=20, seed=0, R=16, k=6)
    slow = li.serving_stream(299, seed=3000)[298]
    ctx = fock.Context(0)
    alone = [ctx.solve([q], check=False)[0] for q in (fast, slow)]
    ctx.close()
    assert alone[0]["iters"] < alone[1]["iters"]
    srv = fock.Server(0, slots=1, max_batch=8)
    tb = srv.submit(_cases.with_table(li.config3(0)))
    tf = srv.submit(fast)
    ts = srv.submit(slow)
    rf = srv.poll(tf, timeout_ms=300000)
    rs = srv.poll(ts, timeout_ms=300000)
    rb = srv.poll(tb, timeout_ms=300000)
    st = srv.stats()
    srv.stop()
    assert rb["status"] == 0 and rb["batch_id"] < rf["batch_id"]
    assert rf["batch_id"] == rs["batch_id"] and rf["batch_size"] == 2
    assert rf["t_done_ns"] < rs["t_done_ns"]
    assert st["completed"] == 3
    for r, a in zip((rf, rs), alone):
        assert r["status"] == a["status"] == 0
        assert r["iters"] == a["iters"]
        assert np.array_equal(r["evals"], a["evals"])

"""Host logic of the serving loop (no GPU): admission by HBM budget, continuous batching into free slots, retirement,
cancellation, rejection of requests that can never fit, and eviction of idle operators."""
import numpy as np
import pytest

from paper_2603_00383_gb300 import serve


def req(rid, geom, steps=3, arrival=0.0):
    return serve.Request(rid=rid, geom=geom, steps=steps, seed=rid, arrival=arrival)


def kinds(actions):
    return [a[0] for a in actions]


def test_poisson_trace_rate_and_ranges():
    tr = serve.poisson_trace(n_geom=4, rate=20.0, duration=60.0, steps_lo=1000, steps_hi=20000)
    assert 1000 < len(tr) < 1400                      # 1200 expected
    gaps = np.diff([0.0] + [r.arrival for r in tr])
    assert abs(gaps.mean() - 1 / 20.0) < 0.01 and np.all(gaps > 0)
    assert min(r.steps for r in tr) >= 1000 and max(r.steps for r in tr) <= 20000
    assert {r.geom for r in tr} == {0, 1, 2, 3}
    assert serve.poisson_trace(4, 20.0, 60.0, 1000, 20000)[7].seed == tr[7].seed


def test_requests_fill_slots_of_one_group_then_open_another():
    s = serve.Scheduler(geom_bytes=[100], group_bytes=[10], budget=1000, batch=2)
    for k in range(3):
        s.submit(req(k, 0))
    a = s.plan(0.0)
    assert kinds(a) == ["build", "group", "admit", "admit", "group", "admit"]
    assert s.used == 100 + 2 * 10
    assert [r.slot for r in s.requests.values()] == [(0, 0), (0, 1), (1, 0)]


def test_finished_member_frees_its_slot_for_the_next_arrival():
    s = serve.Scheduler([100], [10], budget=1000, batch=2)
    s.submit(req(0, 0, steps=2))
    s.submit(req(1, 0, steps=5))
    s.submit(req(2, 0, steps=5, arrival=1.0))
    s.plan(0.0)
    for _ in range(2):
        s.step_done(0)
        s.step_done(1)
    assert s.requests[0].state == "done"
    a = s.plan(1.0)
    assert a[0] == ("retire", 0, 0, 0)
    assert ("admit", 0, 0, 2) in a and "group" not in kinds(a)     # reuses the slot: no new group
    assert s.requests[2].slot == (0, 0) and s.requests[0].finished == 1.0


def test_request_that_can_never_fit_is_rejected_and_others_proceed():
    s = serve.Scheduler([100, 5000], [10, 10], budget=1000, batch=4)
    s.submit(req(0, 1))
    s.submit(req(1, 0))
    a = s.plan(0.0)
    assert ("reject", 0) in a and s.requests[0].state == "rejected"
    assert s.requests[1].state == "active"


def test_admission_waits_for_memory_and_evicts_idle_operators_lru():
    s = serve.Scheduler([400, 400, 400], [50, 50, 50], budget=1000, batch=1)
    s.submit(req(0, 0, steps=1))
    s.submit(req(1, 1, steps=1))
    s.plan(0.0)
    assert s.used == 900
    s.submit(req(2, 2, steps=1, arrival=0.5))
    a = s.plan(0.5)                                    # no room: geometry 2 waits (0 and 1 are busy)
    assert kinds(a) == [] and s.requests[2].state == "queued"
    s.step_done(0)                                     # request 0 finishes: its group and operator become idle
    a = s.plan(1.0)
    assert kinds(a) == ["retire", "drop", "evict", "build", "group", "admit"]
    assert ("evict", 0) in a and s.requests[2].state == "active" and s.used == 900


def test_cancel_queued_and_active_requests():
    s = serve.Scheduler([100], [10], budget=1000, batch=1)
    s.submit(req(0, 0, steps=10))
    s.submit(req(1, 0, steps=10, arrival=5.0))
    s.plan(0.0)
    s.cancel(1)                                        # still queued: leaves the queue
    s.cancel(0)                                        # active: retired at the next plan
    assert s.requests[1].state == "cancelled" and 1 not in s.queue
    a = s.plan(1.0)
    assert a == [("retire", 0, 0, 0)] and s.requests[0].state == "cancelled"
    assert s.plan(6.0) == []


def test_future_arrivals_do_not_pin_idle_operators():
    s = serve.Scheduler([600, 600], [10, 10], budget=1000, batch=1)
    s.submit(req(0, 0, steps=1))
    s.plan(0.0)
    s.step_done(0)
    s.submit(req(1, 0, steps=1, arrival=100.0))        # geometry 0 is wanted again, but only much later
    s.submit(req(2, 1, steps=1, arrival=1.0))
    a = s.plan(1.0)
    assert ("evict", 0) in a and s.requests[2].state == "active"

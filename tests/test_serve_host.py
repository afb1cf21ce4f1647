"""Host logic of the continuous-batching service (no GPU): admission by memory
footprint with backfill, slot reuse, concurrency, completion of every request."""
import threading
import time

import pytest

from paper_2603_10514_gb300.serve import Request, Server, latency_stats


class FakeMatrix:
    def __init__(self, n, cplx):
        self.shape = (n, n)
        self._esz = 16 if cplx else 8

    def element_size(self):
        return self._esz


def make(rid, n, cplx=False, nev=4, nex=2):
    return Request(rid=rid, A=FakeMatrix(n, cplx), V0=None, nev=nev, nex=nex, bounds=(0, 0, 1))


class Recorder:
    def __init__(self, budget, delay=0.02):
        self.lock = threading.Lock()
        self.active = {}
        self.max_bytes = 0
        self.max_active = 0
        self.order = []
        self.budget = budget
        self.delay = delay

    def __call__(self, slot, req):
        with self.lock:
            assert slot not in self.active, "slot used twice at once"
            self.active[slot] = req.footprint()
            self.max_bytes = max(self.max_bytes, sum(self.active.values()))
            self.max_active = max(self.max_active, len(self.active))
            self.order.append(req.rid)
        time.sleep(self.delay * (1 + req.n / 1000))
        with self.lock:
            del self.active[slot]
        return 0, [float(req.rid)], [0.0], {"slot": slot}


def test_all_requests_complete_within_budget_and_slots():
    reqs = [make(i, n) for i, n in enumerate([500, 3000, 800, 2000, 700, 4000, 600, 1200])]
    budget = max(r.footprint() for r in reqs) + reqs[0].footprint()
    rec = Recorder(budget)
    srv = Server(slots=3, hbm_budget=budget, solve_fn=rec)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert sorted(r.rid for r in srv.completed) == list(range(len(reqs)))
    assert rec.max_bytes <= budget
    assert rec.max_active <= 3
    assert all(r.status == 0 and r.evals == [float(r.rid)] for r in reqs)
    st = latency_stats(reqs)
    assert st["count"] == len(reqs) and st["p99_s"] >= st["p50_s"] > 0


def test_backfill_admits_small_request_past_a_blocked_large_one():
    big, small_running, small_later = make(0, 4000), make(1, 3000), make(2, 500)
    budget = big.footprint()  # the big one cannot run beside anything else
    started = {}

    def solve(slot, req):
        started[req.rid] = time.perf_counter()
        time.sleep(0.15 if req.rid == 1 else 0.02)
        return 0, [], [], {}

    srv = Server(slots=4, hbm_budget=budget, solve_fn=solve)
    srv.submit(small_running)   # occupies memory, so the big one must wait
    time.sleep(0.05)
    srv.submit(big)
    srv.submit(small_later)     # fits beside small_running: admitted before the big one
    srv.drain()
    assert started[2] < started[0]
    assert len(srv.completed) == 3


def test_continuous_admission_while_others_run():
    """Requests arriving while others are in flight start as soon as a slot frees."""
    rec = Recorder(1 << 60, delay=0.05)
    srv = Server(slots=2, solve_fn=rec)
    first = [srv.submit(make(i, 1000)) for i in range(2)]
    time.sleep(0.02)
    later = [srv.submit(make(10 + i, 1000)) for i in range(3)]
    srv.drain()
    assert rec.max_active == 2
    assert len(srv.completed) == 5
    assert max(r.t_done for r in first) <= max(r.t_done for r in later)


def test_request_larger_than_budget_is_rejected():
    srv = Server(slots=1, hbm_budget=10, solve_fn=lambda s, r: (0, [], [], {}))
    with pytest.raises(ValueError):
        srv.submit(make(0, 100))
    srv.drain()


def test_solver_exception_does_not_stall_the_service():
    def solve(slot, req):
        if req.rid == 1:
            raise RuntimeError("device error")
        return 0, [], [], {}

    srv = Server(slots=2, solve_fn=solve)
    for i in range(4):
        srv.submit(make(i, 300))
    srv.drain()
    st = {r.rid: r.status for r in srv.completed}
    assert st[1] == -999 and st[0] == st[2] == st[3] == 0

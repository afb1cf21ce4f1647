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


# --------------------------------------------------------------------------
# BatchServer: requests as problems of one batch session, advanced per step
# --------------------------------------------------------------------------

class FakeBatch:
    """Stands in for the library's batch session: a problem of order n ends after
    ceil(n / 500) steps; records how many problems were in flight at every step."""

    def __init__(self):
        self.live = {}
        self.next = 0
        self.inflight = []
        self.closed = False

    def add(self, prob):
        prob.id = self.next
        self.next += 1
        self.live[prob.id] = [prob, -(-prob.A.shape[0] // 500)]
        return prob

    def pending(self):
        return len(self.live)

    def step(self):
        self.inflight.append(len(self.live))
        out = []
        for pid in list(self.live):
            ent = self.live[pid]
            ent[1] -= 1
            if ent[1] == 0:
                prob = ent[0]
                prob.status = 0
                prob.evals = [float(prob.A.shape[0])]
                out.append(prob)
                del self.live[pid]
        time.sleep(0.002)
        return out

    def close(self):
        self.closed = True


class FakeBatchProblem:
    def __init__(self, A, V0, nev, nex, bounds, cfg=None):
        self.A, self.nev, self.nex = A, nev, nex
        self.status, self.evals, self.resid, self.stats, self.id = None, None, None, None, -1


@pytest.fixture
def fake_problem(monkeypatch):
    import paper_2603_10514_gb300 as P
    monkeypatch.setattr(P, "BatchProblem", FakeBatchProblem)


def test_batch_server_completes_every_request_within_budget(fake_problem):
    from paper_2603_10514_gb300.serve import BatchServer
    reqs = [make(i, n) for i, n in enumerate([500, 3000, 800, 2000, 700, 4000, 600, 1200])]
    fb = FakeBatch()
    budget = max(r.footprint() for r in reqs) + 2 * reqs[0].footprint()
    srv = BatchServer(hbm_budget=budget, make_batch=lambda: fb, workspace_bytes=lambda r: 0,
                      max_in_flight=3)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert sorted(r.rid for r in srv.completed) == list(range(len(reqs)))
    assert all(r.status == 0 and r.evals == [float(r.n)] for r in reqs)
    assert max(fb.inflight) <= 3 and fb.closed
    assert srv.in_use == 0
    st = latency_stats(reqs)
    assert st["count"] == len(reqs) and st["p99_s"] >= st["p50_s"] > 0


def test_batch_server_admits_while_others_are_in_flight(fake_problem):
    """A request arriving while a long one iterates joins the session at the next step
    (continuous batching) and, being short, finishes first."""
    from paper_2603_10514_gb300.serve import BatchServer
    fb = FakeBatch()
    srv = BatchServer(make_batch=lambda: fb, workspace_bytes=lambda r: 0)
    long_req = srv.submit(make(0, 20000))
    time.sleep(0.01)
    short_req = srv.submit(make(1, 400))
    srv.drain()
    assert short_req.t_done < long_req.t_done
    assert max(fb.inflight) == 2


def test_batch_server_backfills_past_a_request_that_does_not_fit(fake_problem):
    from paper_2603_10514_gb300.serve import BatchServer
    fb = FakeBatch()
    big, small = make(0, 3000), make(1, 600)
    first = make(2, 2800)
    budget = big.footprint() + small.footprint()  # big fits alone, first + small together
    srv = BatchServer(hbm_budget=budget, make_batch=lambda: fb, workspace_bytes=lambda r: 0)
    srv.submit(first)
    time.sleep(0.01)
    srv.submit(big)     # does not fit while `first` runs
    srv.submit(small)   # fits beside `first`: admitted before `big`
    srv.drain()
    assert small.t_admit < big.t_admit
    assert all(r.status == 0 for r in (first, big, small))

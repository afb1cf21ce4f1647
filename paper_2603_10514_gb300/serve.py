"""Continuous-batching eigensolver service on one GPU.

Two engines.  BatchServer (the default one of the benchmark): the requests in flight are
problems of one batch session, advanced together one outer iteration of Algorithm 1 at a
time with their filter steps in shared launches; queued requests join between iterations
as memory frees up, finished ones leave at once.  Server: whole solves on a fixed number
of concurrent slot handles, described next.

Requests (dense Hermitian / symmetric eigenproblems of different orders) arrive at
any time.  A request is admitted as soon as a solver slot is idle and its HBM
footprint fits in the memory left by the requests in flight; admission is
first-come-first-served with backfill (a smaller later request may start while a
larger one at the head of the queue waits for memory).  Each slot owns a chase
handle with its own CUDA stream, and its workspace is reserved once at start-up for
the largest admissible problem, so that no device allocation happens while
requests run.  Admitted requests run concurrently: their kernels overlap on the
device through the slots' streams.  A request's result does not depend on what
else is running, because every kernel's arithmetic order is fixed by the problem's
own shape (split-K reductions in a fixed order, exact integer accumulation in the
tensor-core products).

Latency of a request = completion time - arrival time (queueing included).
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    A: object              # column-major CUDA tensor (float64 / complex128), resident
    V0: object             # column-major CUDA tensor n x (nev + nex), overwritten by the solve
    nev: int
    nex: int
    bounds: tuple
    cfg: object = None
    t_arrive: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    status: int = -1
    evals: np.ndarray = None
    resid: np.ndarray = None
    stats: dict = None
    slot: int = -1
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def n(self):
        return self.A.shape[0]

    def footprint(self):
        """Device bytes the request occupies while in flight besides the slot's reserved
        workspace: its matrix and its search block."""
        esz = self.A.element_size()
        return esz * self.n * self.n + esz * self.n * (self.nev + self.nex)


class Server:
    """Runs requests on `slots` concurrent solver slots.

    solve_fn(slot, request) -> (status, evals, resid, stats) performs one solve; the
    default uses the slot's chase handle (created by `make_handle(slot)`)."""

    def __init__(self, slots=4, hbm_budget=1 << 62, solve_fn=None, make_handle=None,
                 slot_workspace=0):
        self.nslots = slots
        self.handles = [make_handle(i) for i in range(slots)] if make_handle else [None] * slots
        if slot_workspace:
            for h in self.handles:
                h.reserve(slot_workspace)
        self.solve_fn = solve_fn or self._chase_solve
        self.budget = hbm_budget
        self.in_use = 0
        self.queue = collections.deque()
        self.idle = collections.deque(range(slots))
        self.cv = threading.Condition()
        self.closing = False
        self.completed = []
        self.workers = []
        self.max_in_flight = 0
        self.sched = threading.Thread(target=self._schedule, daemon=True)
        self.sched.start()

    # -- default solver -------------------------------------------------------
    def _chase_solve(self, slot, req):
        from . import chase_solve
        rc, ev, res, st, _ = chase_solve(self.handles[slot], req.A, req.V0, req.nev, req.nex,
                                         req.bounds, req.cfg, check=False)
        return rc, ev, res, st

    # -- client side ----------------------------------------------------------
    def submit(self, req: Request):
        req.t_arrive = time.perf_counter()
        with self.cv:
            if req.footprint() > self.budget:
                raise ValueError("request %d needs more memory than the whole budget" % req.rid)
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def drain(self):
        """Wait until every submitted request has completed, then stop the scheduler."""
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        self.sched.join()
        for t in self.workers:
            t.join()

    def close(self):
        self.drain()
        for h in self.handles:
            if h is not None:
                h.close()

    # -- scheduler ------------------------------------------------------------
    def _pick(self):
        """Index of the first queued request that fits (FCFS with backfill), or None."""
        if not self.idle:
            return None
        for i, req in enumerate(self.queue):
            if self.in_use + req.footprint() <= self.budget:
                return i
        return None

    def _schedule(self):
        with self.cv:
            while True:
                i = self._pick()
                if i is not None:
                    req = self.queue[i]
                    del self.queue[i]
                    slot = self.idle.popleft()
                    self.in_use += req.footprint()
                    req.t_admit = time.perf_counter()
                    req.slot = slot
                    inflight = self.nslots - len(self.idle)
                    self.max_in_flight = max(self.max_in_flight, inflight)
                    t = threading.Thread(target=self._run, args=(slot, req), daemon=True)
                    self.workers.append(t)
                    t.start()
                    continue
                if self.closing and not self.queue and len(self.idle) == self.nslots:
                    return
                self.cv.wait(timeout=0.05)

    def _run(self, slot, req):
        try:
            req.status, req.evals, req.resid, req.stats = self.solve_fn(slot, req)
        except Exception:  # keep the service alive; the request reports the failure
            req.status = -999
        finally:
            req.t_done = time.perf_counter()
            with self.cv:
                self.in_use -= req.footprint()
                self.idle.append(slot)
                self.completed.append(req)
                self.cv.notify_all()
            req.done.set()


def latency_stats(reqs):
    lat = np.array([r.t_done - r.t_arrive for r in reqs])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "count": int(len(lat))}


class BatchServer:
    """Continuous batching at the granularity of the method's outer iterations: admitted
    requests live in ONE batch session (chase_batch_*), whose every step advances all of
    them by one iteration of Algorithm 1 with their filter steps sharing launches (and their
    QR / Rayleigh-Ritz phases overlapping on per-request streams).  Between steps the
    scheduler admits queued requests whose device-memory footprint (matrix, search block and
    solver workspace) fits what the requests in flight leave free -- first come, first
    served, with backfill past a request that does not fit yet -- and completes the requests
    that ended.  A request's result is the one chase_solve computes alone (the grouped
    products are exact integer products; the rest runs per request).

    make_batch() returns the session (default: a Batch on a new handle); `max_in_flight`
    bounds the requests in one session."""

    def __init__(self, hbm_budget=1 << 62, make_batch=None, workspace_bytes=None, max_in_flight=64):
        self.budget = hbm_budget
        self.max_in_flight = max_in_flight
        self._make_batch = make_batch or self._default_batch
        self._workspace_bytes = workspace_bytes or self._chase_workspace_bytes
        self.in_use = 0
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.closing = False
        self.completed = []
        self.max_seen_in_flight = 0
        self.steps = 0
        self._handle = None
        self.sched = threading.Thread(target=self._schedule, daemon=True)
        self.sched.start()

    # -- defaults (the library) -------------------------------------------------
    def _default_batch(self):
        from . import Batch, Handle
        self._handle = Handle(0)
        return Batch(self._handle)

    @staticmethod
    def _chase_workspace_bytes(req):
        import ctypes

        from . import CHASE_C128, CHASE_R64, config_default, lib
        cfg = req.cfg if req.cfg is not None else config_default()
        dt = CHASE_C128 if req.A.element_size() == 16 else CHASE_R64
        b = ctypes.c_size_t()
        lib().chase_workspace_bytes(dt, req.n, req.nev, req.nex, cfg.prec, ctypes.byref(b))
        return int(b.value)

    def footprint(self, req):
        return req.footprint() + self._workspace_bytes(req)

    # -- client side ----------------------------------------------------------------
    def submit(self, req: Request):
        req.t_arrive = time.perf_counter()
        with self.cv:
            if self.footprint(req) > self.budget:
                raise ValueError("request %d needs more memory than the whole budget" % req.rid)
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def drain(self):
        with self.cv:
            self.closing = True
            self.cv.notify_all()
        self.sched.join()

    def close(self):
        self.drain()
        if self._handle is not None:
            self._handle.close()
            self._handle = None

    # -- scheduler ------------------------------------------------------------------
    def _admit(self, batch, live):
        """Moves queued requests that fit into the session (FCFS with backfill)."""
        i = 0
        while i < len(self.queue) and len(live) < self.max_in_flight:
            req = self.queue[i]
            fp = self.footprint(req)
            if self.in_use + fp > self.budget:
                i += 1
                continue
            del self.queue[i]
            self.in_use += fp
            req.t_admit = time.perf_counter()
            req.slot = 0
            from . import BatchProblem
            prob = BatchProblem(req.A, req.V0, req.nev, req.nex, req.bounds, req.cfg)
            try:
                batch.add(prob)
            except Exception:  # the request reports the failure, the service carries on
                self.in_use -= fp
                self._complete(req, -999, None, None, None)
                continue
            live[prob.id] = (req, prob, fp)
            self.max_seen_in_flight = max(self.max_seen_in_flight, len(live))

    def _complete(self, req, status, evals, resid, stats):
        req.status, req.evals, req.resid, req.stats = status, evals, resid, stats
        req.t_done = time.perf_counter()
        self.completed.append(req)
        req.done.set()

    def _schedule(self):
        batch = self._make_batch()
        live = {}
        try:
            while True:
                with self.cv:
                    self._admit(batch, live)
                    if not live:
                        if self.closing and not self.queue:
                            return
                        self.cv.wait(timeout=0.02)
                        continue
                try:
                    finished = batch.step()
                except Exception:  # a session failure ends every request in it
                    finished = list(p for (_, p, _) in live.values())
                    for p in finished:
                        p.status = -999
                self.steps += 1
                with self.cv:
                    for p in finished:
                        req, prob, fp = live.pop(p.id)
                        self.in_use -= fp
                        self._complete(req, prob.status, prob.evals, prob.resid, prob.stats)
                    self.cv.notify_all()
        finally:
            batch.close()

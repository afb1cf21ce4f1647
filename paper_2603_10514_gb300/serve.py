"""Continuous-batching eigensolver service on one GPU.

Requests (dense Hermitian / symmetric eigenproblems of different orders) arrive at
any time.  A request is admitted as soon as a solver slot is idle and its HBM
footprint (A, the search block and the solver workspace) fits in the memory that
admitted requests leave free; admission is first-come-first-served with backfill
(a smaller later request may start while a large one at the head of the queue
waits for memory).  Each slot owns a chase handle with its own CUDA stream and a
workspace sized once, at start-up, for the largest admissible problem, so that
no device allocation happens while requests are in flight.  Admitted requests
run concurrently: their kernels overlap on the device through the slots'
streams, and a request's result does not depend on what else is running (every
kernel's arithmetic order is fixed by the problem's shape only).

Latency of a request = completion time - arrival time (queueing included).
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import (CHASE_C128, CHASE_R64, Handle, chase_solve, config_default, lib)


@dataclass
class Request:
    rid: int
    A: object              # column-major CUDA tensor (float64 / complex128)
    V0: object             # column-major CUDA tensor, n x (nev + nex)
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
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def n(self):
        return self.A.shape[0]

    def footprint(self):
        import ctypes
        dt = CHASE_C128 if self.A.is_complex() else CHASE_R64
        b = ctypes.c_size_t()
        rc = lib().chase_workspace_bytes(dt, self.n, self.nev, self.nex, 0, ctypes.byref(b))
        if rc:
            raise ValueError("invalid request shape")
        esz = self.A.element_size()
        # the workspace is pre-reserved per slot; the request's own device memory is its
        # search block (A is already resident when the request arrives)
        return b.value, esz * self.n * (self.nev + self.nex)


class Server:
    """Runs requests on `slots` concurrent solver slots of one GPU."""

    def __init__(self, device=0, slots=4, max_n=8000, max_ell=480, complex_=True,
                 hbm_budget=None):
        import torch
        self.device = device
        torch.cuda.set_device(device)
        self.handles = [Handle(device) for _ in range(slots)]
        # size every slot's workspace once for the largest admissible problem
        import ctypes
        b = ctypes.c_size_t()
        lib().chase_workspace_bytes(CHASE_C128 if complex_ else CHASE_R64, max_n,
                                    max(1, max_ell - max_ell // 6), max_ell // 6, 0, ctypes.byref(b))
        self.slot_ws = b.value
        self.max_n = max_n
        self._warm(max_n, max_ell, complex_)
        free, _ = torch.cuda.mem_get_info(device)
        self.budget = hbm_budget if hbm_budget is not None else int(0.9 * free)
        self.in_use = 0
        self.queue = collections.deque()
        self.idle = collections.deque(range(slots))
        self.lock = threading.Condition()
        self.stop = False
        self.completed = []
        self.threads = []
        self.sched = threading.Thread(target=self._schedule, daemon=True)
        self.sched.start()

    def _warm(self, max_n, max_ell, complex_):
        """Grow each handle's workspace to the largest admissible size now, so that no
        device allocation happens while requests run."""
        for h in self.handles:
            h.reserve(self.slot_ws)

    def submit(self, req: Request):
        req.t_arrive = time.perf_counter()
        with self.lock:
            self.queue.append(req)
            self.lock.notify_all()
        return req

    def _schedule(self):
        while True:
            with self.lock:
                while not self.stop and not self._admit_one():
                    self.lock.wait(timeout=0.05)
                if self.stop and not self.queue:
                    return

    def _admit_one(self):
        if not self.queue or not self.idle:
            return False
        for i, req in enumerate(self.queue):
            _, need = req.footprint()
            if self.in_use + need <= self.budget and req.n <= self.max_n:
                del self.queue[i]
                slot = self.idle.popleft()
                self.in_use += need
                req.t_admit = time.perf_counter()
                t = threading.Thread(target=self._run, args=(slot, req, need), daemon=True)
                self.threads.append(t)
                t.start()
                return True
        return False

    def _run(self, slot, req, need):
        h = self.handles[slot]
        try:
            rc, ev, res, st, _ = chase_solve(h, req.A, req.V0, req.nev, req.nex, req.bounds,
                                             req.cfg, check=False)
            req.status, req.evals, req.resid, req.stats = rc, ev, res, st
        finally:
            req.t_done = time.perf_counter()
            with self.lock:
                self.in_use -= need
                self.idle.append(slot)
                self.completed.append(req)
                self.lock.notify_all()
            req.done.set()

    def drain(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        self.sched.join()
        for t in self.threads:
            t.join()

    def close(self):
        self.drain()
        for h in self.handles:
            h.close()


def latency_stats(reqs):
    lat = np.array([r.t_done - r.t_arrive for r in reqs])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "count": len(lat)}

#!/usr/bin/env python
"""Benchmark: time-to-solution of Chebyshev-filtered subspace iteration on one GB300.

Workload (default): complex Hermitian n = 10000, A = Q diag(lambda) Q^H with Q
unitary from the QR of a seeded complex Gaussian matrix; the lowest 600
eigenvalues clustered geometrically in [-2, -1], the rest uniform in [-1, 50];
nev = 500, nex = 100, optimised degrees in [10, 36] (first filter degree 20),
tol 1e-10.  Synthetic, seeded stand-in for the paper's DFT/BSE matrices.

One step = one complete chase_solve (Algorithm 1: filter, kappa-driven QR,
Rayleigh-Ritz, residuals, locking) from the same random start block, inputs
resident in HBM.  A (1.6 GB) is far larger than the 129 MB L2, so no flush is
needed between steps.  Several GPUs (torchrun) run independent replicas.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("time-to-solution for nev pairs at resid<=1e-10 & filter TFLOP/s vs FP64 peak; "
          "solves/s, p50/p99")
# FP64 DFMA peak of GB300 derived from unit counts and the maximum SM clock:
# 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (a DFMA probe measured 1.203 TFLOP/s at ~2.0 GHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Dense BF16 tensor peaks measured on GB300 with cuBLAS (burst, and back to back for seconds
# under the power cap), read from MEASURED_PEAKS.json next to this file when it is present;
# the numbers below are the ones it held when this was written.
def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"])
    except (OSError, KeyError, ValueError, TypeError):
        return 1978.3, 1717.0


BF16_PEAK_TFLOPS, BF16_SUSTAINED_TFLOPS = _measured_peaks()
# BF16 tensor-core work per FP64-equivalent flop in the emulated mode: one modular product per
# modulus of the Ozaki scheme II (17 moduli <= 256); a complex product is three real products
# of order n (Gauss's form: Ar Vr, Ai Vi, (Ar + Ai)(Vr + Vi)), 3 x 2 n^2 per column against the
# 8 n^2 FP64-equivalent flops of a complex column MatVec: 17 x 3/4 = 12.75 (17 for real).
OZAKI_MODULI = 17
OZAKI_PAIRS = OZAKI_MODULI * 0.75   # the default workload is complex
# DRAM bytes (read + write) of one emulated product of the default workload (complex
# n = 10000, 600 active columns), measured by one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum, 1 pass): the grouped modular products of the three real products
# 12.12 GB read and 0.456 GB written; the reconstruction 0.404 GB read and 0.076 GB written.
# Launches with fewer active columns read the same residue planes of A, which are most of it.
OZ_TRAFFIC_PER_LAUNCH = 12.125e9 + 0.456e9 + 0.404e9 + 0.076e9
# Column MatVecs of one complete solve of the default workload as counted by the GPU path
# (filter MatVecs plus the 2 (ell - k) products of Rayleigh-Ritz and residuals per
# iteration); used to scale the oracle's timed sample to a whole solve.  Measured on a
# GB300: 114037 filter MatVecs + 8690 Rayleigh-Ritz / residual products over 9 iterations.
REF_MATVECS_PER_SOLVE = 122727


DTYPES = {"fp64": "f64 (complex128, DFMA)",
          "fp64_emu": "f64 (complex128; A*V by the Ozaki scheme on bf16 tensor cores, exact "
                      "integer accumulation; QR/RR/residuals f64)",
          "bf16x3": "bf16x3 filter with f32 accumulation, then f64-emulated filter; f64 QR/RR"}
PRECS = {"fp64": lambda P: P.CHASE_FP64, "fp64_emu": lambda P: P.CHASE_FP64_EMU,
         "bf16x3": lambda P: P.CHASE_BF16X3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--nev", type=int, default=500)
    ap.add_argument("--nex", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-cols", type=int, default=8)
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "filter", "sequence", "serve", "kappa", "batch"],
                    help="solve: the headline time-to-solution; filter: chase_filter alone "
                         "(kernel-level timing and small cases for profilers); sequence: 20 "
                         "correlated real problems with warm starts; serve: a stream of "
                         "requests through the continuous-batching service; batch: many uneven "
                         "problems in one batch session against one at a time")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--seq-len", type=int, default=20)
    ap.add_argument("--serve-count", type=int, default=256)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="Poisson arrival rate (requests/s); 0 = measure the saturated "
                         "throughput first and use 0.8 of it")
    ap.add_argument("--caps", default="36,48,64",
                    help="kappa mode: degree caps of the optimised-degree runs")
    ap.add_argument("--ncols", type=int, default=600, help="filter mode: block width")
    ap.add_argument("--degree", type=int, default=20, help="filter mode: degree of every column")
    ap.add_argument("--autotune", type=int, default=0, choices=[0, 1],
                    help="1: the emulated products tune their launch plans during the warm-up "
                         "solves (chase_config.autotune); the timed solves use the picks")
    ap.add_argument("--prec", default="fp64_emu", choices=["fp64", "fp64_emu", "bf16x3"],
                    help="A*V arithmetic: fp64 (DFMA), fp64_emu (Ozaki scheme on the BF16 tensor "
                         "cores, FP64-accurate), bf16x3 (BF16x3 filter while residuals are large, "
                         "then fp64_emu)")
    return ap.parse_args()


def run_filter(args):
    """chase_filter on n x ncols, every column at the same degree: filter TFLOP/s from CUDA
    events on the handle's stream (FP64 complex, 8 n^2 flops per column MatVec)."""
    import numpy as np
    import torch

    import paper_2603_10514_gb300 as P
    import workloads as W
    P.build()
    n, k = args.n, args.ncols
    lam = W.spectrum_clustered(n, min(k, n), 2)
    A = W.known_spectrum_matrix(lam, 2, True, device="cuda")
    V = torch.from_numpy(np.ascontiguousarray(W.start_block(n, k, 2, True).T)).cuda().mT
    out = torch.empty_like(V.mT).mT
    l1, le, bs = W.bounds_for(lam, k)
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    stream = torch.cuda.current_stream()
    h = P.Handle(0, stream=stream.cuda_stream)
    degs = [args.degree] * k
    prec = PRECS[args.prec](P)
    for _ in range(args.warmup):
        P.chase_filter(h, A, V, degs, c, e, l1, out=out, prec=prec)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        P.chase_filter(h, A, V, degs, c, e, l1, out=out, prec=prec)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    flops = 8.0 * n * n * k * args.degree
    h.close()
    line = {"mode": "filter", "prec": args.prec, "n": n, "ncols": k, "degree": args.degree,
            "s_per_filter": t, "tflops_fp64_equivalent": flops / t / 1e12}
    if args.prec == "fp64":
        line["frac_of_fp64_peak"] = flops / t / 1e12 / FP64_PEAK_TFLOPS
    else:
        # BF16 tensor-core work per step: BF16x3 three products of the stacked real operator
        # (2n x 2n); the Ozaki scheme II 17 modular products of each of Gauss's three real
        # products of order n
        if args.prec == "bf16x3":
            tc = 3 * 2.0 * (2 * n) * (2 * n) * k * args.degree / t / 1e12
        else:
            tc = OZAKI_MODULI * 3 * 2.0 * n * n * k * args.degree / t / 1e12
        line["bf16_tensor_tflops"] = tc
        line["frac_of_bf16_peak"] = tc / BF16_PEAK_TFLOPS
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_aggregate(local_seconds, steps, world, dist=None, device=None):
    """Replicas only: every rank solves its own problem.  The job's time is the slowest
    rank's (max over ranks); the job's throughput counts every rank's solves."""
    total = float(local_seconds)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total, world * steps / total


def make_problem(args, device):
    import workloads as W
    prob = W.c2_complex_clustered(n=args.n, nev=args.nev, nex=args.nex, seed=2)
    A = W.known_spectrum_matrix(prob.lam, prob.seed, prob.complex_, device=device)
    V0 = W.start_block(prob.n, prob.ell, prob.seed, prob.complex_)
    return prob, A, V0


def oracle_sample(A_host, prob, cols, deg=2):
    """Times the oracle's filter (Algorithm 4, plain C FP64, OpenMP over rows) on `cols`
    columns of the workload at degree `deg`: returns seconds per column MatVec."""
    import numpy as np

    import oracle
    import workloads as W
    V = W.start_block(prob.n, cols, prob.seed + 99, prob.complex_)
    l1, le, bs = prob.bounds
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.filter(A_host, V, [deg] * cols, c, e, l1)
    dt = time.perf_counter() - t0
    return dt / (cols * deg), dt


def device_view(ptr, n, ncols, ld, complex_):
    """A torch view (no copy) of a column-major device block given by its raw pointer,
    through the CUDA array interface."""
    import torch

    class _Block:
        __cuda_array_interface__ = {
            "shape": (ncols, ld), "typestr": "<c16" if complex_ else "<f8",
            "data": (int(ptr), False), "version": 3, "strides": None}

    return torch.as_tensor(_Block(), device="cuda").mT[:n, :]


def run_kappa(args):
    """Figure 2 analogue: per iteration, the estimate of Eq. full-est (kappa_est, logged by
    the solver) against the exact kappa_2 of the block [Y V] Algorithm 3 factors (singular
    values of a host copy, taken through the solver's filtered-block hook), without degree
    optimisation (degree 20) and with it (first degree 20, caps from --caps: 36 as in the
    paper's runs, and higher)."""
    import numpy as np
    import torch

    import paper_2603_10514_gb300 as P
    import workloads as W
    P.build()
    n = args.n if args.n != 10000 else 3000
    nev = args.nev if args.nev != 500 else 150
    nex = args.nex if args.nex != 100 else 30
    out = {"mode": "kappa", "prec": args.prec, "n": n, "nev": nev, "nex": nex, "runs": []}
    for name, prob in [("complex clustered", W.c2_complex_clustered(n=n, nev=nev, nex=nex, seed=2)),
                       ("real uniform", W.Problem("real", n, nev, nex, False, 1,
                                                  W.spectrum_uniform(n, -1, 1, 1)))]:
        A = W.known_spectrum_matrix(prob.lam, prob.seed, prob.complex_, device="cuda")
        V0 = W.start_block(n, prob.ell, prob.seed, prob.complex_)
        caps = [int(x) for x in args.caps.split(",") if x]
        for opt, cap in [(False, 36)] + [(True, c) for c in caps]:
            kap = {}

            def hook(ptr, nn, ll, ld, it):
                X = device_view(ptr, nn, ll, ld, prob.complex_).cpu().numpy()
                sv = np.linalg.svd(X, compute_uv=False)
                kap[it] = float(sv[0] / sv[-1])

            h = P.Handle(0)
            cfg = P.config_default(opt_degree=int(opt), deg_init=20, deg_max=cap,
                                   prec=PRECS[args.prec](P))
            keep = P.with_filtered_hook(cfg, hook)
            Vd = torch.from_numpy(np.ascontiguousarray(V0.T)).cuda().mT
            rc, ev, res, st, logs = P.chase_solve(h, A, Vd, nev, nex, prob.bounds, cfg)
            h.close()
            del keep
            rows = [{"it": g["iteration"], "locked": g["locked_before"], "variant": g["variant"],
                     "log10_kappa_est": g["log_cond_est_paper"] / np.log(10.0),
                     "log10_kappa_est_locked_aware": g["log_cond_est_locked"] / np.log(10.0),
                     "log10_kappa_exact": float(np.log10(kap[g["iteration"]]))} for g in logs]
            ratio = [r["log10_kappa_est"] - r["log10_kappa_exact"] for r in rows]
            out["runs"].append({"problem": name, "opt": opt, "deg_max": cap, "status": rc,
                                "iterations": st["iterations"], "matvecs": st["matvecs"],
                                "t_total_s": st["t_total"],
                                "qr_variants": [r["variant"] for r in rows],
                                "log10_est_over_exact_max": max(ratio) if ratio else None,
                                "log10_est_over_exact_min": min(ratio) if ratio else None,
                                "estimate_bounds_exact_before_locking":
                                    all(r["log10_kappa_est"] >= r["log10_kappa_exact"]
                                        for r in rows if r["locked"] == 0),
                                "estimate_bounds_exact_in_all_iterations":
                                    all(r["log10_kappa_est"] >= r["log10_kappa_exact"] for r in rows),
                                "locked_aware_bounds_exact_in_all_iterations":
                                    all(r["log10_kappa_est_locked_aware"] >= r["log10_kappa_exact"]
                                        for r in rows),
                                "per_iteration": rows})
    print(json.dumps(out), flush=True)


def run_sequence(args):
    """SCF-like sequence: A_0 real symmetric (n = 8000, lambda uniform in [-1, 1]),
    A_{k+1} = A_k + 1e-3 (G + G^T)/(2 sqrt n); each problem (nev 400, nex 80) is
    warm-started from the previous problem's final block.  All matrices are generated
    and resident before the timed region; the timed region is the whole chain."""
    import numpy as np
    import torch

    import paper_2603_10514_gb300 as P
    import workloads as W
    P.build()
    n = args.n if args.n != 10000 else 8000
    nev = args.nev if args.nev != 500 else 400
    nex = args.nex if args.nex != 100 else 80
    prob = W.c4_sequence_base(n=n, nev=nev, nex=nex, seed=4)
    As = [W.known_spectrum_matrix(prob.lam, prob.seed, False, device="cuda")]
    g = torch.Generator(device="cuda").manual_seed(4)
    for k in range(1, args.seq_len):
        G = torch.randn(n, n, generator=g, device="cuda", dtype=torch.float64)
        E = 1e-3 * (G + G.T) / (2.0 * n ** 0.5)
        As.append((As[-1] + E).mT.contiguous().mT)
        del G, E
    V0 = torch.from_numpy(np.ascontiguousarray(W.start_block(n, prob.ell, 4, False).T)).cuda().mT
    stream = torch.cuda.current_stream()
    h = P.Handle(0, stream=stream.cuda_stream)
    cfg = P.config_default(opt_degree=1, prec=PRECS[args.prec](P))
    l1, le, bs = prob.bounds

    def chain():
        V = V0.clone()
        out = []
        lam1 = l1
        for k, A in enumerate(As):
            bounds = (lam1, le, bs + 3e-3 * k)
            rc, ev, res, st, _ = P.chase_solve(h, A, V, prob.nev, prob.nex, bounds, cfg)
            out.append((rc, float(res.max()), st["iterations"], st["matvecs"]))
            lam1 = float(ev[0]) - 1e-2
        return out

    chain()  # warm-up (workspace, code paths)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    res = chain()
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    h.close()
    print(json.dumps({"mode": "sequence", "prec": args.prec, "n": n, "nev": nev, "nex": nex,
                      "problems": len(As), "seconds": t, "problems_per_s": len(As) / t,
                      "all_converged": all(r[0] == 0 and r[1] < 1e-10 for r in res),
                      "iterations": [r[2] for r in res], "matvecs": [r[3] for r in res]}), flush=True)


def run_serve(args):
    """Serving stream: requests with n log-uniform in [500, 8000], real / complex 50/50,
    nev = 5% of n, nex = nev/5, lambda uniform in [-1, 1], Poisson arrivals at a fixed
    seed, admitted by HBM footprint.  Two engines on the same stream: `batch` (the requests
    in flight share one batch session, their filter steps in shared launches, admitted and
    completed between outer iterations) and `streams` (whole solves overlapping on
    concurrent slot handles).  Each engine's saturated rate (all requests at once) is
    measured; the batch engine is then driven at 0.8 of its saturated rate for latency."""
    import numpy as np
    import torch

    import paper_2603_10514_gb300 as P
    import workloads as W
    from paper_2603_10514_gb300.serve import BatchServer, Request, Server, latency_stats
    P.build()
    specs = W.serving_stream(count=args.serve_count, seed=5)
    mats = []
    for s_ in specs:
        lam = W.spectrum_uniform(s_["n"], -1.0, 1.0, s_["seed"])
        A = W.known_spectrum_matrix(lam, s_["seed"], s_["complex"], device="cuda")
        V0 = W.start_block(s_["n"], s_["nev"] + s_["nex"], s_["seed"], s_["complex"])
        V0 = torch.from_numpy(np.ascontiguousarray(V0.T)).cuda().mT
        mats.append((s_, lam, A, V0))
    cfg = P.config_default(opt_degree=1, prec=PRECS[args.prec](P))
    import ctypes
    b = ctypes.c_size_t()
    P.lib().chase_workspace_bytes(P.CHASE_C128, 8000, 400, 80, PRECS[args.prec](P), ctypes.byref(b))
    free, _ = torch.cuda.mem_get_info()
    budget_streams = int(0.85 * free) - args.serve_slots * b.value
    budget_batch = int(0.85 * free)

    def run(engine, rate, seed):
        if engine == "batch":
            srv = BatchServer(hbm_budget=budget_batch)
        else:
            srv = Server(slots=args.serve_slots, hbm_budget=budget_streams,
                         make_handle=lambda i: P.Handle(0), slot_workspace=b.value)
        rng = np.random.default_rng(seed)
        reqs = []
        t0 = time.perf_counter()
        t_next = 0.0
        for (s_, lam, A, V0) in mats:
            if rate > 0:
                t_next += rng.exponential(1.0 / rate)
                delay = t0 + t_next - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            req = Request(rid=s_["id"], A=A, V0=V0.clone(), nev=s_["nev"], nex=s_["nex"],
                          bounds=W.bounds_for(lam, s_["nev"] + s_["nex"]), cfg=cfg)
            reqs.append((srv.submit(req), lam))
        srv.drain()
        wall = time.perf_counter() - t0
        inflight = srv.max_seen_in_flight if engine == "batch" else srv.max_in_flight
        srv.close()
        ok = all(r.status == 0 and float(np.max(r.resid)) < 1e-10 and
                 float(np.abs(r.evals - lam[:r.nev]).max()) <= 1e-10 for r, lam in reqs)
        return [r for r, _ in reqs], wall, ok, inflight

    out = {"mode": "serve", "prec": args.prec, "requests": len(mats)}
    sat = {}
    for engine in ("streams", "batch"):
        reqs, wall, ok, inflight = run(engine, 0.0, 0)
        sat[engine] = len(mats) / wall
        out["saturated_" + engine] = {"solves_per_s": sat[engine], "wall_s": wall, "all_correct": ok,
                                      "max_in_flight": inflight, "latency": latency_stats(reqs)}
    rate = args.serve_rate if args.serve_rate > 0 else 0.8 * sat["batch"]
    reqs, wall, ok, inflight = run("batch", rate, 5)
    out.update({"engine": "batch", "arrival_rate_per_s": rate, "solves_per_s": len(reqs) / wall,
                "wall_s": wall, "latency": latency_stats(reqs), "all_correct": ok,
                "max_in_flight": inflight, "streams_slots": args.serve_slots,
                "batch_over_streams_saturated": sat["batch"] / sat["streams"]})
    print(json.dumps(out), flush=True)


def oracle_full_solve_c1():
    """One complete oracle solve (Algorithm 1, every step) of the small real workload
    (n = 1000, nev 20, nex 10, fixed degree 20): the measured anchor of the extrapolated
    CPU baseline.  Returns seconds, column MatVecs (filter + Rayleigh-Ritz / residual
    products) and the status."""
    import oracle
    import workloads as W
    prob = W.c1_real_small()
    A = W.known_spectrum_matrix(prob.lam, prob.seed, False, device="cpu").numpy()
    V0 = W.start_block(prob.n, prob.ell, prob.seed, False)
    l1, le, bs = prob.bounds
    oracle.lib()
    t0 = time.perf_counter()
    r = oracle.solve(A, V0, prob.nev, prob.nex, opt_degree=False, deg_init=prob.deg_init,
                     lambda1=l1, lambda_ell=le, b_sup=bs)
    dt = time.perf_counter() - t0
    mv = r["summary"]["matvecs"] + 2 * sum(prob.ell - g["locked_before"] for g in r["logs"])
    return dt, mv, r["status"], prob.n


def cpu_anchor(per_mv_c2, n_c2):
    """The C1 full solve timed and set beside the C2 sample: the oracle computes in complex
    arithmetic whatever the input type, so a column MatVec costs ~n^2 work at any size and the
    C1 per-MatVec time scaled by (n_C2 / n_C1)^2 predicts the C2 sample's."""
    dt, mv, status, n1 = oracle_full_solve_c1()
    per_mv_c1 = dt / mv
    return {"workload": "real symmetric n=%d, nev 20, nex 10, degree 20 (complete oracle solve)" % n1,
            "solve_s": dt, "status": status, "column_matvecs": mv, "s_per_matvec": per_mv_c1,
            "s_per_matvec_scaled_to_n%d" % n_c2: per_mv_c1 * (n_c2 / n1) ** 2,
            "s_per_matvec_sampled_at_n%d" % n_c2: per_mv_c2}


def run_batch(args):
    """Many uneven problems at once: `--batch-count` requests of the serving mix (n
    log-uniform in [500, 4000], real / complex 50/50, nev = 5 % of n, nex = nev / 5, lambda
    uniform in [-1, 1]) solved by one batch session (their filter steps grouped into shared
    launches) and, for comparison, one chase_solve after another on the same handle.
    Inputs resident; CUDA events on the handle's stream; every result checked against the
    known spectrum."""
    import numpy as np
    import torch

    import paper_2603_10514_gb300 as P
    import workloads as W
    P.build()
    specs = W.serving_stream(count=args.batch_count, seed=6, n_lo=500, n_hi=4000)
    cfg = P.config_default(opt_degree=1, prec=PRECS[args.prec](P))
    mats = []
    for s_ in specs:
        lam = W.spectrum_uniform(s_["n"], -1.0, 1.0, s_["seed"])
        A = W.known_spectrum_matrix(lam, s_["seed"], s_["complex"], device="cuda")
        V0 = W.start_block(s_["n"], s_["nev"] + s_["nex"], s_["seed"], s_["complex"])
        mats.append((s_, lam, A, torch.from_numpy(np.ascontiguousarray(V0.T)).cuda().mT))
    stream = torch.cuda.current_stream()
    h = P.Handle(0, stream=stream.cuda_stream)

    def batched():
        probs = [P.BatchProblem(A, V0.clone(), s_["nev"], s_["nex"],
                                W.bounds_for(lam, s_["nev"] + s_["nex"]), cfg) for (s_, lam, A, V0) in mats]
        P.chase_solve_batch(h, probs, cfg)
        return [(p.status, p.evals, p.resid) for p in probs]

    def one_by_one():
        out = []
        for (s_, lam, A, V0) in mats:
            rc, ev, res, _, _ = P.chase_solve(h, A, V0.clone(), s_["nev"], s_["nex"],
                                              W.bounds_for(lam, s_["nev"] + s_["nex"]), cfg)
            out.append((rc, ev, res))
        return out

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    batched()  # warm-up (workspace pool, code paths)
    one_by_one()
    rb, tb = timed(batched)
    rs, ts = timed(one_by_one)
    h.close()

    def correct(res):
        return all(r[0] == 0 and float(np.max(r[2])) < 1e-10 and
                   float(np.abs(r[1] - lam[:s_["nev"]]).max()) <= 1e-10 * float(np.abs(lam).max())
                   for r, (s_, lam, _, _) in zip(res, mats))

    same = all(np.array_equal(a[1], b[1]) for a, b in zip(rb, rs))
    print(json.dumps({"mode": "batch", "prec": args.prec, "problems": len(mats),
                      "n_range": [min(s_["n"] for s_, _, _, _ in mats), max(s_["n"] for s_, _, _, _ in mats)],
                      "batched_s": tb, "batched_solves_per_s": len(mats) / tb,
                      "one_by_one_s": ts, "one_by_one_solves_per_s": len(mats) / ts,
                      "speedup": ts / tb, "all_correct": correct(rb) and correct(rs),
                      "batched_equals_single_bitwise": same}), flush=True)


def run_reference(args, rank):
    """The oracle arm: the CPU oracle timed on the host cores (rank 0 only).  A complete
    oracle solve of this workload takes hours, so each step times a bounded sample of it
    (the oracle's filter on a few columns of the same matrix); `ms_per_step` is the measured
    time of that sample and `value` the solves/s it implies for a whole solve (the sample's
    time per column MatVec times the MatVecs of a solve)."""
    if rank != 0:
        return
    import numpy as np

    import workloads as W
    prob = W.c2_complex_clustered(n=args.n, nev=args.nev, nex=args.nex, seed=2)
    A = W.known_spectrum_matrix(prob.lam, prob.seed, prob.complex_, device="cpu").numpy()
    default = (prob.n, prob.nev, prob.nex) == (10000, 500, 100)
    mv = REF_MATVECS_PER_SOLVE if default else _estimate_matvecs(prob)
    for _ in range(args.warmup):
        oracle_sample(A, prob, max(1, args.cpu_sample_cols // 4), deg=1)
    per_mv, sample_s = [], []
    for _ in range(args.steps):
        pm, dt = oracle_sample(A, prob, args.cpu_sample_cols)
        per_mv.append(pm)
        sample_s.append(dt)
    t_solve = statistics.mean(per_mv) * mv
    cores = os.cpu_count()
    value = 1.0 / t_solve
    sample = ("each step: the oracle's filter on %d columns x degree 2 of the n=%d matrix "
              "(%.1f s measured); solves/s = 1 / (its time per column MatVec x %d column MatVecs "
              "per solve)" % (args.cpu_sample_cols, prob.n, statistics.mean(sample_s), mv))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(sample_s) * 1e3, "ms_per_solve_extrapolated": t_solve * 1e3,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)", "data": "synthetic",
        "config": _config(args, prob),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _estimate_matvecs(prob):
    # a conservative count when no GPU run is at hand: two full-width filters of degree 20
    # plus three more iterations at the mean optimised degree, and their RR products
    return int(prob.ell * 20 * 2 + prob.ell * 23 * 3 + 2 * prob.ell * 5)


def _config(args, prob):
    prec = getattr(args, "prec", "fp64_emu")
    return {"workload": "complex Hermitian n=%d, nev=%d, nex=%d, clustered lowest %d in [-2,-1], "
                        "rest U[-1,50], degrees 10-36 (init 20), tol 1e-10, %s filter"
                        % (prob.n, prob.nev, prob.nex, prob.ell, prec.upper()),
            "n": prob.n, "nev": prob.nev, "nex": prob.nex, "dtype": "complex128",
            "precision": prec, "l2": "inputs larger than L2 (A is %.1f GB)" % (16 * prob.n ** 2 / 1e9),
            "parallelism": "replicas (1 problem per GPU)" if args.gpus > 1 else "single GPU"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.mode == "filter":
        run_filter(args)
        return
    if args.mode == "sequence":
        run_sequence(args)
        return
    if args.mode == "kappa":
        run_kappa(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "batch":
        run_batch(args)
        return
    import numpy as np
    import torch

    import paper_2603_10514_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    P.build()
    device = "cuda:%d" % local
    prob, A, V0 = make_problem(args, device)
    n, l = prob.n, prob.ell
    V0d = torch.from_numpy(np.ascontiguousarray(V0.T)).to(device).mT
    Vw = torch.empty_like(V0d.mT).mT
    stream = torch.cuda.current_stream()
    h = P.Handle(local, stream=stream.cuda_stream)
    cfg = P.config_default(opt_degree=1, deg_init=prob.deg_init, deg_min=prob.deg_min,
                           deg_max=prob.deg_max, tol=prob.tol,
                           prec=PRECS[args.prec](P), autotune=args.autotune)
    bounds = prob.bounds

    def one_solve():
        Vw.copy_(V0d)
        return P.chase_solve(h, A, Vw, prob.nev, prob.nex, bounds, cfg)

    for _ in range(args.warmup):
        rc, ev, res, st, logs = one_solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    results = []
    evs[0].record(stream)
    for s in range(args.steps):
        rc, ev, res, st, logs = one_solve()
        evs[s + 1].record(stream)
        results.append((rc, ev, res, st, logs))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_s = [evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(args.steps)]
    total, value = replica_aggregate(evs[0].elapsed_time(evs[-1]) / 1e3, args.steps, world, dist,
                                     device)
    # correctness of every timed solve
    lam = prob.lam[:prob.nev]
    ok = all(r[0] == 0 and float(r[2].max()) < prob.tol for r in results)
    eval_err = max(float(np.abs(r[1] - lam).max()) for r in results)
    rc, ev, res, st, logs = results[-1]
    launches = sum(r[3]["kernel_launches"] for r in results)
    # roofline of the dominant kernel: the filter product (CUDA events around each product
    # launch on the handle's stream, summed by the library, divided by the launch count).
    # achieved = the method's algorithmic work (column MatVecs x 8 n^2 complex / 2 n^2 real
    # flops, FP64) per launch / the launch's duration.
    nl = max(1, st["filter_launches"])
    dur_launch = st["t_filter_product"] / nl
    fl_launch = st["filter_flops"] / nl
    achieved = fl_launch / dur_launch / 1e12 if dur_launch > 0 else None
    # algorithmic DRAM bytes of one full-width product: A once (16 n^2 complex / 8 n^2 real)
    # plus V_{i-1}, V_{i-2} read and V_i written (3 x 16 n ell)
    esz = 16 if prob.complex_ else 8
    alg_bytes = esz * n * n + 3 * esz * n * l
    if args.prec == "fp64":
        roof = {"kernel": "gemm_kernel (FP64 DFMA filter product, fused three-term epilogue)",
                "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz", "traffic": None,
                "algorithmic_bytes": alg_bytes}
    else:
        # the FP64-accurate products run on the BF16 tensor cores: the method's FP64 work is
        # set against the BF16 pipe's measured sustained peak (frac), and the BF16 modular
        # products the kernels actually issue (OZAKI_PAIRS per FP64-equivalent flop; 3 for the
        # BF16x3 filter iterations) give the tensor pipe's own efficiency (frac_tensor_pipe)
        lp = st["filter_flops_lowprec"]
        tc_flops = OZAKI_PAIRS * (st["filter_flops"] - lp) + 3.0 * lp
        pipe = tc_flops / nl / dur_launch / 1e12 if dur_launch > 0 else None
        traffic = (OZ_TRAFFIC_PER_LAUNCH if (OZ_TRAFFIC_PER_LAUNCH and lp == 0 and args.n == 10000
                                             and args.prec == "fp64_emu") else None)
        roof = {"kernel": "ozm_group_kernel + crt3_kernel (Ozaki scheme II FP64 product: 17 modular "
                          "BF16 tcgen05 products of each of Gauss's three real products, CRT "
                          "reconstruction)" +
                          (" + tc_filter_bf16x3_kernel" if lp > 0 else ""),
                "bound": "tensor", "achieved": achieved, "peak": BF16_SUSTAINED_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / BF16_SUSTAINED_TFLOPS if achieved else None,
                "achieved_meaning": "FP64-equivalent flops of the method (column MatVecs x 8 n^2) "
                                    "per product launch / its CUDA-event duration",
                "peak_source": "measured: cuBLAS bf16, sustained (MEASURED_PEAKS.json)",
                "tensor_pipe_tflops": pipe,
                "frac_tensor_pipe": pipe / BF16_SUSTAINED_TFLOPS if pipe else None,
                "tensor_pipe_meaning": "BF16 modular-product flops issued (%.2f per FP64-equivalent "
                                       "flop) per launch / duration" % OZAKI_PAIRS,
                "vs_fp64_dfma_peak": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": traffic, "algorithmic_bytes": alg_bytes,
                "traffic_vs_algorithmic": traffic / alg_bytes if traffic else None}
    fp64_equiv = st["filter_flops"] / st["t_filter"] / 1e12 if st["t_filter"] > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.prec], "data": "synthetic",
        "config": _config(args, prob),
        "time_to_solution_s": {"mean": total / args.steps, "p50": statistics.median(step_s),
                               "p99": max(step_s)},
        "filter_tflops": fp64_equiv,
        "filter_frac_of_fp64_peak": fp64_equiv / FP64_PEAK_TFLOPS if fp64_equiv else None,
        "converged": ok, "max_abs_eval_err_vs_known": eval_err, "max_resid": float(res.max()),
        "iterations": st["iterations"], "matvecs": st["matvecs"],
        "qr_variants": {"cholqr1": st["n_chol1"], "cholqr2": st["n_chol2"],
                        "shifted_cholqr2": st["n_shifted"], "householder": st["n_hhqr"]},
        "phase_s": {k: st[k] for k in ("t_filter", "t_qr", "t_rr", "t_rr_eig", "t_resid", "t_total",
                                        "t_filter_lowprec")},
        "jacobi_sweeps": st["jacobi_sweeps"],
        "lowprec_iterations": st["n_lowprec_iters"],
        "iteration_log": [{"it": g["iteration"], "locked": g["locked_before"],
                           "variant": g["variant"], "log10_cond_est": g["log_cond_est"] / 2.302585092994046,
                           "matvecs": g["matvecs"], "deg": [g["deg_min"], g["deg_max"]]} for g in logs],
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # end to end through the public API with host buffers
    if not args.no_e2e:
        def pinned(rows, cols):  # column-major pinned host buffer
            return torch.empty((cols, rows), dtype=A.dtype, pin_memory=True).mT

        def devbuf(rows, cols):  # column-major device buffer
            return torch.empty((cols, rows), dtype=A.dtype, device=device).mT

        A_h, V0_h, Y_h = pinned(n, n), pinned(n, l), pinned(n, prob.nev)
        A_h.copy_(A)
        V0_h.copy_(V0d)
        A_d, V_d = devbuf(n, n), devbuf(n, l)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            A_d.copy_(A_h, non_blocking=True)
            V_d.copy_(V0_h, non_blocking=True)
            rc2, ev2, res2, st2, _ = P.chase_solve(h, A_d, V_d, prob.nev, prob.nex, bounds, cfg)
            Y_h.copy_(V_d[:, :prob.nev], non_blocking=True)
            torch.cuda.synchronize()
        t_e2e, _ = replica_aggregate(time.perf_counter() - t0, args.steps, world, dist, device)
        h2d = A_h.numel() * A_h.element_size() + V0_h.numel() * V0_h.element_size()
        d2h = Y_h.numel() * Y_h.element_size() + 2 * 8 * prob.nev
        line["e2e"] = {"value": world * args.steps / t_e2e, "unit": "solves/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                       "converged": bool(rc2 == 0 and float(res2.max()) < prob.tol),
                       "iterations": st2["iterations"],
                       "max_abs_eval_err_vs_known": float(np.abs(ev2 - lam).max())}
        del A_d, V_d
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        A_host = A.cpu().numpy()
        per_mv, dt = oracle_sample(A_host, prob, args.cpu_sample_cols)
        mv_solve = st["matvecs"] + 2 * sum(l - g["locked_before"] for g in logs)
        t_cpu = per_mv * mv_solve
        line["cpu_baseline"] = {
            "value": 1.0 / t_cpu, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle filter (plain C FP64, OpenMP) on %d columns x degree 2 of the same A, "
                      "%.1f s; scaled by the %d column MatVecs of the GPU solve (filter + RR + "
                      "residual products; QR and Jacobi not counted)" % (args.cpu_sample_cols, dt, mv_solve),
            "measured_anchor": cpu_anchor(per_mv, n)}
    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Python binding of the GB300 Chebyshev-filtered subspace iteration library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libchase_gb300.so`` behind the C ABI of ``include/chase_gb300.h``.
There is no CPU fallback; if the library has not been built (``build()``) or no
CUDA device is present, the calls raise.

Device buffers are torch tensors on the handle's device in column-major layout
(strides (1, ld)); host arrays are numpy.  The entry points keep the C names:
``chase_solve``, ``chase_filter``, ``chase_qr``, ``chase_cond_est``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchase_gb300.so")

CHASE_R64, CHASE_C128 = 0, 1
CHASE_FP64, CHASE_TF32, CHASE_BF16X3, CHASE_FP64_EMU = 0, 1, 2, 3
CHASE_OK, CHASE_NOT_CONVERGED, CHASE_CHOL_FAILED = 0, 1, 2
CHASE_ERR_CUDA, CHASE_ERR_OOM, CHASE_ERR_TIMEOUT, CHASE_ERR_NONFINITE, CHASE_ERR_UNSUPPORTED = 3, 4, 5, 6, 7
CHASE_ERR_TOO_LARGE = 8
CHASE_FILTER_NOALLOC_MAX_BYTES = 32 << 20
QR_VARIANTS = {1: "cholqr1", 2: "cholqr2", 3: "shifted_cholqr2", 4: "householder"}
CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy

EXPORTED = ["chase_create", "chase_destroy", "chase_config_default", "chase_workspace_bytes",
            "chase_solve", "chase_filter", "chase_qr", "chase_qr_prec", "chase_cond_est",
            "chase_status_string",
            "chase_filter_noalloc", "chase_reserve_workspace", "chase_lanczos_bounds",
            "chase_selftest_wait_timeout", "chase_batch_create", "chase_batch_destroy",
            "chase_batch_add", "chase_batch_step", "chase_batch_pending", "chase_solve_batch",
            "chase_autotune_table", "chase_autotune_clear"]


class ChaseError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %d (%s)" % (where, code, status_string(code)))


class Config(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("deg_init", ctypes.c_int),
                ("deg_min", ctypes.c_int), ("deg_max", ctypes.c_int), ("opt_degree", ctypes.c_int),
                ("eta", ctypes.c_double), ("cond_hi", ctypes.c_double), ("cond_lo", ctypes.c_double),
                ("qr_force", ctypes.c_int), ("prec", ctypes.c_int), ("mp_switch", ctypes.c_double),
                ("filtered_hook", ctypes.c_void_p), ("filtered_hook_ctx", ctypes.c_void_p),
                ("cond_est_mode", ctypes.c_int), ("graph_filter", ctypes.c_int),
                ("autotune", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


FILTERED_HOOK = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int)


class Bounds(ctypes.Structure):
    _fields_ = [("lambda1", ctypes.c_double), ("lambda_ell", ctypes.c_double), ("b_sup", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("locked", ctypes.c_int), ("matvecs", ctypes.c_longlong),
                ("n_chol1", ctypes.c_int), ("n_chol2", ctypes.c_int), ("n_shifted", ctypes.c_int),
                ("n_hhqr", ctypes.c_int), ("n_chol_failures", ctypes.c_int),
                ("t_total", ctypes.c_double), ("t_filter", ctypes.c_double), ("t_qr", ctypes.c_double),
                ("t_rr", ctypes.c_double), ("t_resid", ctypes.c_double), ("filter_flops", ctypes.c_double),
                ("kernel_launches", ctypes.c_int), ("filter_launches", ctypes.c_int),
                ("n_lowprec_iters", ctypes.c_int), ("t_filter_lowprec", ctypes.c_double),
                ("filter_flops_lowprec", ctypes.c_double), ("t_rr_eig", ctypes.c_double),
                ("jacobi_sweeps", ctypes.c_int), ("t_filter_product", ctypes.c_double),
                ("t_graph_build", ctypes.c_double), ("graph_launches", ctypes.c_int),
                ("autotune_trials", ctypes.c_int)]


class IterLog(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int), ("locked_before", ctypes.c_int),
                ("locked_after", ctypes.c_int), ("variant", ctypes.c_int),
                ("chol_fail_info", ctypes.c_int), ("deg_min", ctypes.c_int), ("deg_max", ctypes.c_int),
                ("matvecs", ctypes.c_longlong), ("log_cond_est", ctypes.c_double),
                ("c", ctypes.c_double), ("e", ctypes.c_double), ("mu1", ctypes.c_double),
                ("mu_ell", ctypes.c_double), ("log_cond_est_paper", ctypes.c_double),
                ("log_cond_est_locked", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("n", ctypes.c_int), ("dA", ctypes.c_void_p),
                ("lda", ctypes.c_int), ("nev", ctypes.c_int), ("nex", ctypes.c_int),
                ("bounds", ctypes.c_void_p), ("dV", ctypes.c_void_p), ("ldv", ctypes.c_int),
                ("evals", ctypes.c_void_p), ("resid", ctypes.c_void_p), ("stats", ctypes.c_void_p)]


_lib = None


def build(verbose=False):
    """Compile the CUDA library for sm_103a (see _buildlib.py)."""
    from . import _buildlib
    return _buildlib.build(verbose=verbose)


def lib():
    """Load ``libchase_gb300.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libchase_gb300.so is not built: run paper_2603_10514_gb300.build() "
                               "(nvcc, sm_103a) first; there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        P, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.chase_create.argtypes = [ctypes.POINTER(P), i, P]
        L.chase_destroy.argtypes = [P]
        L.chase_config_default.argtypes = [ctypes.POINTER(Config)]
        L.chase_workspace_bytes.argtypes = [i, i, i, i, i, ctypes.POINTER(ctypes.c_size_t)]
        L.chase_reserve_workspace.argtypes = [P, ctypes.c_size_t]
        L.chase_lanczos_bounds.argtypes = [P, i, i, P, i, i, P, i, i, i, ctypes.POINTER(Bounds)]
        L.chase_solve.argtypes = [P, i, i, P, i, i, i, ctypes.POINTER(Config), ctypes.POINTER(Bounds),
                                  P, i, P, P, ctypes.POINTER(Stats), P, i]
        L.chase_filter.argtypes = [P, i, i, P, i, i, P, i, P, d, d, d, i, P, i]
        L.chase_qr.argtypes = [P, i, i, i, P, i, d, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.chase_qr_prec.argtypes = [P, i, i, i, P, i, d, i, i, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.chase_cond_est.argtypes = [i, i, P, P, d, d, d, d, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.chase_filter_noalloc.argtypes = [i, i, P, i, i, P, i, P, d, d, d, P, i, P]
        L.chase_selftest_wait_timeout.argtypes = [P, d]
        L.chase_batch_create.argtypes = [ctypes.POINTER(P), P]
        L.chase_batch_destroy.argtypes = [P]
        L.chase_batch_pending.argtypes = [P]
        L.chase_batch_add.argtypes = [P, i, i, P, i, i, i, ctypes.POINTER(Config), ctypes.POINTER(Bounds),
                                      P, i, P, P, ctypes.POINTER(Stats), P, i, ctypes.POINTER(i)]
        L.chase_batch_step.argtypes = [P, P, P, i, ctypes.POINTER(i)]
        L.chase_solve_batch.argtypes = [P, i, P, ctypes.POINTER(Config), P]
        L.chase_autotune_table.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.chase_autotune_clear.argtypes = []
        L.chase_status_string.argtypes = [i]
        L.chase_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def status_string(code):
    try:
        return lib().chase_status_string(int(code)).decode()
    except Exception:  # library missing: still format the error
        return "status %d" % code


def config_default(**kw):
    cfg = Config()
    rc = lib().chase_config_default(ctypes.byref(cfg))
    if rc:
        raise ChaseError(rc, "chase_config_default")
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return CHASE_R64
    if t.dtype == torch.complex128:
        return CHASE_C128
    raise TypeError("tensor dtype must be float64 or complex128, got %s" % t.dtype)


def _ld(t, name):
    """Leading dimension of a column-major 2-D CUDA tensor."""
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dim() == 2 and t.numel() == 0:
        return max(1, t.shape[0])
    if t.dim() == 2 and t.shape[1] == 1 and (t.stride(0) == 1 or t.shape[0] == 1):
        return max(1, t.shape[0])   # one column: the column stride is never used
    if t.dim() == 2 and t.shape[0] == 1 and t.stride(1) >= 1:
        return t.stride(1)          # one row: the row stride is never used
    if t.dim() != 2 or t.stride(0) != 1 or t.stride(1) < max(1, t.shape[0]):
        raise ValueError("%s must be column-major (strides (1, ld)), got strides %s" % (name, t.stride()))
    return t.stride(1)


def colmajor(t):
    """A column-major copy (strides (1, rows)) of a 2-D tensor."""
    return t.mT.contiguous().mT


class Handle:
    """Owns a chase_handle: a device, a CUDA stream and the device workspace."""

    def __init__(self, device=0, stream=None):
        """stream: a cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream) or
        None for a stream of the handle's own.  0, CUDA's legacy default stream (torch's default
        stream), is passed as cudaStreamLegacy: the C ABI reads NULL as "make a new stream"."""
        self._h = ctypes.c_void_p()
        if stream is not None and int(stream) == 0:
            stream = CUDA_STREAM_LEGACY
        s = ctypes.c_void_p(stream) if stream is not None else None
        rc = lib().chase_create(ctypes.byref(self._h), int(device), s)
        if rc:
            raise ChaseError(rc, "chase_create")
        self.device = device

    def close(self):
        if self._h:
            lib().chase_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self._h

    def reserve(self, nbytes):
        """Grow the workspace to nbytes now (no allocation later for problems that fit)."""
        rc = lib().chase_reserve_workspace(self._h, int(nbytes))
        if rc:
            raise ChaseError(rc, "chase_reserve_workspace")


def with_filtered_hook(cfg, fn):
    """Attach fn(dX_ptr, n, ell, ldx, iteration) -- called after each filter with the device
    block [Y V] about to be factored -- to cfg.  Keep the returned object alive while the
    solve runs."""
    cb = FILTERED_HOOK(lambda ctx, ptr, n, l, ld, it: fn(ptr, n, l, ld, it))
    cfg.filtered_hook = ctypes.cast(cb, ctypes.c_void_p)
    cfg.filtered_hook_ctx = None
    return cb


def chase_solve(h, A, V, nev, nex, bounds, cfg=None, log_cap=64, check=True):
    """Algorithm 1.  A: (n, n) column-major CUDA tensor; V: (n, nev+nex) column-major CUDA
    tensor holding V0 on entry and the final block (eigenvectors first) on exit.
    bounds = (lambda1, lambda_ell, b_sup).  Returns (status, evals, resid, stats dict, logs)."""
    n = A.shape[0]
    dt = _dtype_code(A)
    if _dtype_code(V) != dt:
        raise TypeError("A and V must have the same dtype")
    lda, ldv = _ld(A, "A"), _ld(V, "V")
    if cfg is None:
        cfg = config_default()
    b = Bounds(*[float(x) for x in bounds]) if bounds is not None else None
    evals = np.zeros(nev)
    resid = np.zeros(nev)
    st = Stats()
    logs = (IterLog * max(1, log_cap))()
    rc = lib().chase_solve(h.ptr, dt, n, ctypes.c_void_p(A.data_ptr()), lda, nev, nex, ctypes.byref(cfg),
                           ctypes.byref(b) if b is not None else None, ctypes.c_void_p(V.data_ptr()), ldv,
                           evals.ctypes.data_as(ctypes.c_void_p), resid.ctypes.data_as(ctypes.c_void_p),
                           ctypes.byref(st), ctypes.cast(logs, ctypes.c_void_p), log_cap)
    if check and rc not in (CHASE_OK, CHASE_NOT_CONVERGED):
        raise ChaseError(rc, "chase_solve")
    stats = {f: getattr(st, f) for f, _ in Stats._fields_}
    lg = [{f: getattr(logs[j], f) for f, _ in IterLog._fields_} for j in range(min(st.iterations, log_cap))]
    return rc, evals, resid, stats, lg


def chase_filter(h, A, V, degrees, c, e, lambda1, out=None, prec=CHASE_FP64):
    """Algorithm 4 with per-column degrees; returns the filtered block (new tensor unless out)."""
    import torch
    n, ncols = V.shape
    dt = _dtype_code(A)
    lda, ldv = _ld(A, "A"), _ld(V, "V")
    if out is None:
        out = colmajor(torch.empty_like(V))
    ldo = _ld(out, "out")
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    rc = lib().chase_filter(h.ptr, dt, n, ctypes.c_void_p(A.data_ptr()), lda, ncols,
                            ctypes.c_void_p(V.data_ptr()), ldv, deg.ctypes.data_as(ctypes.c_void_p),
                            float(c), float(e), float(lambda1), int(prec),
                            ctypes.c_void_p(out.data_ptr()), ldo)
    if rc:
        raise ChaseError(rc, "chase_filter")
    return out


def chase_qr(h, X, est_cond, qr_force=0, check=True, prec=None):
    """Algorithm 3 in place on the CUDA tensor X.  Returns (status, variant, chol_info).
    prec=None calls chase_qr (FP64 products); otherwise chase_qr_prec."""
    n, l = X.shape
    dt = _dtype_code(X)
    ldx = _ld(X, "X")
    v, info = ctypes.c_int(0), ctypes.c_int(0)
    if prec is None:
        rc = lib().chase_qr(h.ptr, dt, n, l, ctypes.c_void_p(X.data_ptr()), ldx, float(est_cond),
                            int(qr_force), ctypes.byref(v), ctypes.byref(info))
    else:
        rc = lib().chase_qr_prec(h.ptr, dt, n, l, ctypes.c_void_p(X.data_ptr()), ldx,
                                 float(est_cond), int(qr_force), int(prec), ctypes.byref(v),
                                 ctypes.byref(info))
    if check and rc not in (CHASE_OK, CHASE_CHOL_FAILED):
        raise ChaseError(rc, "chase_qr")
    return rc, v.value, info.value


def chase_selftest_wait_timeout(h, seconds=0.01):
    """Runs a device wait that nothing completes; returns the status the library reports
    (CHASE_ERR_TIMEOUT when the bounded wait ran out and was reported, as designed)."""
    return lib().chase_selftest_wait_timeout(h.ptr, float(seconds))


def chase_lanczos_bounds(h, A, V0, steps, ell):
    """(lambda1, lambda_ell, b_sup) from Lanczos runs started at the columns of V0 (CUDA)."""
    n = A.shape[0]
    dt = _dtype_code(A)
    lda, ldv = _ld(A, "A"), _ld(V0, "V0")
    out = Bounds()
    rc = lib().chase_lanczos_bounds(h.ptr, dt, n, ctypes.c_void_p(A.data_ptr()), lda, V0.shape[1],
                                    ctypes.c_void_p(V0.data_ptr()), ldv, int(steps), int(ell),
                                    ctypes.byref(out))
    if rc:
        raise ChaseError(rc, "chase_lanczos_bounds")
    return out.lambda1, out.lambda_ell, out.b_sup


def chase_cond_est(ritz, degrees, nlocked, lambda1, c, e, eta=1.0):
    """Eq. full-est.  Returns (est, log_est)."""
    r = np.ascontiguousarray(ritz, dtype=np.float64)
    d = np.ascontiguousarray(degrees, dtype=np.int32)
    est, lest = ctypes.c_double(), ctypes.c_double()
    rc = lib().chase_cond_est(len(r), int(nlocked), r.ctypes.data_as(ctypes.c_void_p),
                              d.ctypes.data_as(ctypes.c_void_p), float(lambda1), float(c), float(e),
                              float(eta), ctypes.byref(est), ctypes.byref(lest))
    if rc:
        raise ChaseError(rc, "chase_cond_est")
    return est.value, lest.value


def chase_filter_noalloc(A, V, degrees, c, e, lambda1, out=None, stream=None):
    """The filter of chase_filter for callers that cannot allocate device memory (inside
    a CUDA graph capture, under a pre-reserved memory pool, or in latency-critical loops
    where cudaMalloc would synchronise the device).  Its scratch is a fixed 32 MiB device
    array inside the library; `out` (if given) and V are the caller's buffers.  Work is
    ordered on `stream` (default: torch's current stream of V's device).  Raises
    ChaseError(CHASE_ERR_TOO_LARGE) when n * ncols elements exceed the fixed scratch."""
    import torch
    n, ncols = V.shape
    dt = _dtype_code(A)
    lda, ldv = _ld(A, "A"), _ld(V, "V")
    if out is None:
        out = colmajor(torch.empty_like(V))
    ldo = _ld(out, "out")
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    if stream is None:
        stream = torch.cuda.current_stream(V.device).cuda_stream
    with torch.cuda.device(V.device):
        rc = lib().chase_filter_noalloc(dt, n, ctypes.c_void_p(A.data_ptr()), lda, ncols,
                                        ctypes.c_void_p(V.data_ptr()), ldv,
                                        deg.ctypes.data_as(ctypes.c_void_p), float(c), float(e),
                                        float(lambda1), ctypes.c_void_p(out.data_ptr()), ldo,
                                        ctypes.c_void_p(stream))
    if rc:
        raise ChaseError(rc, "chase_filter_noalloc")
    return out


class BatchProblem:
    """One problem of a batch session: the inputs (kept alive while in flight) and, once the
    session reports it finished, its results (status, evals, resid, stats)."""

    def __init__(self, A, V, nev, nex, bounds, cfg=None, log_cap=0):
        self.A, self.V, self.nev, self.nex = A, V, nev, nex
        self.bounds = Bounds(*[float(x) for x in bounds]) if bounds is not None else None
        self.cfg = cfg if cfg is not None else config_default()
        self.evals = np.zeros(nev)
        self.resid = np.zeros(nev)
        self._stats = Stats()
        self.logs = (IterLog * max(1, log_cap))()
        self.log_cap = log_cap
        self.status = None
        self.id = -1

    @property
    def stats(self):
        return {f: getattr(self._stats, f) for f, _ in Stats._fields_}


class Batch:
    """A batch session (chase_batch_*): problems in flight advance one outer iteration per
    step(), their emulated-FP64 filter steps sharing launches.  add() may be called between
    steps.  step() returns the BatchProblems that ended in that step."""

    def __init__(self, handle):
        self.handle = handle
        self._b = ctypes.c_void_p()
        rc = lib().chase_batch_create(ctypes.byref(self._b), handle.ptr)
        if rc:
            raise ChaseError(rc, "chase_batch_create")
        self._live = {}

    def add(self, prob):
        A, V = prob.A, prob.V
        dt = _dtype_code(A)
        if _dtype_code(V) != dt:
            raise TypeError("A and V must have the same dtype")
        n = A.shape[0]
        lda, ldv = _ld(A, "A"), _ld(V, "V")
        pid = ctypes.c_int(-1)
        rc = lib().chase_batch_add(self._b, dt, n, ctypes.c_void_p(A.data_ptr()), lda, prob.nev, prob.nex,
                                   ctypes.byref(prob.cfg),
                                   ctypes.byref(prob.bounds) if prob.bounds is not None else None,
                                   ctypes.c_void_p(V.data_ptr()), ldv,
                                   prob.evals.ctypes.data_as(ctypes.c_void_p),
                                   prob.resid.ctypes.data_as(ctypes.c_void_p), ctypes.byref(prob._stats),
                                   ctypes.cast(prob.logs, ctypes.c_void_p), prob.log_cap, ctypes.byref(pid))
        if rc:
            raise ChaseError(rc, "chase_batch_add")
        prob.id = pid.value
        self._live[prob.id] = prob
        return prob

    def pending(self):
        return lib().chase_batch_pending(self._b)

    def step(self):
        cap = max(1, len(self._live))
        ids = (ctypes.c_int * cap)()
        sts = (ctypes.c_int * cap)()
        nd = ctypes.c_int(0)
        rc = lib().chase_batch_step(self._b, ctypes.cast(ids, ctypes.c_void_p), ctypes.cast(sts, ctypes.c_void_p),
                                    cap, ctypes.byref(nd))
        if rc:
            raise ChaseError(rc, "chase_batch_step")
        out = []
        for j in range(nd.value):
            prob = self._live.pop(ids[j])
            prob.status = sts[j]
            out.append(prob)
        return out

    def close(self):
        if self._b:
            lib().chase_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chase_solve_batch(h, problems, cfg=None):
    """Solves the BatchProblems together (chase_solve_batch); fills each one's status,
    evals, resid and stats."""
    cfg = cfg if cfg is not None else config_default()
    arr = (Problem * max(1, len(problems)))()
    keep = []
    for i, p in enumerate(problems):
        A, V = p.A, p.V
        dt = _dtype_code(A)
        b = ctypes.pointer(p.bounds) if p.bounds is not None else None
        keep.append(b)
        arr[i] = Problem(dt, A.shape[0], A.data_ptr(), _ld(A, "A"), p.nev, p.nex,
                         ctypes.cast(b, ctypes.c_void_p) if b is not None else None, V.data_ptr(),
                         _ld(V, "V"), p.evals.ctypes.data, p.resid.ctypes.data,
                         ctypes.addressof(p._stats))
    status = (ctypes.c_int * max(1, len(problems)))()
    rc = lib().chase_solve_batch(h.ptr, len(problems), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(cfg),
                                 ctypes.cast(status, ctypes.c_void_p))
    if rc:
        raise ChaseError(rc, "chase_solve_batch")
    for i, p in enumerate(problems):
        p.status = status[i]
    return [p.status for p in problems]


def autotune_table():
    """The autotuner's picks (chase_autotune_table) as a list of text lines."""
    need = ctypes.c_size_t(0)
    lib().chase_autotune_table(None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(max(1, need.value))
    lib().chase_autotune_table(buf, len(buf), None)
    return [ln for ln in buf.value.decode().splitlines() if ln]


def autotune_clear():
    lib().chase_autotune_clear()

"""Plain FP64 CPU oracle for Chebyshev-filtered subspace iteration (ChASE).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never calls it and shares no code with it.

The arithmetic lives in ``chase_oracle.c`` (plain C, FP64, one definition per
step of the paper: Algorithm 4 filter, Eq. simple-est / full-est estimate,
Algorithms 2 and 3 QR selection, Householder QR, cyclic Jacobi eigensolver for
the Rayleigh-Ritz step, one-sided Jacobi SVD for the exact kappa_2, and the
Algorithm 1 outer loop).  This module compiles it with gcc on first use and
marshals numpy arrays through ctypes.  Real problems are promoted to
complex128; the C code maps real data to real data.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chase_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, -O2, OpenMP) if missing or stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(os.path.join(_HERE, "chase_oracle.h")))):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("deg_init", ctypes.c_int),
                ("deg_min", ctypes.c_int), ("deg_max", ctypes.c_int), ("opt_degree", ctypes.c_int),
                ("eta", ctypes.c_double), ("cond_hi", ctypes.c_double), ("cond_lo", ctypes.c_double),
                ("qr_force", ctypes.c_int), ("lambda1", ctypes.c_double),
                ("lambda_ell", ctypes.c_double), ("b_sup", ctypes.c_double),
                ("cond_est_mode", ctypes.c_int), ("log_exact_kappa", ctypes.c_int)]


class IterLog(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int), ("locked_before", ctypes.c_int),
                ("locked_after", ctypes.c_int), ("variant", ctypes.c_int),
                ("chol_fail_info", ctypes.c_int), ("deg_min", ctypes.c_int),
                ("deg_max", ctypes.c_int), ("matvecs", ctypes.c_longlong),
                ("log_cond_est", ctypes.c_double), ("c", ctypes.c_double), ("e", ctypes.c_double),
                ("mu1", ctypes.c_double), ("mu_ell", ctypes.c_double),
                ("log_cond_est_paper", ctypes.c_double), ("log_cond_est_locked", ctypes.c_double),
                ("log_kappa_exact", ctypes.c_double)]


class Summary(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("locked", ctypes.c_int), ("n_chol1", ctypes.c_int),
                ("n_chol2", ctypes.c_int), ("n_shifted", ctypes.c_int), ("n_hhqr", ctypes.c_int),
                ("matvecs", ctypes.c_longlong)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i, d = ctypes.c_int, ctypes.c_double
            _lib.orc_filter.argtypes = [i, P, i, i, P, i, P, d, d, d]
            _lib.orc_abs_rho.argtypes = [d, d, d]
            _lib.orc_abs_rho.restype = d
            _lib.orc_log_cond_est.argtypes = [d, i, i, d, d, d, d]
            _lib.orc_log_cond_est.restype = d
            _lib.orc_cholesky_upper.argtypes = [i, P, i]
            _lib.orc_right_solve_upper.argtypes = [i, i, P, i, P, i]
            _lib.orc_cholqr.argtypes = [i, i, P, i, i]
            _lib.orc_shifted_chol_step.argtypes = [i, i, P, i]
            _lib.orc_householder_qr.argtypes = [i, i, P, i]
            _lib.orc_qr_dynamic.argtypes = [i, i, P, i, d, d, d, i, P]
            _lib.orc_jacobi_eig.argtypes = [i, P, i, P, P, i]
            _lib.orc_jacobi_svd.argtypes = [i, i, P, i, P]
            _lib.orc_lanczos_bounds.argtypes = [i, P, i, i, P, i, i, i, P, P]
            _lib.orc_solve.argtypes = [i, P, i, i, i, P, i, ctypes.POINTER(Params), P, P, P,
                                       ctypes.POINTER(Summary)]
        return _lib


def _c128(x):
    """Column-major complex128 COPY (Fortran order): the C routines work in place,
    so the caller's array is never aliased."""
    return np.array(x, dtype=np.complex128, order="F", copy=True)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _out(a, like_real):
    return a.real.copy() if like_real else a


def filter(A, V, degrees, c, e, lambda1):
    """p_{m_a}(A) v_a for every column (Algorithm 4 with per-column degrees)."""
    real = not np.iscomplexobj(A) and not np.iscomplexobj(V)
    A_, V_ = _c128(A), _c128(V)
    n, nc = V_.shape
    deg = np.ascontiguousarray(degrees, dtype=np.int32)
    rc = lib().orc_filter(n, _ptr(A_), n, nc, _ptr(V_), n, _ptr(deg), c, e, lambda1)
    if rc != 0:
        raise ValueError("orc_filter returned %d" % rc)
    return _out(V_, real)


def abs_rho(x, c, e):
    return lib().orc_abs_rho(x, c, e)


def log_cond_est(theta_k1, m_k1, m_ell, lambda1, c, e, eta=1.0):
    return lib().orc_log_cond_est(theta_k1, m_k1, m_ell, lambda1, c, e, eta)


def gram(X):
    """X^H X, Hermitised (the first step of Algorithm 2)."""
    X_ = np.asarray(X)
    G = X_.conj().T @ X_
    return 0.5 * (G + G.conj().T)


def cholesky_upper(G):
    """Returns (R, info) with G = R^H R."""
    real = not np.iscomplexobj(G)
    G_ = _c128(G)
    info = lib().orc_cholesky_upper(G_.shape[0], _ptr(G_), G_.shape[0])
    return _out(G_, real), info


def right_solve_upper(X, R):
    real = not np.iscomplexobj(X) and not np.iscomplexobj(R)
    X_, R_ = _c128(X), _c128(R)
    lib().orc_right_solve_upper(X_.shape[0], X_.shape[1], _ptr(X_), X_.shape[0], _ptr(R_), R_.shape[0])
    return _out(X_, real)


def cholqr(X, passes):
    real = not np.iscomplexobj(X)
    X_ = _c128(X)
    info = lib().orc_cholqr(X_.shape[0], X_.shape[1], _ptr(X_), X_.shape[0], passes)
    return _out(X_, real), info


def shifted_chol_step(X):
    real = not np.iscomplexobj(X)
    X_ = _c128(X)
    info = lib().orc_shifted_chol_step(X_.shape[0], X_.shape[1], _ptr(X_), X_.shape[0])
    return _out(X_, real), info


def householder_qr(X):
    real = not np.iscomplexobj(X)
    X_ = _c128(X)
    lib().orc_householder_qr(X_.shape[0], X_.shape[1], _ptr(X_), X_.shape[0])
    return _out(X_, real)


VARIANTS = {1: "cholqr1", 2: "cholqr2", 3: "shifted_cholqr2", 4: "householder"}


def qr_dynamic(X, log_est, cond_hi=1e8, cond_lo=20.0, force=0):
    """Algorithm 3.  Returns (Q, variant, first_failing_cholesky_info)."""
    real = not np.iscomplexobj(X)
    X_ = _c128(X)
    info = ctypes.c_int(0)
    v = lib().orc_qr_dynamic(X_.shape[0], X_.shape[1], _ptr(X_), X_.shape[0], log_est, cond_hi,
                             cond_lo, force, ctypes.byref(info))
    return _out(X_, real), v, info.value


def jacobi_eig(H):
    """Cyclic Jacobi: (w ascending, W, sweeps)."""
    real = not np.iscomplexobj(H)
    H_ = _c128(H)
    l = H_.shape[0]
    w = np.zeros(l)
    W = np.zeros((l, l), dtype=np.complex128, order="F")
    sweeps = lib().orc_jacobi_eig(l, _ptr(H_), l, _ptr(w), _ptr(W), l)
    return w, _out(W, real), sweeps


def jacobi_svd(X):
    """Singular values (descending) by one-sided Jacobi."""
    X_ = _c128(X)
    sv = np.zeros(X_.shape[1])
    lib().orc_jacobi_svd(X_.shape[0], X_.shape[1], _ptr(X_), X_.shape[0], _ptr(sv))
    return sv


def lanczos_bounds(A, V0, steps, ell):
    """(lambda1, lambda_ell, b_sup) estimates from Lanczos runs started at the columns of V0,
    plus every run's Ritz values (nruns x steps)."""
    A_, V_ = _c128(A), _c128(V0)
    n, r = V_.shape
    out = np.zeros(3)
    ritz = np.zeros((r, steps))
    lib().orc_lanczos_bounds(n, _ptr(A_), n, r, _ptr(V_), n, steps, ell, _ptr(out), _ptr(ritz))
    return tuple(out), ritz


def solve(A, V0, nev, nex, *, tol=1e-10, max_iter=25, deg_init=20, deg_min=10, deg_max=36,
          opt_degree=False, eta=1.0, cond_hi=1e8, cond_lo=20.0, qr_force=0, lambda1, lambda_ell,
          b_sup, cond_est_mode=0, log_exact_kappa=False):
    """Algorithm 1.  Returns a dict with evals, resid, Y (n x nev), V (final block),
    per-iteration logs and the summary counters."""
    real = not np.iscomplexobj(A) and not np.iscomplexobj(V0)
    A_, V_ = _c128(A), _c128(V0)
    n = A_.shape[0]
    l = nev + nex
    assert V_.shape == (n, l)
    prm = Params(tol, max_iter, deg_init, deg_min, deg_max, int(opt_degree), eta, cond_hi, cond_lo,
                 qr_force, lambda1, lambda_ell, b_sup, cond_est_mode, int(log_exact_kappa))
    evals = np.zeros(nev)
    resid = np.zeros(nev)
    logs = (IterLog * max(max_iter, 1))()
    summ = Summary()
    status = lib().orc_solve(n, _ptr(A_), n, nev, nex, _ptr(V_), n, ctypes.byref(prm), _ptr(evals),
                             _ptr(resid), ctypes.cast(logs, ctypes.c_void_p), ctypes.byref(summ))
    it = summ.iterations
    log = [{f: getattr(logs[j], f) for f, _ in IterLog._fields_} for j in range(it)]
    V_out = _out(V_, real)
    return {"status": status, "evals": evals, "resid": resid, "Y": V_out[:, :nev].copy(),
            "V": V_out, "logs": log,
            "summary": {f: getattr(summ, f) for f, _ in Summary._fields_}}

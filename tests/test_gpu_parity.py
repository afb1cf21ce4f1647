"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element on the same seeded inputs.

Tolerances (FP64, derived from the arithmetic):
  * filter: per-column normwise relative difference <= 1e-11, and every entry
    within 1e-11 of its column's largest entry (up to sqrt(n) stricter per
    entry).  Each step is a length-n dot product (error <= n u |A||v|) followed
    by the three-term combination; summation order differs between the two
    implementations, so the columns agree to ~m sqrt(n) u times the growth of the
    recurrence relative to the result, which stays far below 1e-11 for the
    degrees used.  (A rigorous entrywise running-error bound through |A|^m is
    orders of magnitude looser after a few dozen steps, so it would test
    nothing.)
  * QR (Cholesky variants, kappa <= 1e4): Q is the unique factor with positive
    diagonal R; elementwise |dQ| <= 1e-9 (kappa^2 u-level for CholQR2).
  * eigenvalues: |lambda_gpu - lambda_oracle| <= 1e-10 ||A|| (the target the
    method states), residuals <= tol, ||Y^H Y - I||_F <= 1e-12.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_10514_gb300 as P
    P.build()
    return P


@pytest.fixture(scope="module")
def handle(cl):
    h = cl.Handle(0)
    yield h
    h.close()


def dev(x):
    """numpy (n, m) -> column-major CUDA tensor."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda()
    return t.mT


def host(t):
    return t.cpu().numpy()


def random_unitary(n, seed, complex_):
    G = W.gaussian((n, n), seed, complex_)
    Q, R = np.linalg.qr(G)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def sv_matrix(n, l, sv, seed, complex_):
    U = random_unitary(n, seed, complex_)[:, :l]
    Wq = random_unitary(l, seed + 1, complex_)
    return (U * sv) @ Wq.conj().T


# --------------------------------------------------------------------------
# Filter (Algorithm 4)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,degs", [
    (333, [0, 1, 2, 2, 5, 8, 8, 8, 13, 20, 20, 27, 36]),          # ragged n, mixed degrees
    (1000, [20] * 30),                                             # small real workload shape
    (517, list(range(10, 47))),                                    # > 32 columns, every degree
])
def test_filter_matches_oracle(cl, handle, complex_, n, degs):
    lam = W.spectrum_uniform(n, -1.0, 1.0, 5)
    A = W.known_spectrum_matrix(lam, 5, complex_).numpy()
    V = W.start_block(n, len(degs), 6, complex_)
    lambda1, mu_ell, bsup = lam[0], lam[len(degs) - 1], lam[-1] + 1e-3
    c, e = 0.5 * (bsup + mu_ell), 0.5 * (bsup - mu_ell)
    ref = oracle.filter(A, V, degs, c, e, lambda1)
    out = cl.chase_filter(handle, dev(A), dev(V), degs, c, e, lambda1)
    got = host(out)
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-11, err.max()
    assert entrywise_err(got, ref) <= 1e-11


def entrywise_err(got, ref):
    """max over entries of |got - ref| / (largest |entry| of the column of ref); an
    all-zero column (degree 0 of a zero vector) must match exactly."""
    scale = np.abs(ref).max(axis=0)
    d = np.abs(got - ref)
    if np.any(scale == 0):
        assert np.all(d[:, scale == 0] == 0)
    return float((d[:, scale > 0] / scale[scale > 0]).max()) if np.any(scale > 0) else 0.0


def test_filter_in_place_and_empty(cl, handle):
    n = 64
    A = W.known_spectrum_matrix(W.spectrum_uniform(n, -1, 1, 2), 2, False)
    A = A.cuda()
    V = dev(W.start_block(n, 4, 3, False))
    ref = oracle.filter(host(A), host(V), [3, 3, 4, 7], 0.5, 0.6, -1.2)
    cl.chase_filter(handle, A, V, [3, 3, 4, 7], 0.5, 0.6, -1.2, out=V)
    assert np.abs(host(V) - ref).max() <= 1e-12 * np.abs(ref).max()
    # zero columns: nothing to do
    Z = dev(np.zeros((n, 0)))
    cl.chase_filter(handle, A, Z, [], 0.5, 0.6, -1.2, out=Z)


def test_filter_rejects_bad_arguments(cl, handle):
    n = 16
    A = dev(np.eye(n))
    V = dev(np.ones((n, 2)))
    with pytest.raises(cl.ChaseError):
        cl.chase_filter(handle, A, V, [3, 2], 0.5, 0.6, -1.2)  # descending degrees
    with pytest.raises(cl.ChaseError):
        cl.chase_filter(handle, A, V, [2, 3], 0.5, -0.6, -1.2)  # e <= 0
    with pytest.raises(cl.ChaseError):
        cl.chase_filter(handle, A, V, [2, 3], 0.5, 0.6, 0.3)  # lambda1 inside the interval


def test_filter_rejects_outputs_that_overlap_its_inputs(cl, handle):
    """The filter reads its input block and A while it writes the output: an output that is
    the input shifted by a column, or that lies inside A, is rejected (-14) before any device
    work; the input block itself (same leading dimension) is the in-place filter."""
    n = 32
    A = dev(np.eye(n) * 0.1)
    buf = dev(np.arange(n * 5, dtype=np.float64).reshape(5, n).T)  # n x 5
    before = host(buf)
    for out, V in ((buf[:, 1:4], buf[:, 0:3]), (A[:, 2:5], buf[:, 0:3])):
        with pytest.raises(cl.ChaseError) as ex:
            cl.chase_filter(handle, A, V, [1, 2, 3], 0.5, 0.6, -1.2, out=out)
        assert ex.value.code == -14
    np.testing.assert_array_equal(host(buf), before)
    assert np.abs(host(A) - 0.1 * np.eye(n)).max() == 0.0


# --------------------------------------------------------------------------
# QR (Algorithms 2 and 3)
# --------------------------------------------------------------------------

def _orth(Q):
    return np.linalg.norm(Q.conj().T @ Q - np.eye(Q.shape[1]))


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("force,log10k", [(1, 0), (2, 2), (2, 4), (3, 4), (3, 10), (4, 12)])
def test_qr_variant_matches_oracle(cl, handle, complex_, force, log10k):
    n, l = 421, 37
    X = sv_matrix(n, l, np.logspace(0, -log10k, l), 40 + log10k, complex_)
    Qo, vo, io = oracle.qr_dynamic(X, 0.0, force=force)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=force)
    Q = host(Xd)
    assert rc == 0 and v == force and io == 0 and info == 0
    assert _orth(Q) <= 1e-12 if force != 1 else _orth(Q) <= 1e-10
    if force == 4:
        ph = np.sum(Qo.conj() * Q, axis=0)   # same columns up to unit phases
        np.testing.assert_allclose(np.abs(ph), 1.0, atol=1e-9)
    elif 10.0 ** log10k <= 1e4:
        assert np.abs(Q - Qo).max() <= 1e-9
    # X = Q R with R upper triangular
    R = Q.conj().T @ X
    assert np.linalg.norm(np.tril(R, -1)) <= 1e-10 * np.linalg.norm(X)


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,l", [
    (700, 96),     # panels of 32, three exactly
    (900, 100),    # panels of 32, ragged last panel (4 columns)
    (1300, 200),   # panels of 64, ragged last panel (8 columns)
    (2000, 333),   # panels of 64, several trailing updates per panel
])
def test_householder_blocked_matches_oracle(cl, handle, complex_, n, l):
    """The compact-WY Householder QR (forced fallback, l >= 96) against the oracle's
    Householder QR: the same reflectors, so the same columns up to unit phases; orthonormal
    to 1e-12 even at kappa 1e12; X = Q R with R upper triangular."""
    X = sv_matrix(n, l, np.logspace(0, -12, l), 900 + l, complex_)
    Qo, vo, io = oracle.qr_dynamic(X, 0.0, force=4)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=4)
    Q = host(Xd)
    assert rc == 0 and v == 4 and vo == 4 and info == 0
    assert _orth(Q) <= 1e-12
    ph = np.sum(Qo.conj() * Q, axis=0)
    np.testing.assert_allclose(np.abs(ph), 1.0, atol=1e-9)
    R = Q.conj().T @ X
    assert np.linalg.norm(np.tril(R, -1)) <= 1e-10 * np.linalg.norm(X)


@pytest.mark.parametrize("est,want", [(1.0, 1), (19.0, 1), (20.0, 2), (1e7, 2), (1e9, 3)])
def test_qr_auto_selection(cl, handle, est, want):
    X = sv_matrix(300, 16, np.logspace(0, -1, 16), 77, True)
    rc, v, info = cl.chase_qr(handle, dev(X), est)
    assert rc == 0 and v == want


def test_qr_escalates_and_forced_failure_reports(cl, handle):
    """kappa ~ 1e15: CholQR2 chosen by a (wrong) small estimate fails, escalates, and the
    result is still orthonormal; a forced CholQR2 reports CHASE_CHOL_FAILED, X unchanged."""
    X = sv_matrix(300, 20, np.logspace(0, -15, 20), 78, True)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 100.0)
    assert rc == 0 and v in (3, 4) and info != 0
    assert _orth(host(Xd)) <= 1e-11
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=2)
    assert rc == cl.CHASE_CHOL_FAILED and info > 0
    np.testing.assert_array_equal(host(Xd), X)


# --------------------------------------------------------------------------
# Whole solve (Algorithm 1)
# --------------------------------------------------------------------------

def _run_both(cl, handle, prob, **kw):
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, prob.complex_, device="cuda")
    A = host(A_t)
    V0 = W.start_block(prob.n, prob.ell, prob.seed, prob.complex_)
    l1, le, bs = prob.bounds
    cfg = cl.config_default(tol=prob.tol, deg_init=prob.deg_init, deg_min=prob.deg_min,
                            deg_max=prob.deg_max, opt_degree=int(prob.opt_degree), **kw)
    ref = oracle.solve(A, V0, prob.nev, prob.nex, tol=prob.tol, deg_init=prob.deg_init,
                       deg_min=prob.deg_min, deg_max=prob.deg_max, opt_degree=prob.opt_degree,
                       lambda1=l1, lambda_ell=le, b_sup=bs, qr_force=kw.get("qr_force", 0))
    Vd = dev(V0)
    rc, ev, res, stats, logs = cl.chase_solve(handle, A_t, Vd, prob.nev, prob.nex, (l1, le, bs), cfg)
    return A, ref, rc, ev, res, stats, logs, host(Vd)


@pytest.mark.parametrize("complex_", [False, True])
def test_solve_small_real_workload(cl, handle, complex_):
    """The small workload (n = 1000, nev 20, nex 10, degree 20, plain method), real and
    complex: eigenvalues vs oracle and known spectrum, residuals, orthogonality, and the
    oracle's decisions (iterations, QR variants)."""
    prob = W.c1_real_small()
    prob.complex_ = complex_
    A, ref, rc, ev, res, stats, logs, V = _run_both(cl, handle, prob)
    normA = np.abs(prob.lam).max()
    assert rc == 0 and ref["status"] == 0
    assert np.abs(ev - ref["evals"]).max() <= 1e-10 * normA
    assert np.abs(ev - prob.lam[:prob.nev]).max() <= 1e-10 * normA
    assert res.max() < prob.tol
    Y = V[:, :prob.nev]
    assert _orth(Y) <= 1e-12
    assert np.linalg.norm(A @ Y - Y * ev, axis=0).max() <= 2 * prob.tol
    assert abs(stats["iterations"] - ref["summary"]["iterations"]) <= 1
    assert [g["variant"] for g in logs][:2] == [g["variant"] for g in ref["logs"]][:2]
    assert stats["matvecs"] == sum(prob.deg_init * (prob.ell - g["locked_before"]) for g in logs)


def test_solve_clustered_complex_optimised_degrees(cl, handle):
    """Complex Hermitian, clustered lowest part, optimised degrees in [10, 36]."""
    prob = W.c2_complex_clustered(n=1200, nev=40, nex=12, seed=8)
    A, ref, rc, ev, res, stats, logs, V = _run_both(cl, handle, prob)
    normA = np.abs(prob.lam).max()
    assert rc == 0 and ref["status"] == 0
    assert np.abs(ev - ref["evals"]).max() <= 1e-10 * normA
    assert np.abs(ev - prob.lam[:prob.nev]).max() <= 1e-10 * normA
    assert res.max() < prob.tol
    assert _orth(V[:, :prob.nev]) <= 1e-12
    assert abs(stats["iterations"] - ref["summary"]["iterations"]) <= 1
    assert abs(stats["matvecs"] - ref["summary"]["matvecs"]) <= 0.05 * ref["summary"]["matvecs"]


def test_solve_householder_forced_matches_dynamic(cl, handle):
    """Table 3 behaviour on the GPU: forced Householder QR vs the kappa-driven choice."""
    prob = W.Problem("t", 700, 24, 8, True, 31, W.spectrum_uniform(700, -1, 1, 31), opt_degree=True)
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    out = {}
    for force in (0, 4):
        cfg = cl.config_default(opt_degree=1, qr_force=force)
        rc, ev, res, stats, logs = cl.chase_solve(handle, A_t, dev(V0), prob.nev, prob.nex,
                                                  prob.bounds, cfg)
        assert rc == 0
        out[force] = (ev, stats)
    assert abs(out[0][1]["iterations"] - out[4][1]["iterations"]) <= 1
    assert abs(out[0][1]["matvecs"] - out[4][1]["matvecs"]) <= 0.1 * out[4][1]["matvecs"]
    assert out[4][1]["n_hhqr"] == out[4][1]["iterations"]
    assert out[0][1]["n_hhqr"] == 0
    np.testing.assert_allclose(out[0][0], out[4][0], atol=1e-11)


def test_solve_tiny_and_ragged(cl, handle):
    """Tiny ragged problem (n = 37, ell = 7) against a dense eigendecomposition."""
    n, nev, nex = 37, 4, 3
    G = W.gaussian((n, n), 5, True)
    A = 0.5 * (G + G.conj().T)
    lam = np.linalg.eigvalsh(A)
    rc, ev, res, stats, logs = cl.chase_solve(handle, dev(A), dev(W.start_block(n, 7, 5, True)), nev,
                                              nex, (lam[0], lam[6], lam[-1] + 1e-3))
    assert rc == 0
    np.testing.assert_allclose(ev, lam[:nev], atol=1e-11)


def test_solve_rejects_nonfinite(cl, handle):
    n = 40
    A = np.eye(n)
    A[3, 5] = np.nan
    rc, *_ = cl.chase_solve(handle, dev(A), dev(np.ones((n, 4))), 2, 2, (-1.0, 0.0, 2.0), check=False)
    assert rc == cl.CHASE_ERR_NONFINITE


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("l,log10k", [(200, 3), (330, 6), (330, 12)])
def test_qr_blocked_cholesky_paths(cl, handle, complex_, l, log10k):
    """Blocks wider than 128 columns use the blocked Cholesky (64-wide diagonal blocks,
    ragged last block): CholQR2 / shifted CholQR2 results stay orthonormal and agree
    with the oracle where the factor is unique."""
    n = 1500
    X = sv_matrix(n, l, np.logspace(0, -log10k, l), 90 + l, complex_)
    force = 2 if log10k <= 6 else 3
    Qo, vo, io = oracle.qr_dynamic(X, 0.0, force=force)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=force)
    Q = host(Xd)
    assert rc == 0 and v == force and info == 0 and io == 0
    assert _orth(Q) <= 1e-12
    if log10k <= 6:
        assert np.abs(Q - Qo).max() <= 1e-8
    R = Q.conj().T @ X
    assert np.linalg.norm(np.tril(R, -1)) <= 1e-10 * np.linalg.norm(X)


@pytest.mark.parametrize("complex_", [False, True])
def test_lanczos_bounds_match_oracle(cl, handle, complex_):
    n, ell = 700, 40
    lam = W.spectrum_clustered(n, 60, 3) if complex_ else W.spectrum_uniform(n, -1, 1, 3)
    A_t = W.known_spectrum_matrix(lam, 3, complex_, device="cuda")
    V = W.start_block(n, 4, 77, complex_)
    ref, _ = oracle.lanczos_bounds(host(A_t), V, 25, ell)
    got = cl.chase_lanczos_bounds(handle, A_t, dev(V), 25, ell)
    scale = lam[-1] - lam[0]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-9 * scale)
    assert got[2] >= lam[-1] and got[0] >= lam[0] - 1e-12


def test_solve_without_bounds_runs_lanczos(cl, handle):
    """bounds = NULL: the solve estimates them by Lanczos from its start block and still
    reaches the known spectrum."""
    prob = W.c2_complex_clustered(n=900, nev=30, nex=10, seed=21)
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    V0 = dev(W.start_block(prob.n, prob.ell, prob.seed, True))
    rc, ev, res, st, _ = cl.chase_solve(handle, A_t, V0, prob.nev, prob.nex, None,
                                        cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU))
    assert rc == 0 and res.max() < prob.tol
    assert np.abs(ev - prob.lam[:prob.nev]).max() <= 1e-10 * np.abs(prob.lam).max()


def test_condition_estimate_logs_match_oracle_and_bound_exact_kappa(cl, handle):
    """Per iteration the solver's estimate (Eq. full-est) equals the oracle's and picks the
    same QR variant; against the exact kappa_2 of the block [Y V] that Algorithm 3 factors
    (read through the filtered-block hook): the printed estimate bounds it while no pair is
    locked, the locked-aware form (cond_est_mode 1) in every iteration."""
    import bench
    prob = W.c2_complex_clustered(n=700, nev=30, nex=10, seed=14)
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    l1, le, bs = prob.bounds
    kap = {}

    def hook(ptr, n, l, ld, it):
        X = bench.device_view(ptr, n, l, ld, True).cpu().numpy()
        sv = np.linalg.svd(X, compute_uv=False)
        kap[it] = math.log(sv[0] / sv[-1])

    cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU)
    keep = cl.with_filtered_hook(cfg, hook)
    rc, ev, res, st, logs = cl.chase_solve(handle, A_t, dev(V0), prob.nev, prob.nex, prob.bounds, cfg)
    del keep
    ref = oracle.solve(host(A_t), V0, prob.nev, prob.nex, opt_degree=True, lambda1=l1,
                       lambda_ell=le, b_sup=bs)
    assert rc == 0 and len(kap) == st["iterations"] == ref["summary"]["iterations"]
    locked_seen = False
    for g, r in zip(logs, ref["logs"]):
        assert g["variant"] == r["variant"]
        assert abs(g["log_cond_est_paper"] - r["log_cond_est_paper"]) <= 1e-6 * max(1.0, abs(r["log_cond_est_paper"]))
        assert g["log_cond_est"] == g["log_cond_est_paper"]          # default mode 0
        assert g["log_cond_est_locked"] >= kap[g["iteration"]] - 1e-6
        if g["locked_before"] == 0:
            assert g["log_cond_est_paper"] >= kap[g["iteration"]] - 1e-6
        else:
            locked_seen = True
    assert locked_seen

"""Pins for the CPU oracle (no GPU).

Each test ties one oracle function to something other than itself: a closed
form from the paper, a textbook/library routine, an invariant, or brute force
on tiny inputs.  Citations name the paper's sections, equations and algorithms.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _cheb_coeffs():
    rows = {}
    for line in open(os.path.join(GOLDEN, "chebyshev_coeffs.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        m, rest = line.split(":")
        rows[int(m)] = [int(x) for x in rest.split()]
    return rows


def cheb_closed_form(m, t):
    """C_m(t) from the cos / cosh definition (Section 2.2) in long double."""
    t = np.asarray(t, dtype=np.longdouble)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ti = t[~inside]
    out[~inside] = np.sign(ti) ** m * np.cosh(m * np.arccosh(np.abs(ti)))
    return out


def random_unitary(n, seed, complex_):
    G = W.gaussian((n, n), seed, complex_)
    Q, R = np.linalg.qr(G)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def matrix_with_singular_values(n, l, sv, seed, complex_):
    Uq = random_unitary(n, seed, complex_)[:, :l]
    Wq = random_unitary(l, seed + 1, complex_)
    return np.asfortranarray((Uq * sv) @ Wq.conj().T)


# --------------------------------------------------------------------------
# Chebyshev filter (Algorithm 4, Section 2.3)
# --------------------------------------------------------------------------

def test_golden_coefficients_match_definition():
    """The stored coefficients equal cos(m arccos t) / cosh(m arccosh t)."""
    t = np.linspace(-3, 3, 61)
    for m, co in _cheb_coeffs().items():
        poly = np.polynomial.polynomial.polyval(t, co)
        np.testing.assert_allclose(poly, cheb_closed_form(m, t).astype(float), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("complex_", [False, True])
def test_filter_matches_closed_form(complex_):
    """p_{m_a}(A) v_a = Q diag(C_m(t(lam)) / C_m(t(lambda1))) Q^H v_a for A = Q diag(lam) Q^H
    (Theorem th:approx, Section 2.3), per-column degrees ascending incl. m = 0 and m = 1."""
    n = 80
    lam = W.spectrum_uniform(n, -1.0, 1.0, 11)
    Q = random_unitary(n, 12, complex_)
    A = np.asfortranarray((Q * lam) @ Q.conj().T)
    A = 0.5 * (A + A.conj().T)
    degs = [0, 1, 2, 3, 5, 8, 8, 13, 20, 27]
    V = W.start_block(n, len(degs), 13, complex_)
    lambda1, mu_ell, bsup = lam[0] - 0.05, lam[9], lam[-1] + 0.01
    c, e = 0.5 * (bsup + mu_ell), 0.5 * (bsup - mu_ell)
    out = oracle.filter(A, V, degs, c, e, lambda1)
    t = (lam - c) / e
    t1 = (lambda1 - c) / e
    for a, m in enumerate(degs):
        gain = (cheb_closed_form(m, t) / cheb_closed_form(m, np.array([t1]))).astype(float)
        ref = Q @ (gain * (Q.conj().T @ V[:, a]))
        err = np.linalg.norm(out[:, a] - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err < 1e-12, (a, m, err)


def test_filter_golden_polynomials_on_diagonal():
    """On a diagonal matrix the filter output is exactly C_m(t)/C_m(t1) times the input,
    with C_m from the stored integer coefficients (Eq. recur)."""
    lam = np.array([-1.3, -0.9, -0.2, 0.0, 0.4, 0.95])
    A = np.diag(lam)
    V = np.eye(6)[:, :1].repeat(1, axis=1) * 0 + np.ones((6, 1))
    coeffs = _cheb_coeffs()
    c, e, lambda1 = 0.0, 1.0, -1.3
    for m in range(0, 9):
        out = oracle.filter(A, V, [m], c, e, lambda1)[:, 0]
        expect = np.polynomial.polynomial.polyval(lam, coeffs[m]) / np.polynomial.polynomial.polyval(lambda1, coeffs[m])
        np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-15)


def test_filter_degree_one_is_affine_map():
    """m = 1: V_1 = (sigma_1/e)(A - cI)V with sigma_1 = e/(lambda1 - c) (Algorithm 4)."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((7, 7)); A = A + A.T
    V = rng.standard_normal((7, 2))
    c, e, lambda1 = 0.7, 2.0, -3.0
    out = oracle.filter(A, V, [1, 1], c, e, lambda1)
    ref = (A - c * np.eye(7)) @ V / (lambda1 - c)
    np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-14)


def test_filter_preserves_lambda1_component():
    """p_m(lambda1) = 1: an eigenvector for the eigenvalue lambda1 passes unchanged."""
    n = 40
    lam = W.spectrum_uniform(n, -1.0, 1.0, 5)
    Q = random_unitary(n, 6, True)
    A = (Q * lam) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    c, e = 0.5 * (lam[-1] + 0.01 + lam[5]), 0.5 * (lam[-1] + 0.01 - lam[5])
    out = oracle.filter(A, Q[:, :1], [17], c, e, lam[0])
    np.testing.assert_allclose(out[:, 0], Q[:, 0], atol=1e-11)


def test_filter_rejects_descending_degrees():
    with pytest.raises(ValueError):
        oracle.filter(np.eye(3), np.ones((3, 2)), [3, 2], 0.0, 1.0, -2.0)


# --------------------------------------------------------------------------
# Convergence ratio and kappa_2 estimate (Definition conv_ratio, Eq. simple-est,
# Eq. full-est, Proposition th:2-2)
# --------------------------------------------------------------------------

def test_abs_rho_closed_form():
    """|rho| = |t| + sqrt(t^2-1) satisfies cosh(ln|rho|) = |t| (Eq. polyas) and is 1 inside."""
    c, e = 1.0, 2.0
    for x in [-5.0, -1.5, -1.0000001, 3.5, 10.0]:
        r = oracle.abs_rho(x, c, e)
        t = abs((x - c) / e)
        assert r > 1.0
        assert math.isclose(math.cosh(math.log(r)), t, rel_tol=1e-12)
    for x in [-1.0, 0.0, 1.0, 3.0]:
        assert oracle.abs_rho(x, c, e) == 1.0


def test_cond_est_reduces_to_simple_estimate():
    """k = 0 and one degree m: Eq. full-est equals eta |rho_1|^m (Eq. simple-est), and
    |rho_1|^m is 2 C_m(|t_1|) up to the |rho|^-m term (Eq. polyas)."""
    c, e, lam1 = 2.0, 1.0, -1.0
    for m in [1, 5, 20, 36]:
        lest = oracle.log_cond_est(lam1, m, m, lam1, c, e, 1.0)
        t1 = abs((lam1 - c) / e)
        cm = float(cheb_closed_form(m, np.array([t1]))[0])
        rho_m = math.exp(lest)
        assert math.isclose(rho_m + 1.0 / rho_m, 2.0 * cm, rel_tol=1e-12)
    # eta multiplies
    assert math.isclose(oracle.log_cond_est(lam1, 7, 7, lam1, c, e, 3.0)
                        - oracle.log_cond_est(lam1, 7, 7, lam1, c, e, 1.0), math.log(3.0), rel_tol=1e-12)


def test_cond_est_full_form_exponents():
    """Eq. full-est: log est = m_{k+1} ln|rho_{k+1}| + (m_ell - m_{k+1}) ln|rho_1|."""
    c, e = 3.0, 2.0
    lam1, theta = -2.0, -0.5
    r1 = oracle.abs_rho(lam1, c, e)
    rk = oracle.abs_rho(theta, c, e)
    lest = oracle.log_cond_est(theta, 12, 30, lam1, c, e, 1.0)
    assert math.isclose(lest, 12 * math.log(rk) + 18 * math.log(r1), rel_tol=1e-13)
    # a Ritz value inside the damped interval contributes |rho| = 1
    assert math.isclose(oracle.log_cond_est(2.0, 12, 30, lam1, c, e, 1.0), 18 * math.log(r1), rel_tol=1e-13)


@pytest.mark.parametrize("m", [6, 12, 20])
def test_cond_est_bounds_exact_kappa_no_locking(m):
    """Proposition th:2-2: kappa_2(p_m(A)V) <= eta |rho_1|^m with
    eta = (|rho_ell|^m + 1) / (|rho_ell|^m (|rho_ell|^m - 1)), for orthonormal V;
    exact kappa_2 from the oracle's one-sided Jacobi SVD."""
    n, l = 120, 10
    lam = W.spectrum_uniform(n, -1.0, 1.0, 21)
    Q = random_unitary(n, 22, False)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    V, _ = np.linalg.qr(W.start_block(n, l, 23, False))
    bsup = lam[-1] + 1e-3
    c, e = 0.5 * (bsup + lam[l - 1]), 0.5 * (bsup - lam[l - 1])
    Vf = oracle.filter(A, V, [m] * l, c, e, lam[0])
    sv = oracle.jacobi_svd(Vf)
    kappa = sv[0] / sv[-1]
    rl = oracle.abs_rho(lam[l - 1] - 1e-12, c, e) ** m
    rl = max(rl, 1.0 + 1e-12)
    eta = (rl + 1) / (rl * (rl - 1)) if rl > 1.0 + 1e-9 else np.inf
    est_eta1 = math.exp(oracle.log_cond_est(lam[0], m, m, lam[0], c, e, 1.0))
    assert kappa <= max(eta, 1.0) * est_eta1 * (1 + 1e-8)
    # with eta = 1 (the paper's practical choice) the estimate still bounds kappa here
    assert kappa <= est_eta1 * (1 + 1e-8)


def test_deflation_theorem_brute_force():
    """Theorem th:deflation on tiny [A B] with A^H B = 0, singular values from the oracle's
    Jacobi SVD: kappa(M) <= (s1(A) + s1(B)) / min(s_q(A), s_p(B))."""
    rng = np.random.default_rng(8)
    for trial in range(20):
        n, q, p = 9, 2 + trial % 3, 1 + trial % 4
        U0 = random_unitary(n, 100 + trial, True)
        a = U0[:, :q] @ (rng.standard_normal((q, q)) + 1j * rng.standard_normal((q, q)))
        b = U0[:, q:q + p] @ (rng.standard_normal((p, p)) * (10.0 ** rng.uniform(-3, 3)))
        M = np.hstack([a, b])
        sM, sA, sB = oracle.jacobi_svd(M), oracle.jacobi_svd(a), oracle.jacobi_svd(b)
        assert sM[0] / sM[-1] <= (sA[0] + sB[0]) / min(sA[-1], sB[-1]) * (1 + 1e-10)


# --------------------------------------------------------------------------
# Cholesky, triangular solve, CholeskyQR variants, Householder QR
# (Algorithms 2 and 3, Table 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
def test_cholesky_matches_library(complex_):
    X = W.gaussian((50, 12), 31, complex_)
    G = X.conj().T @ X
    R, info = oracle.cholesky_upper(G)
    assert info == 0
    L = np.linalg.cholesky(G)
    np.testing.assert_allclose(R, L.conj().T, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0)


def test_cholesky_reports_failing_pivot():
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    _, info = oracle.cholesky_upper(G)
    assert info == 3
    G = np.array([[1.0, 2.0], [2.0, 1.0]])  # indefinite: second pivot 1 - 4 < 0
    _, info = oracle.cholesky_upper(G)
    assert info == 2


@pytest.mark.parametrize("complex_", [False, True])
def test_right_solve_matches_library(complex_):
    X = W.gaussian((30, 8), 41, complex_)
    R = np.triu(W.gaussian((8, 8), 42, complex_)) + 4 * np.eye(8)
    out = oracle.right_solve_upper(X, R)
    np.testing.assert_allclose(out @ R, X, rtol=1e-12, atol=1e-12)


def _qr_unique(X):
    """Thin QR with positive real diagonal of R (unique for full column rank)."""
    Q, R = np.linalg.qr(X)
    d = np.diag(R)
    ph = d / np.abs(d)
    return Q * ph


def _orth_err(Q):
    return np.linalg.norm(Q.conj().T @ Q - np.eye(Q.shape[1]))


def _table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "qr_ranges.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            rows[k] = float(v)
    return rows


@pytest.mark.parametrize("complex_", [False, True])
def test_cholqr_equals_unique_qr_when_well_conditioned(complex_):
    """CholeskyQR2 produces the Q of the QR factorisation with positive diagonal."""
    X = matrix_with_singular_values(60, 10, np.logspace(0, 3, 10), 51, complex_)
    Q, info = oracle.cholqr(X, 2)
    assert info == 0
    np.testing.assert_allclose(Q, _qr_unique(X), atol=1e-12)


@pytest.mark.parametrize("complex_", [False, True])
def test_householder_qr_spans_and_is_orthonormal(complex_):
    Xbad = matrix_with_singular_values(60, 10, np.logspace(0, 15, 10), 52, complex_)
    assert _orth_err(oracle.householder_qr(Xbad)) < 1e-13  # any kappa (Table 1)
    X = matrix_with_singular_values(60, 10, np.logspace(0, 6, 10), 52, complex_)
    Q = oracle.householder_qr(X)
    assert _orth_err(Q) < 1e-13
    Qu = _qr_unique(X)
    # same columns up to a unit phase each (Householder chooses R_jj = -e^{i arg x_0} ||x||)
    ph = np.sum(Qu.conj() * Q, axis=0)
    np.testing.assert_allclose(np.abs(ph), 1.0, atol=1e-8)
    R = Q.conj().T @ X
    assert np.linalg.norm(np.tril(R, -1)) < 1e-12 * np.linalg.norm(X)


@pytest.mark.parametrize("log10k", [0, 1, 4, 7, 10, 13])
def test_qr_variants_follow_table1(log10k):
    """Success pattern of Table 1: CholQR2 keeps orthogonality up to kappa ~ u^-1/2,
    shifted CholQR2 up to ~u^-1, Householder for any kappa; CholQR1 loses
    orthogonality like kappa^2 u."""
    kappa = 10.0 ** log10k
    X = matrix_with_singular_values(200, 12, np.logspace(0, -log10k, 12), 60 + log10k, True)
    tb = _table1()
    # Householder: always orthonormal
    assert _orth_err(oracle.householder_qr(X)) < 1e-13
    q1, info1 = oracle.cholqr(X, 1)
    q2, info2 = oracle.cholqr(X, 2)
    if kappa ** 2 * U < 1e-3:  # kappa below u^-1/2 by a margin: CholQR2 must succeed
        assert info2 == 0 and _orth_err(q2) < 1e-13
        assert info1 == 0 and _orth_err(q1) < 50 * kappa ** 2 * U + 1e-13
    if kappa > 1e9:  # far beyond u^-1/2: CholQR1 fails or loses orthogonality completely
        assert info1 != 0 or _orth_err(q1) > 1e-3
    if kappa * U < 1e-2:  # within u^-1: shifted step then CholQR2 succeeds
        qs, infos = oracle.shifted_chol_step(X)
        assert infos == 0
        qs, infos2 = oracle.cholqr(qs, 2)
        assert infos2 == 0 and _orth_err(qs) < 1e-13
        # spans the same space: residual of projection
        P = qs @ (qs.conj().T @ X)
        assert np.linalg.norm(P - X) < 1e-12 * np.linalg.norm(X) * max(1.0, kappa * 1e-3)
    assert tb["cholqr2"] == 0.5 and tb["shifted_cholqr2"] == 1.0


def test_shift_uses_squared_frobenius_norm():
    """Reading of Algorithm 3's shift: s = 11 (m n + n(n+1)) u ||X||_F^2.  Scaling X by the
    exact power of two 2^20 scales the Gram matrix and a squared-norm shift by 2^40, so the
    shifted step returns a bitwise-identical Q; an unsquared norm would not."""
    X = matrix_with_singular_values(80, 6, np.logspace(0, -12, 6), 71, False)
    qa, ia = oracle.shifted_chol_step(X)
    qb, ib = oracle.shifted_chol_step(X * 2.0 ** 20)
    assert ia == 0 and ib == 0
    np.testing.assert_array_equal(qa, qb)
    # and the shift matters at this conditioning: without it CholQR1's Cholesky fails or
    # produces a visibly different Q
    q1, i1 = oracle.cholqr(X, 1)
    assert i1 != 0 or np.abs(q1 - qa).max() > 1e-12


def test_qr_dynamic_selects_by_thresholds():
    """Algorithm 3: est > 1e8 -> shifted CholQR2, est < 20 -> CholQR1, else CholQR2."""
    X = matrix_with_singular_values(100, 8, np.logspace(0, -2, 8), 81, True)
    for est, want in [(1e9, 3), (1e8 * 1.0001, 3), (19.9, 1), (20.0, 2), (1e8, 2), (1e3, 2)]:
        _, v, _ = oracle.qr_dynamic(X, math.log(est))
        assert v == want, (est, v, want)
    _, v, _ = oracle.qr_dynamic(X, 0.0, force=4)
    assert v == 4


def test_qr_dynamic_escalates_on_cholesky_failure():
    """A CholQR2 chosen for a block whose Gram matrix is singular in FP64 escalates
    (shifted, then Householder) and still returns an orthonormal basis."""
    X = matrix_with_singular_values(100, 8, np.logspace(0, -14, 8), 82, True)
    Q, v, info = oracle.qr_dynamic(X, math.log(100.0))
    assert v in (3, 4) and info != 0
    assert _orth_err(Q) < 1e-12
    # a forced CholQR2 reports the failure instead
    _, v, info = oracle.qr_dynamic(X, 0.0, force=2)
    assert v == 2 and info != 0


# --------------------------------------------------------------------------
# Jacobi eigensolver and SVD (Rayleigh-Ritz step of Algorithm 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("l", [1, 2, 7, 40])
def test_jacobi_eig_matches_library(complex_, l):
    H = W.gaussian((l, l), 90 + l, complex_)
    H = 0.5 * (H + H.conj().T)
    w, Wm, sweeps = oracle.jacobi_eig(H)
    assert sweeps >= 0
    np.testing.assert_allclose(w, np.linalg.eigvalsh(H), atol=1e-13 * max(1, np.abs(w).max()))
    assert np.linalg.norm(H @ Wm - Wm * w) < 1e-12 * np.linalg.norm(H)
    assert _orth_err(Wm) < 1e-13
    assert np.all(np.diff(w) >= 0)


def test_jacobi_eig_degenerate_and_diagonal():
    H = np.diag([3.0, -1.0, 3.0, 0.5])
    w, Wm, _ = oracle.jacobi_eig(H)
    np.testing.assert_array_equal(w, [-1.0, 0.5, 3.0, 3.0])
    H = np.ones((5, 5))  # rank one: eigenvalues 0,0,0,0,5
    w, Wm, _ = oracle.jacobi_eig(H)
    np.testing.assert_allclose(w, [0, 0, 0, 0, 5], atol=1e-14)


@pytest.mark.parametrize("complex_", [False, True])
def test_jacobi_svd_matches_library(complex_):
    X = matrix_with_singular_values(50, 9, np.logspace(2, -6, 9), 95, complex_)
    sv = oracle.jacobi_svd(X)
    np.testing.assert_allclose(sv, np.logspace(2, -6, 9), rtol=1e-9)


# --------------------------------------------------------------------------
# Whole solve (Algorithm 1)
# --------------------------------------------------------------------------

def _solve(prob, **kw):
    A = W.known_spectrum_matrix(prob.lam, prob.seed, prob.complex_).numpy()
    V0 = W.start_block(prob.n, prob.ell, prob.seed, prob.complex_)
    l1, le, bs = prob.bounds
    args = dict(tol=prob.tol, deg_init=prob.deg_init, deg_min=prob.deg_min, deg_max=prob.deg_max,
                opt_degree=prob.opt_degree, lambda1=l1, lambda_ell=le, b_sup=bs)
    args.update(kw)
    return A, oracle.solve(A, V0, prob.nev, prob.nex, **args)


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("opt", [False, True])
def test_solve_known_spectrum(complex_, opt):
    """Eigenvalues within 1e-10 ||A|| of the known spectrum, residuals < tol,
    orthonormal locked vectors, ||AY - Y Lambda|| small."""
    prob = W.Problem("t", 240, 12, 6, complex_, 7, W.spectrum_uniform(240, -1, 1, 7), opt_degree=opt)
    A, r = _solve(prob)
    assert r["status"] == 0
    normA = np.abs(prob.lam).max()
    assert np.abs(r["evals"] - prob.lam[:prob.nev]).max() <= 1e-10 * normA
    assert r["resid"].max() < prob.tol
    Y = r["Y"]
    assert _orth_err(Y) < 10 * prob.ell * U * 10
    assert np.linalg.norm(A @ Y - Y * r["evals"], axis=0).max() < 2 * prob.tol
    assert r["summary"]["matvecs"] == r["logs"][-1]["matvecs"]


def test_solve_tiny_matches_dense_eigendecomposition():
    """Brute force: tiny random Hermitian matrix (no structure), compare with eigvalsh."""
    n, nev, nex = 24, 4, 3
    G = W.gaussian((n, n), 123, True)
    A = np.asfortranarray(0.5 * (G + G.conj().T))
    lam = np.linalg.eigvalsh(A)
    V0 = W.start_block(n, nev + nex, 123, True)
    r = oracle.solve(A, V0, nev, nex, lambda1=lam[0], lambda_ell=lam[nev + nex - 1],
                     b_sup=lam[-1] + 1e-3, opt_degree=True)
    assert r["status"] == 0
    np.testing.assert_allclose(r["evals"], lam[:nev], atol=1e-11)


def test_solve_clustered_complex_small():
    """Clustered lowest part (the complex workload's structure at a small size)."""
    prob = W.c2_complex_clustered(n=300, nev=15, nex=5, seed=9)
    A, r = _solve(prob)
    assert r["status"] == 0
    assert np.abs(r["evals"] - prob.lam[:prob.nev]).max() <= 1e-10 * np.abs(prob.lam).max()
    assert r["resid"].max() < prob.tol


def test_householder_forced_matches_dynamic_behaviour():
    """Table 3 behaviour: forcing Householder QR in every iteration gives the same
    iteration count and MatVecs within a few percent as the kappa-driven choice."""
    prob = W.Problem("t", 260, 14, 6, True, 17, W.spectrum_uniform(260, -1, 1, 17), opt_degree=True)
    _, rd = _solve(prob)
    _, rh = _solve(prob, qr_force=4)
    assert rd["status"] == 0 and rh["status"] == 0
    assert abs(rd["summary"]["iterations"] - rh["summary"]["iterations"]) <= 1
    assert abs(rd["summary"]["matvecs"] - rh["summary"]["matvecs"]) <= 0.1 * rh["summary"]["matvecs"]
    assert rh["summary"]["n_hhqr"] == rh["summary"]["iterations"]
    np.testing.assert_allclose(rd["evals"], rh["evals"], atol=1e-11)


def test_fixed_degree_matvec_count():
    """No-opt: every unlocked column is filtered with the same degree; MatVecs =
    sum over iterations of degree x unlocked columns (Table 3 footnote)."""
    prob = W.c1_real_small(n=200, nev=8, nex=4, seed=19)
    _, r = _solve(prob)
    expect = 0
    for g in r["logs"]:
        expect += prob.deg_init * (prob.ell - g["locked_before"])
    assert r["summary"]["matvecs"] == expect


def test_estimate_bounds_exact_kappa_in_solve_first_iteration():
    """At the first iteration (no locking, single degree) the estimate of Eq. simple-est
    bounds the exact kappa_2 of the filtered block (observed in all the paper's cases)."""
    prob = W.c1_real_small(n=200, nev=8, nex=4, seed=29)
    A = W.known_spectrum_matrix(prob.lam, prob.seed, False).numpy()
    V0 = W.start_block(prob.n, prob.ell, prob.seed, False)
    V, _ = np.linalg.qr(V0)
    l1, le, bs = prob.bounds
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    Vf = oracle.filter(A, V, [prob.deg_init] * prob.ell, c, e, l1)
    sv = oracle.jacobi_svd(Vf)
    est = math.exp(oracle.log_cond_est(l1, prob.deg_init, prob.deg_init, l1, c, e, 1.0))
    assert sv[0] / sv[-1] <= est


# --------------------------------------------------------------------------
# Lanczos spectral bounds (Algorithm 1's estimation step)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
def test_lanczos_bounds_bracket_the_spectrum(complex_):
    """Ritz values lie inside [lambda_1, lambda_n] (Cauchy interlacing), so the lambda1
    estimate is >= lambda_1; b_sup = theta_max + |beta_m| is >= lambda_n; both are close
    after 25 steps on spectra with well-separated ends."""
    for seed, spec in [(3, W.spectrum_uniform(300, -1, 1, 3)), (4, W.spectrum_clustered(300, 40, 4))]:
        A = W.known_spectrum_matrix(spec, seed, complex_).numpy()
        V = W.start_block(300, 4, seed + 50, complex_)
        (l1, lell, bsup), ritz = oracle.lanczos_bounds(A, V, 25, 30)
        assert l1 >= spec[0] - 1e-12 and l1 - spec[0] < 0.05 * (spec[-1] - spec[0])
        assert bsup >= spec[-1]
        assert ritz.min() >= spec[0] - 1e-12 and ritz.max() <= spec[-1] + 1e-12
        assert l1 <= lell <= bsup


def test_lanczos_full_length_reproduces_the_spectrum():
    """n steps with full re-orthogonalisation on a tiny matrix span the whole space: the
    Ritz values of each run are the eigenvalues (brute force against eigvalsh), the last
    beta vanishes, and the spectral-density estimate counts all n eigenvalues (the weights
    of a run sum to one)."""
    n = 12
    G = W.gaussian((n, n), 8, True)
    A = 0.5 * (G + G.conj().T)
    lam = np.linalg.eigvalsh(A)
    V = W.start_block(n, 2, 9, True)
    (l1, lell, bsup), ritz = oracle.lanczos_bounds(A, V, n, n)
    for r in range(2):
        np.testing.assert_allclose(np.sort(ritz[r]), lam, atol=1e-9)
    assert abs(l1 - lam[0]) < 1e-9
    assert abs(bsup - lam[-1]) < 1e-8
    assert abs(lell - lam[-1]) < 1e-9
    # fewer steps: interlacing Ritz values inside the spectrum
    (_, _, _), ritz = oracle.lanczos_bounds(A, V, n - 1, n)
    assert ritz.min() >= lam[0] - 1e-12 and ritz.max() <= lam[-1] + 1e-12


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,seed", [(12, 8), (16, 9), (14, 21)])
def test_lanczos_density_estimate_counts_eigenvalues_exactly(complex_, n, seed):
    """Pins the lambda_ell output.  With nruns = n full-length runs started at the columns
    of the identity, every run's Ritz values are the eigenvalues and its weight on
    eigenvalue lambda_k is tau = |u_k[r]|^2 (the squared r-th component of the unit
    eigenvector u_k).  Summed over the runs these weights are ||u_k||^2 = 1, and the scale
    n / nruns is 1, so the spectral-density estimate is the exact eigenvalue count: it
    reaches ell at lambda_ell for EVERY ell = 1..n (brute force against eigvalsh).  A weight
    taken from another component of the tridiagonal's eigenvector, or another scale than
    n / nruns, moves lambda_ell off the ell-th eigenvalue."""
    G = W.gaussian((n, n), seed, complex_)
    A = 0.5 * (G + G.conj().T)
    lam = np.linalg.eigvalsh(A)
    V = np.eye(n, dtype=np.complex128 if complex_ else np.float64)
    for ell in range(1, n + 1):
        (l1, lell, bsup), ritz = oracle.lanczos_bounds(A, V, n, ell)
        assert abs(lell - lam[ell - 1]) <= 1e-9 * max(1.0, abs(lam).max()), (ell, lell, lam[ell - 1])
        assert abs(l1 - lam[0]) <= 1e-9 * max(1.0, abs(lam).max())


@pytest.mark.parametrize("opt", [False, True])
def test_condition_estimate_against_exact_kappa_per_iteration(opt):
    """Figure 2's comparison on a synthetic spectrum, exact kappa_2 of [Y V] from the oracle's
    one-sided Jacobi SVD before every QR.  Before any pair is locked the printed estimate
    (Eq. full-est, eta = 1) bounds kappa_2 (Proposition th:2-2's regime); the locked-aware
    form max(Eq. full-est, |rho_1|^{m_ell}) bounds it in every iteration; and both forms
    coincide while nothing is locked."""
    prob = W.c2_complex_clustered(n=360, nev=18, nex=6, seed=33)
    A = W.known_spectrum_matrix(prob.lam, prob.seed, True).numpy()
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    l1, le, bs = prob.bounds
    r = oracle.solve(A, V0, prob.nev, prob.nex, opt_degree=opt, lambda1=l1, lambda_ell=le,
                     b_sup=bs, cond_est_mode=1, log_exact_kappa=True)
    assert r["status"] == 0
    locked_seen = False
    for g in r["logs"]:
        assert g["log_cond_est_locked"] >= g["log_cond_est_paper"]
        assert g["log_cond_est_locked"] >= g["log_kappa_exact"] - 1e-9
        if g["locked_before"] == 0:
            assert g["log_cond_est_paper"] >= g["log_kappa_exact"] - 1e-9
        else:
            locked_seen = True
        assert g["log_cond_est"] == g["log_cond_est_locked"]
    assert locked_seen

"""The seeded input recipes (no GPU): the synthetic problems have the spectra, structure and
determinism the design states for the stand-ins of the paper's workloads."""
import math

import numpy as np
import pytest

import workloads as W


def test_clustered_spectrum_recipe():
    """C2 spectrum: nev + nex values geometric in [-2, -1] (lambda_i = -2 + 2^{(i-1)/(c-1)} - 1,
    densest near -2), the rest uniform in [-1, 50], ascending."""
    n, c = 2000, 120
    lam = W.spectrum_clustered(n, c, 2)
    assert lam.shape == (n,) and np.all(np.diff(lam) >= 0)
    i = np.arange(c)
    expect = -2.0 + (np.power(2.0, i / (c - 1)) - 1.0)
    np.testing.assert_array_equal(lam[:c], expect)  # the cluster sorts below the rest
    assert lam[0] == -2.0 and lam[c - 1] == -1.0
    assert lam[c:].min() >= -1.0 and lam[c:].max() <= 50.0
    gaps = np.diff(lam[:c])
    assert np.all(np.diff(gaps) > 0)  # geometric: gaps grow away from -2


def test_uniform_spectrum_and_bounds():
    lam = W.spectrum_uniform(500, -1.0, 1.0, 3)
    assert lam.min() >= -1.0 and lam.max() <= 1.0 and np.all(np.diff(lam) >= 0)
    l1, le, bs = W.bounds_for(lam, 30)
    assert l1 == lam[0] and le == lam[29]
    assert bs == lam[-1] + 1e-3 * max(1.0, lam[-1] - lam[0])


@pytest.mark.parametrize("complex_", [False, True])
def test_known_spectrum_matrix(complex_):
    """A = Q diag(lambda) Q^H: exactly Hermitian, column-major, with the prescribed
    eigenvalues (LAPACK's eigvalsh) and the same matrix for the same seed."""
    lam = W.spectrum_uniform(150, -3.0, 7.0, 4)
    A = W.known_spectrum_matrix(lam, 11, complex_)
    assert A.stride() == (1, 150)
    a = A.numpy()
    np.testing.assert_array_equal(a, a.conj().T)
    np.testing.assert_allclose(np.linalg.eigvalsh(a), lam, atol=1e-12)
    np.testing.assert_array_equal(W.known_spectrum_matrix(lam, 11, complex_).numpy(), a)
    assert not np.array_equal(W.known_spectrum_matrix(lam, 12, complex_).numpy(), a)


def test_start_block_is_seeded_gaussian():
    """V0: (g1 + i g2)/sqrt(2) entries (unit variance), Fortran order, reproducible."""
    V = W.start_block(4000, 50, 9, True)
    assert V.flags.f_contiguous and V.shape == (4000, 50)
    assert abs(np.mean(np.abs(V) ** 2) - 1.0) < 0.02
    assert abs(np.mean(V.real ** 2) - 0.5) < 0.02 and abs(np.mean(V.imag ** 2) - 0.5) < 0.02
    np.testing.assert_array_equal(W.start_block(4000, 50, 9, True), V)
    R = W.start_block(4000, 50, 9, False)
    assert R.dtype == np.float64 and abs(np.mean(R ** 2) - 1.0) < 0.02


def test_problem_configs():
    c1, c2 = W.c1_real_small(), W.c2_complex_clustered()
    assert (c1.n, c1.nev, c1.nex, c1.complex_, c1.deg_init, c1.opt_degree) == (1000, 20, 10, False, 20, False)
    assert (c2.n, c2.nev, c2.nex, c2.complex_) == (10000, 500, 100, True)
    assert (c2.deg_init, c2.deg_min, c2.deg_max, c2.opt_degree, c2.tol) == (20, 10, 36, True, 1e-10)
    assert c2.ell == 600 and c2.bounds[1] == c2.lam[599]
    c4 = W.c4_sequence_base()
    assert (c4.n, c4.nev, c4.nex, c4.complex_) == (8000, 400, 80, False)


def test_sequence_perturbation_is_symmetric_and_scaled():
    """1e-3 (G + G^T) / (2 sqrt(n)): symmetric, spectral norm ~ 1e-3 * sqrt(2) (semicircle
    edge of (G + G^T)/sqrt(2n) is 2, times sqrt(2)/2)."""
    n = 400
    P = W.symmetric_perturbation(n, 5)
    np.testing.assert_array_equal(P, P.T)
    nrm = np.linalg.norm(P, 2)
    assert 0.8e-3 * math.sqrt(2.0) < nrm < 1.2e-3 * math.sqrt(2.0)


def test_serving_stream_recipe():
    """C5: n log-uniform in [500, 8000], dtype about 50/50, nev = ceil(0.05 n), nex = ceil(nev/5)."""
    s = W.serving_stream(256, 5)
    ns = np.array([r["n"] for r in s])
    assert ns.min() >= 500 and ns.max() < 8000
    assert abs(np.median(np.log(ns)) - 0.5 * (math.log(500) + math.log(8000))) < 0.25
    frac = np.mean([r["complex"] for r in s])
    assert 0.35 < frac < 0.65
    for r in s:
        assert r["nev"] == math.ceil(0.05 * r["n"]) and r["nex"] == math.ceil(r["nev"] / 5)
    assert s == W.serving_stream(256, 5)

"""Seeded synthetic eigenproblems shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the smoke check.  It
builds INPUTS only -- Hermitian matrices of known spectrum, start blocks,
spectral bounds -- and holds none of the eigensolver's arithmetic.

Known-spectrum construction: A = Q diag(lambda) Q^H with Q the unitary factor of
the QR factorisation of a seeded (complex) Gaussian matrix, then A is made
exactly Hermitian by (A + A^H)/2.  The Gaussian draws come from numpy's PCG64
so that a seed gives the same matrix on every machine; the O(n^3) QR and
product may run on a CUDA device through torch (input preparation, not the
solver).

The workload sizes are the five stand-ins for the paper's DFT/BSE test matrices
(Table 2): small real (n=1000), complex clustered (n=10000), mixed-precision
complex (n=20000), a correlated sequence (n=8000) and a serving stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(shape, seed: int, complex_: bool) -> np.ndarray:
    """i.i.d. N(0,1) (real) or (g1 + i g2)/sqrt(2) (complex), Fortran order."""
    g = rng(seed)
    if complex_:
        x = (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / math.sqrt(2.0)
    else:
        x = g.standard_normal(shape)
    return np.asfortranarray(x)


def spectrum_uniform(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """n eigenvalues uniform in [lo, hi], ascending."""
    return np.sort(rng(seed + 7919).uniform(lo, hi, n))


def spectrum_clustered(n: int, n_cluster: int, seed: int, lo=-2.0, hi=-1.0, rest=(-1.0, 50.0)):
    """n_cluster values clustered geometrically in [lo, hi] (densest near lo:
    lambda_i = lo + (hi - lo) (2^{(i-1)/(n_cluster-1)} - 1)), the rest uniform in
    `rest`; ascending."""
    i = np.arange(n_cluster, dtype=np.float64)
    clus = lo + (hi - lo) * (np.power(2.0, i / max(n_cluster - 1, 1)) - 1.0)
    others = rng(seed + 104729).uniform(rest[0], rest[1], n - n_cluster)
    return np.sort(np.concatenate([clus, others]))


def known_spectrum_matrix(lam: np.ndarray, seed: int, complex_: bool, device: str = "cpu"):
    """A = Q diag(lam) Q^H as a torch tensor (float64 / complex128) on `device`,
    stored column-major (strides (1, n)), the layout the solver libraries take."""
    import torch

    n = lam.shape[0]
    G = gaussian((n, n), seed, complex_)
    dt = torch.complex128 if complex_ else torch.float64
    Gt = torch.from_numpy(np.ascontiguousarray(G)).to(device=device, dtype=dt)
    Q, R = _qr(Gt)
    # fix the phases so that Q does not depend on the QR routine's sign choice
    d = torch.diagonal(R)
    ph = d / d.abs()
    Q = Q * ph.unsqueeze(0)
    lt = torch.from_numpy(lam).to(device=device, dtype=torch.float64).to(dt)
    A = (Q * lt.unsqueeze(0)) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    del Q, R, Gt
    return A.mT.contiguous().mT


def _qr(Gt):
    """QR of the Gaussian matrix on its device.  torch loads its CUDA linear-algebra
    library lazily by name; under a profiler's injection that lookup can fail, so the
    library is preloaded by path first and the CPU is used as a last resort."""
    import torch

    if Gt.is_cuda:
        import ctypes
        import glob
        import os
        for lib in glob.glob(os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")):
            try:
                ctypes.CDLL(lib, mode=ctypes.RTLD_GLOBAL)
            except OSError:
                pass
        try:
            return torch.linalg.qr(Gt)
        except RuntimeError:
            Q, R = torch.linalg.qr(Gt.cpu())
            return Q.to(Gt.device), R.to(Gt.device)
    return torch.linalg.qr(Gt)


def start_block(n: int, ell: int, seed: int, complex_: bool) -> np.ndarray:
    """The random V0 of Algorithm 1 (Gaussian, n x ell, Fortran order)."""
    return gaussian((n, ell), seed + 15485863, complex_)


def bounds_for(lam: np.ndarray, ell: int, margin: float = 1e-3):
    """(lambda1, lambda_ell, b_sup) estimates: the exact lowest and ell-th values
    and an upper bound slightly above the largest eigenvalue, i.e. what a few
    Lanczos steps deliver for a well-separated top of the spectrum."""
    span = float(lam[-1] - lam[0])
    return float(lam[0]), float(lam[ell - 1]), float(lam[-1] + margin * max(span, 1.0))


@dataclass
class Problem:
    name: str
    n: int
    nev: int
    nex: int
    complex_: bool
    seed: int
    lam: np.ndarray
    deg_init: int = 20
    deg_min: int = 10
    deg_max: int = 36
    opt_degree: bool = False
    tol: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def ell(self):
        return self.nev + self.nex

    @property
    def bounds(self):
        return bounds_for(self.lam, self.ell)


def c1_real_small(n=1000, nev=20, nex=10, seed=1) -> Problem:
    """Real symmetric, lambda uniform in [-1, 1], fixed degree 20."""
    return Problem("real_uniform_n%d" % n, n, nev, nex, False, seed,
                   spectrum_uniform(n, -1.0, 1.0, seed), deg_init=20, opt_degree=False)


def c2_complex_clustered(n=10000, nev=500, nex=100, seed=2, n_cluster=None) -> Problem:
    """Complex Hermitian; the lowest nev+nex values clustered geometrically in
    [-2, -1], the rest uniform in [-1, 50]; optimised degrees in [10, 36]."""
    if n_cluster is None:
        n_cluster = nev + nex
    return Problem("complex_clustered_n%d" % n, n, nev, nex, True, seed,
                   spectrum_clustered(n, n_cluster, seed), deg_init=20, deg_min=10, deg_max=36,
                   opt_degree=True)


def c4_sequence_base(n=8000, nev=400, nex=80, seed=4) -> Problem:
    return Problem("real_sequence_n%d" % n, n, nev, nex, False, seed,
                   spectrum_uniform(n, -1.0, 1.0, seed), deg_init=20, opt_degree=True)


def symmetric_perturbation(n: int, seed: int, scale: float = 1e-3, complex_: bool = False):
    """scale * (G + G^H) / (2 sqrt(n)) -- the SCF-like step between correlated problems."""
    G = gaussian((n, n), seed, complex_)
    return scale * (G + G.conj().T) / (2.0 * math.sqrt(n))


def serving_stream(count=256, seed=5, n_lo=500, n_hi=8000):
    """Request descriptors: n log-uniform in [n_lo, n_hi], dtype 50/50,
    nev = ceil(0.05 n), nex = ceil(nev / 5), lambda uniform in [-1, 1]."""
    g = rng(seed)
    out = []
    for r in range(count):
        n = int(math.floor(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        cplx = bool(g.integers(0, 2))
        nev = int(math.ceil(0.05 * n))
        nex = int(math.ceil(nev / 5))
        out.append({"id": r, "n": n, "complex": cplx, "nev": nev, "nex": nex,
                    "seed": seed * 100003 + r})
    return out

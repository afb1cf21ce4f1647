"""Mixed-precision filter (BF16x3 on tcgen05 tensor cores) through the C ABI.

Tolerances:
  * one step (degree 1) against the same split products evaluated in FP64 from the
    BF16 hi/lo planes: the only difference is FP32 accumulation over K = n (real) or
    2n (complex) terms, <= ~sqrt(K) 2^-24 relative -> 2e-5 normwise per column;
  * one step against exact FP64: the BF16x3 representation error (2^-17 per operand,
    the dropped lo*lo term 2^-32) -> 1e-4 normwise per column;
  * whole filter (degrees up to 36) against the FP64 oracle: the per-step error
    propagates through the recurrence -> 2e-3 normwise per column.
"""
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
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().mT


def split_bf16(x):
    t = torch.from_numpy(np.ascontiguousarray(x))
    hi = t.to(torch.bfloat16).to(torch.float64)
    lo = (t - hi).to(torch.bfloat16).to(torch.float64)
    return hi.numpy(), lo.numpy()


def stacked(A):
    if np.iscomplexobj(A):
        return np.block([[A.real, -A.imag], [A.imag, A.real]])
    return A


def stack_v(V):
    if np.iscomplexobj(V):
        return np.vstack([V.real, V.imag])
    return V


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,ncols", [(333, 37), (1000, 300), (40, 1), (129, 257)])
def test_one_step_matches_split_products(cl, handle, complex_, n, ncols):
    lam = W.spectrum_uniform(n, -1.0, 1.0, 3)
    A = W.known_spectrum_matrix(lam, 3, complex_).numpy()
    V = W.start_block(n, ncols, 4, complex_)
    c, e, l1 = 0.3, 0.9, -1.0
    got = cl.chase_filter(handle, dev(A), dev(V), [1] * ncols, c, e, l1,
                          prec=cl.CHASE_BF16X3).cpu().numpy()
    # degree 1: out = (sigma1/e)(A V - c V), sigma1 = e/(l1 - c)
    s = 1.0 / (l1 - c)
    Ah, Al = split_bf16(stacked(A))
    Vh, Vl = split_bf16(stack_v(V))
    Y = Ah @ Vh + Ah @ Vl + Al @ Vh
    ref_split = s * (Y - c * stack_v(V))
    ref_exact = s * (stack_v(A @ V) - c * stack_v(V))
    g = stack_v(got)
    e_split = np.linalg.norm(g - ref_split, axis=0) / np.linalg.norm(ref_split, axis=0)
    e_exact = np.linalg.norm(g - ref_exact, axis=0) / np.linalg.norm(ref_exact, axis=0)
    assert e_split.max() <= 2e-5, e_split.max()
    assert e_exact.max() <= 1e-4, e_exact.max()


@pytest.mark.parametrize("complex_", [False, True])
def test_filter_matches_oracle_within_mixed_tolerance(cl, handle, complex_):
    n = 700
    degs = [0, 1, 2, 5, 8, 8, 13, 20, 20, 27, 36] + [36] * 140
    lam = W.spectrum_clustered(n, 200, 9) if complex_ else W.spectrum_uniform(n, -1, 1, 9)
    A = W.known_spectrum_matrix(lam, 9, complex_).numpy()
    V = W.start_block(n, len(degs), 10, complex_)
    l1, le, bs = lam[0], lam[len(degs) - 1], lam[-1] + 1e-3
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    ref = oracle.filter(A, V, degs, c, e, l1)
    got = cl.chase_filter(handle, dev(A), dev(V), degs, c, e, l1, prec=cl.CHASE_BF16X3).cpu().numpy()
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err[0] == 0.0  # degree 0: untouched
    assert err.max() <= 2e-3, err.max()


@pytest.mark.parametrize("complex_", [False, True])
def test_mixed_solve_reaches_fp64_accuracy(cl, handle, complex_):
    """Mixed mode: BF16x3 filters while residuals are large, FP64 filters at the end;
    the result meets tol and matches the known spectrum like the FP64 path."""
    prob = W.c2_complex_clustered(n=1500, nev=60, nex=20, seed=12)
    prob.complex_ = complex_
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, complex_, device="cuda")
    V0 = W.start_block(prob.n, prob.ell, prob.seed, complex_)
    out = {}
    for prec in (cl.CHASE_FP64, cl.CHASE_BF16X3):
        cfg = cl.config_default(opt_degree=1, prec=prec)
        rc, ev, res, st, logs = cl.chase_solve(handle, A_t, dev(V0), prob.nev, prob.nex, prob.bounds, cfg)
        assert rc == 0
        assert res.max() < prob.tol
        assert np.abs(ev - prob.lam[:prob.nev]).max() <= 1e-10 * np.abs(prob.lam).max()
        out[prec] = (ev, st)
    ev_mp, st_mp = out[cl.CHASE_BF16X3]
    assert st_mp["n_lowprec_iters"] >= 1
    np.testing.assert_allclose(ev_mp, out[cl.CHASE_FP64][0], atol=1e-10 * np.abs(prob.lam).max())

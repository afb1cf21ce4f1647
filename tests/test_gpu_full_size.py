"""Parity at the full size of the headline workload (complex Hermitian n = 10000, 600
columns, the clustered spectrum), in the configuration the benchmark times (FP64-emulated
products, the handle on the current stream).

* Filter: the whole Chebyshev filter (degrees 10..36 across the block, ascending, as the
  solver orders them) against the oracle on sampled columns, which it computes one by one;
  per-column normwise relative difference <= 1e-11, every entry within 1e-11 of its
  column's largest entry (the FP64 parity tolerances of the
  filter tests).
* Solve: properties that hold at any size, checked with plain torch products on the GPU:
  eigenvalues against the known spectrum (<= 1e-10 ||A||), residuals ||A v - lambda v||
  recomputed for sampled columns (<= 1e-10 ||A||) and the reported ones (< tol),
  orthonormality of the returned block (<= 1e-12).
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
def c2():
    prob = W.c2_complex_clustered()
    A = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    return prob, A


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().mT


def test_full_size_filter_sampled_columns_match_oracle(cl, c2):
    prob, A = c2
    n, k = prob.n, prob.ell
    degs = np.sort(np.random.default_rng(3).integers(10, 37, size=k)).astype(np.int32)
    V = W.start_block(n, k, 21, True)
    l1, le, bs = prob.bounds
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    h = cl.Handle(0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        got = cl.chase_filter(h, A, dev(V), degs, c, e, l1, prec=cl.CHASE_FP64_EMU)
        torch.cuda.synchronize()
    finally:
        h.close()
    cols = [0, 1, k // 3, k // 2, k - 2, k - 1]
    Ah = A.cpu().numpy()
    ref = oracle.filter(Ah, V[:, cols], degs[cols], c, e, l1)
    g = got[:, cols].cpu().numpy()
    err = np.linalg.norm(g - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-11, err
    # entrywise: every entry within 1e-11 of its column's largest entry
    ent = (np.abs(g - ref) / np.abs(ref).max(axis=0)).max()
    assert ent <= 1e-11, ent


def test_full_size_solve_properties(cl, c2):
    prob, A = c2
    V = dev(W.start_block(prob.n, prob.ell, prob.seed, True))
    h = cl.Handle(0, stream=torch.cuda.current_stream().cuda_stream)
    cfg = cl.config_default(opt_degree=1, deg_init=prob.deg_init, deg_min=prob.deg_min,
                            deg_max=prob.deg_max, tol=prob.tol, prec=cl.CHASE_FP64_EMU)
    try:
        rc, ev, res, st, logs = cl.chase_solve(h, A, V, prob.nev, prob.nex, prob.bounds, cfg)
    finally:
        h.close()
    normA = np.abs(prob.lam).max()
    assert rc == 0
    assert res.max() < prob.tol
    assert np.abs(ev - prob.lam[:prob.nev]).max() <= 1e-10 * normA
    Y = V[:, :prob.nev]
    G = Y.mH @ Y
    assert (G - torch.eye(prob.nev, dtype=G.dtype, device=G.device)).abs().max().item() <= 1e-12
    cols = torch.tensor([0, 7, prob.nev // 2, prob.nev - 1], device=Y.device)
    Ys = Y[:, cols]
    lam = torch.tensor(ev[cols.cpu().numpy()], dtype=Ys.dtype, device=Ys.device)
    R = A @ Ys - Ys * lam
    rn = torch.linalg.vector_norm(R, dim=0).cpu().numpy()
    assert rn.max() <= 1e-10 * normA, rn


def test_mixed_precision_workload_full_size(cl, measurements):
    """The mixed-precision workload at its full size: complex Hermitian n = 20000, nev 1000,
    nex 200, the clustered spectrum.  The BF16x3 filter (while the residuals are large, then
    FP64-accurate products) and the FP64-emulated path both converge (residuals < tol) with
    eigenvalues within 1e-10 ||A|| of the known spectrum and of each other; the two times
    are reported in the terminal summary."""
    prob = W.c2_complex_clustered(n=20000, nev=1000, nex=200, seed=3)
    A = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    normA = np.abs(prob.lam).max()
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec in (("bf16x3", cl.CHASE_BF16X3), ("fp64_emu", cl.CHASE_FP64_EMU)):
        h = cl.Handle(0, stream=stream.cuda_stream)
        cfg = cl.config_default(opt_degree=1, deg_init=prob.deg_init, deg_min=prob.deg_min,
                                deg_max=prob.deg_max, tol=prob.tol, prec=prec)
        try:
            V = dev(V0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, ev, res, st, _ = cl.chase_solve(h, A, V, prob.nev, prob.nex, prob.bounds, cfg)
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            h.close()
        del V
        assert rc == 0, name
        assert res.max() < prob.tol, name
        err = float(np.abs(ev - prob.lam[:prob.nev]).max())
        assert err <= 1e-10 * normA, (name, err)
        out[name] = (ev, e0.elapsed_time(e1) / 1e3, st, err)
    assert np.abs(out["bf16x3"][0] - out["fp64_emu"][0]).max() <= 1e-10 * normA
    tb, tf = out["bf16x3"][1], out["fp64_emu"][1]
    measurements.append(
        "mixed-precision workload (complex n=20000, nev 1000, nex 200): bf16x3 %.2f s "
        "(%d iterations, %d in BF16x3, max |dlambda| %.1e), fp64_emu %.2f s (%d iterations, "
        "max |dlambda| %.1e), speed-up %.2fx"
        % (tb, out["bf16x3"][2]["iterations"], out["bf16x3"][2]["n_lowprec_iters"], out["bf16x3"][3],
           tf, out["fp64_emu"][2]["iterations"], out["fp64_emu"][3], tf / tb))

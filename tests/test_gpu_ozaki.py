"""FP64-accurate products by the Ozaki scheme on the BF16 tensor cores (CHASE_FP64_EMU),
through the C ABI.

Tolerances: the emulated product is accurate to ~2^-53 |A||V| per entry (each scaled
operand rounded to a 57-bit integer, the integer product formed exactly from 17 modular
products and the Chinese remainder theorem, then rounded once to FP64), i.e. the same class
as an FP64 GEMM; the tests hold it to the FP64 tolerances of the parity tests:
  * one filter step vs FP64 numpy: every entry within the Ozaki bound
    K 2^-53 max_k|A_mk| max_k|V_kc| (plus 2^-52 for the FP64 recurrence terms), and
    dense columns within 1e-13 normwise, as an FP64 product;
  * whole filter vs the oracle: <= 1e-11 (as the native FP64 filter);
  * solve: eigenvalues within 1e-10 ||A|| of the oracle and of the known spectrum.
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


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,ncols", [
    (333, 37), (517, 70), (1000, 130),
    (40, 1),       # one row block (the pair's odd CTA has no rows), narrowest column tile
    (64, 16),      # K of one or two 64-wide blocks, a 16-column tile (8-row halves)
    (129, 257),    # ragged: two column tiles, two row blocks
])
def test_one_step_is_fp64_accurate(cl, handle, complex_, n, ncols):
    lam = W.spectrum_uniform(n, -3.0, 40.0, 3)
    A = W.known_spectrum_matrix(lam, 3, complex_).numpy()
    V = W.start_block(n, ncols, 4, complex_)
    if ncols > 2:
        V[:, 1] *= 1e-9      # columns of very different scale
        V[5, 2] = 1e3        # one large entry
    c, e, l1 = 20.0, 21.0, -5.0
    got = cl.chase_filter(handle, dev(A), dev(V), [1] * ncols, c, e, l1,
                          prec=cl.CHASE_FP64_EMU).cpu().numpy()
    s = 1.0 / (l1 - c)
    ref = s * (A @ V - c * V)
    # Ozaki-scheme error class: each entry of A V within K 2^-53 max_k|A_mk| max_k|V_kc|
    # (row / column scalings, 56-bit slices), the FP64 recurrence terms within 2^-52
    K = 2 * n if complex_ else n
    bound = abs(s) * (K * 2.0 ** -53 * np.abs(A).max(axis=1)[:, None] * np.abs(V).max(axis=0)[None, :]
                      + abs(c) * np.abs(V) * 2.0 ** -52)
    ratio = np.abs(got - ref) / bound
    assert ratio.max() <= 1.0, ratio.max()
    # and dense columns (all but the two rescaled ones) are as accurate as an FP64 product
    dense = [j for j in range(ncols) if j not in (1, 2)]
    err = np.linalg.norm((got - ref)[:, dense], axis=0) / np.linalg.norm(ref[:, dense], axis=0)
    assert err.max() <= 1e-13, err.max()


@pytest.mark.parametrize("complex_", [False, True])
def test_one_step_long_k_sampled(cl, handle, complex_):
    """K = 8192 with enough output tiles (64 x 10) that no split of K is taken: every CTA
    runs 64 exact chunks and the tail over the whole K.  Sampled rows against FP64 numpy
    within the Ozaki bound, dense columns to 1e-13 normwise (an FP64 product's class)."""
    n = 4096 if complex_ else 8192
    ncols = 640
    lam = W.spectrum_uniform(n, -3.0, 40.0, 13)
    At = W.known_spectrum_matrix(lam, 13, complex_, device="cuda")
    A = At.cpu().numpy()
    V = W.start_block(n, ncols, 14, complex_)
    c, e, l1 = 20.0, 21.0, -5.0
    got = cl.chase_filter(handle, At, dev(V), [1] * ncols, c, e, l1,
                          prec=cl.CHASE_FP64_EMU).cpu().numpy()
    rows = np.sort(np.random.default_rng(5).choice(n, 256, replace=False))
    s = 1.0 / (l1 - c)
    ref = s * (A[rows] @ V - c * V[rows])
    K = 2 * n if complex_ else n
    bound = abs(s) * (K * 2.0 ** -53 * np.abs(A[rows]).max(axis=1)[:, None] * np.abs(V).max(axis=0)[None, :]
                      + abs(c) * np.abs(V[rows]) * 2.0 ** -52)
    assert (np.abs(got[rows] - ref) / bound).max() <= 1.0
    err = np.linalg.norm(got[rows] - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-13, err.max()


@pytest.mark.parametrize("complex_", [False, True])
def test_filter_matches_oracle_fp64_tolerance(cl, handle, complex_):
    n = 517
    degs = [0, 1, 2, 2, 5, 8, 8, 13, 20, 20, 27, 36] + [36] * 60
    lam = W.spectrum_clustered(n, 100, 6) if complex_ else W.spectrum_uniform(n, -1, 1, 6)
    A = W.known_spectrum_matrix(lam, 6, complex_).numpy()
    V = W.start_block(n, len(degs), 7, complex_)
    l1, le, bs = lam[0], lam[len(degs) - 1], lam[-1] + 1e-3
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    ref = oracle.filter(A, V, degs, c, e, l1)
    got = cl.chase_filter(handle, dev(A), dev(V), degs, c, e, l1, prec=cl.CHASE_FP64_EMU).cpu().numpy()
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-11, err.max()
    # entrywise: every entry within 1e-11 of its column's largest entry
    ent = (np.abs(got - ref) / np.abs(ref).max(axis=0)).max()
    assert ent <= 1e-11, ent


@pytest.mark.parametrize("prec_name", ["CHASE_FP64_EMU", "CHASE_BF16X3"])
def test_solve_with_emulated_fp64_matches_oracle(cl, handle, prec_name):
    prob = W.c2_complex_clustered(n=1200, nev=40, nex=12, seed=8)
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    A = A_t.cpu().numpy()
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    l1, le, bs = prob.bounds
    ref = oracle.solve(A, V0, prob.nev, prob.nex, opt_degree=True, lambda1=l1, lambda_ell=le, b_sup=bs)
    cfg = cl.config_default(opt_degree=1, prec=getattr(cl, prec_name))
    rc, ev, res, st, logs = cl.chase_solve(handle, A_t, dev(V0), prob.nev, prob.nex, prob.bounds, cfg)
    normA = np.abs(prob.lam).max()
    assert rc == 0
    assert res.max() < prob.tol
    assert np.abs(ev - ref["evals"]).max() <= 1e-10 * normA
    assert np.abs(ev - prob.lam[:prob.nev]).max() <= 1e-10 * normA
    if prec_name == "CHASE_FP64_EMU":
        assert abs(st["iterations"] - ref["summary"]["iterations"]) <= 1
        assert abs(st["matvecs"] - ref["summary"]["matvecs"]) <= 0.05 * ref["summary"]["matvecs"]


def test_solve_with_graph_launched_filters(cl):
    """chase_config.graph_filter = 1: every filter call of the solve is recorded into a
    CUDA graph and launched as one unit on a handle with its own (capturable) stream.  The
    graph runs the same kernels in the same order, so the results equal the directly
    launched solve's bit for bit, and match the oracle; on torch's default stream (not
    capturable) the option falls back to direct launches with the same results."""
    prob = W.c2_complex_clustered(n=900, nev=30, nex=10, seed=18)
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    l1, le, bs = prob.bounds
    ref = oracle.solve(A_t.cpu().numpy(), V0, prob.nev, prob.nex, opt_degree=True, lambda1=l1,
                       lambda_ell=le, b_sup=bs)
    normA = np.abs(prob.lam).max()
    runs = {}
    for name, stream, graph in (("direct", None, 0), ("graph", None, 1), ("legacy", 0, 1)):
        h = cl.Handle(0, stream=stream)
        try:
            cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU, graph_filter=graph)
            V = dev(V0)
            rc, ev, res, st, _ = cl.chase_solve(h, A_t, V, prob.nev, prob.nex, prob.bounds, cfg)
        finally:
            h.close()
        assert rc == 0, name
        assert res.max() < prob.tol
        assert np.abs(ev - ref["evals"]).max() <= 1e-10 * normA
        runs[name] = (ev, res, V.cpu().numpy(), st)
    assert runs["graph"][3]["graph_launches"] == runs["graph"][3]["iterations"]
    assert runs["graph"][3]["t_graph_build"] > 0.0
    assert runs["direct"][3]["graph_launches"] == 0 and runs["legacy"][3]["graph_launches"] == 0
    for name in ("graph", "legacy"):
        np.testing.assert_array_equal(runs[name][0], runs["direct"][0])
        np.testing.assert_array_equal(runs[name][1], runs["direct"][1])
        np.testing.assert_array_equal(runs[name][2], runs["direct"][2])


# --------------------------------------------------------------------------
# QR with emulated-FP64 block products (Gram X^H X and X R^{-1}, Algorithm 2)
# --------------------------------------------------------------------------

def _unitary(n, seed, complex_):
    Q, R = np.linalg.qr(W.gaussian((n, n), seed, complex_))
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def _sv_matrix(n, l, sv, seed, complex_):
    return (_unitary(n, seed, complex_)[:, :l] * sv) @ _unitary(l, seed + 1, complex_).conj().T


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,l,force,log10k", [
    (421, 37, 1, 0), (421, 37, 2, 4), (421, 37, 3, 10),
    (1500, 150, 2, 2),     # several tiles each way, split-K over the long dimension
    (2100, 200, 3, 8),
])
def test_qr_with_emulated_products_matches_oracle(cl, handle, complex_, n, l, force, log10k):
    """Q against the oracle (unique factor with positive diagonal R) to the FP64 parity
    tolerance, orthogonality to 1e-12 (1e-10 for CholQR1), X = Q R with R upper."""
    X = _sv_matrix(n, l, np.logspace(0, -log10k, l), 500 + n + log10k, complex_)
    Qo, vo, io = oracle.qr_dynamic(X, 0.0, force=force)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=force, prec=cl.CHASE_FP64_EMU)
    Q = Xd.cpu().numpy()
    assert rc == 0 and v == force and io == 0 and info == 0
    orth = np.linalg.norm(Q.conj().T @ Q - np.eye(l))
    assert orth <= (1e-10 if force == 1 else 1e-12)
    if 10.0 ** log10k <= 1e4:
        assert np.abs(Q - Qo).max() <= 1e-9
    R = Q.conj().T @ X
    assert np.linalg.norm(np.tril(R, -1)) <= 1e-10 * np.linalg.norm(X)


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n,l", [(900, 100), (1300, 200)])
def test_householder_blocked_emulated_matches_oracle(cl, handle, complex_, n, l):
    """The compact-WY Householder QR with its block products on the emulated-FP64 engine:
    the oracle's Householder Q up to unit phases, orthonormal to 1e-12, R upper."""
    X = _sv_matrix(n, l, np.logspace(0, -12, l), 700 + l, complex_)
    Qo, vo, io = oracle.qr_dynamic(X, 0.0, force=4)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=4, prec=cl.CHASE_FP64_EMU)
    Q = Xd.cpu().numpy()
    assert rc == 0 and v == 4 and info == 0
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(l)) <= 1e-12
    ph = np.sum(Qo.conj() * Q, axis=0)
    np.testing.assert_allclose(np.abs(ph), 1.0, atol=1e-9)
    R = Q.conj().T @ X
    assert np.linalg.norm(np.tril(R, -1)) <= 1e-10 * np.linalg.norm(X)


def test_qr_emulated_escalates_like_fp64(cl, handle):
    """kappa ~ 1e15: a CholQR2 chosen by a too-small estimate fails and escalates; the
    result is orthonormal; a forced CholQR2 reports the failure with X unchanged."""
    X = _sv_matrix(300, 20, np.logspace(0, -15, 20), 78, True)
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 100.0, prec=cl.CHASE_FP64_EMU)
    assert rc == 0 and v in (3, 4) and info != 0
    Q = Xd.cpu().numpy()
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(20)) <= 1e-11
    Xd = dev(X)
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, qr_force=2, prec=cl.CHASE_FP64_EMU)
    assert rc == cl.CHASE_CHOL_FAILED and info > 0
    np.testing.assert_array_equal(Xd.cpu().numpy(), X)


def test_qr_prec_rejects_other_precisions(cl, handle):
    Xd = dev(W.gaussian((50, 5), 1, False))
    rc, v, info = cl.chase_qr(handle, Xd, 1.0, prec=cl.CHASE_TF32, check=False)
    assert rc == -9


def test_autotuner_records_plans_without_changing_results(cl):
    """autotune = 1: the first solve times the candidate launch plans of its emulated
    products (trials > 0) and records the fastest per shape bucket; the results equal an
    untuned solve's bit for bit (every plan forms the same exact integer products); a second
    tuned solve of the same shapes finds every bucket in the table (no trials)."""
    prob = W.c2_complex_clustered(n=1100, nev=40, nex=12, seed=19)
    A_t = W.known_spectrum_matrix(prob.lam, prob.seed, True, device="cuda")
    V0 = W.start_block(prob.n, prob.ell, prob.seed, True)
    cl.autotune_clear()
    out = []
    for tune in (0, 1, 1):
        h = cl.Handle(0)
        try:
            cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU, autotune=tune)
            V = dev(V0)
            rc, ev, res, st, _ = cl.chase_solve(h, A_t, V, prob.nev, prob.nex, prob.bounds, cfg)
        finally:
            h.close()
        assert rc == 0
        out.append((ev, res, V.cpu().numpy(), st))
    assert out[0][3]["autotune_trials"] == 0
    assert out[1][3]["autotune_trials"] > 0
    assert out[2][3]["autotune_trials"] == 0
    for i in (1, 2):
        np.testing.assert_array_equal(out[i][0], out[0][0])
        np.testing.assert_array_equal(out[i][1], out[0][1])
        np.testing.assert_array_equal(out[i][2], out[0][2])
    table = cl.autotune_table()
    assert table and all(ln.startswith("ozm ") and "tile_cap=" in ln for ln in table)
    cl.autotune_clear()
    assert cl.autotune_table() == []

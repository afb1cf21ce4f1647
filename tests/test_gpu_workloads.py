"""Workload patterns on the GPU: a warm-started sequence of correlated problems and the
continuous-batching service (same result alone and in the mix)."""
import threading

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().mT


def test_sequence_warm_start_matches_oracle(cl):
    """SCF-like chain A_{k+1} = A_k + 1e-3 (G + G^T)/(2 sqrt n): each problem warm-started
    from the previous final block on both sides; eigenvalues agree with the oracle chain, and
    warm starts need fewer iterations than the cold first solve."""
    n, nev, nex, steps = 500, 16, 6, 3
    lam = W.spectrum_uniform(n, -1.0, 1.0, 41)
    A = W.known_spectrum_matrix(lam, 41, False).numpy()
    V_gpu = W.start_block(n, nev + nex, 41, False)
    V_orc = V_gpu.copy()
    h = cl.Handle(0)
    iters = []
    try:
        for k in range(steps):
            if k > 0:
                A = A + W.symmetric_perturbation(n, 1000 + k)
                A = 0.5 * (A + A.T)
            bsup = lam[-1] + 1e-3 + 3e-3 * k
            l1 = (lam[0] if k == 0 else ev[0]) - 1e-2 * (k > 0)
            bounds = (l1, lam[nev + nex - 1], bsup)
            Vd = dev(V_gpu)
            cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU)
            rc, ev, res, st, _ = cl.chase_solve(h, dev(A), Vd, nev, nex, bounds, cfg)
            ref = oracle.solve(A, V_orc, nev, nex, opt_degree=True, lambda1=bounds[0],
                               lambda_ell=bounds[1], b_sup=bounds[2])
            assert rc == 0 and ref["status"] == 0
            assert res.max() < 1e-10
            np.testing.assert_allclose(ev, ref["evals"], atol=1e-10 * np.abs(lam).max())
            np.testing.assert_allclose(ev, np.linalg.eigvalsh(A)[:nev], atol=1e-10 * np.abs(lam).max())
            iters.append(st["iterations"])
            V_gpu = Vd.cpu().numpy()
            V_orc = ref["V"]
    finally:
        h.close()
    assert max(iters[1:]) < iters[0]


def _requests(cl, specs, seed0=0):
    from paper_2603_10514_gb300.serve import Request
    reqs = []
    for i, (n, cplx) in enumerate(specs):
        nev = max(4, int(np.ceil(0.05 * n)))
        nex = max(2, int(np.ceil(nev / 5)))
        lam = W.spectrum_uniform(n, -1.0, 1.0, seed0 + i)
        A = W.known_spectrum_matrix(lam, seed0 + i, cplx, device="cuda")
        V0 = dev(W.start_block(n, nev + nex, seed0 + i, cplx))
        cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU)
        reqs.append((Request(rid=i, A=A, V0=V0, nev=nev, nex=nex,
                             bounds=W.bounds_for(lam, nev + nex), cfg=cfg), lam))
    return reqs


def test_service_results_same_alone_and_in_the_mix(cl):
    from paper_2603_10514_gb300.serve import Server
    specs = [(300, False), (520, True), (410, False), (700, True), (350, True), (610, False)]
    reqs = _requests(cl, specs, seed0=70)
    # alone: one at a time on one handle
    alone = {}
    h = cl.Handle(0)
    try:
        for req, lam in reqs:
            V = req.V0.clone()
            rc, ev, res, st, _ = cl.chase_solve(h, req.A, V, req.nev, req.nex, req.bounds, req.cfg)
            assert rc == 0 and res.max() < 1e-10
            assert np.abs(ev - lam[:req.nev]).max() <= 1e-10
            alone[req.rid] = (ev.copy(), res.copy(), V.cpu().numpy())
    finally:
        h.close()
    # in the mix: all submitted at once to 3 concurrent slots (own handles and streams)
    srv = Server(slots=3, make_handle=lambda i: cl.Handle(0))
    try:
        for req, _ in reqs:
            srv.submit(req)
        srv.drain()
    finally:
        srv.close()
    assert srv.max_in_flight >= 2
    for req, _ in reqs:
        ev_a, res_a, V_a = alone[req.rid]
        assert req.status == 0
        np.testing.assert_array_equal(req.evals, ev_a)      # bitwise: same kernels, same order
        np.testing.assert_array_equal(req.resid, res_a)
        np.testing.assert_array_equal(req.V0.cpu().numpy(), V_a)


def test_batch_service_results_same_alone_and_in_the_mix(cl):
    """The batch-session service: requests submitted together and while others iterate
    share one session (their filter steps in shared launches); each result equals the
    request's solve alone bit for bit."""
    from paper_2603_10514_gb300.serve import BatchServer
    specs = [(300, False), (520, True), (410, False), (700, True), (350, True), (610, False),
             (900, True), (260, False)]
    reqs = _requests(cl, specs, seed0=90)
    alone = {}
    h = cl.Handle(0)
    try:
        for req, lam in reqs:
            V = req.V0.clone()
            rc, ev, res, st, _ = cl.chase_solve(h, req.A, V, req.nev, req.nex, req.bounds, req.cfg)
            assert rc == 0 and res.max() < 1e-10
            assert np.abs(ev - lam[:req.nev]).max() <= 1e-10
            alone[req.rid] = (ev.copy(), res.copy(), V.cpu().numpy())
    finally:
        h.close()
    srv = BatchServer()
    try:
        for req, _ in reqs[:5]:
            srv.submit(req)
        import time
        time.sleep(0.05)  # the rest arrive while the first ones iterate
        for req, _ in reqs[5:]:
            srv.submit(req)
        srv.drain()
    finally:
        srv.close()
    assert srv.max_seen_in_flight >= 2
    for req, _ in reqs:
        ev_a, res_a, V_a = alone[req.rid]
        assert req.status == 0
        np.testing.assert_array_equal(req.evals, ev_a)
        np.testing.assert_array_equal(req.resid, res_a)
        np.testing.assert_array_equal(req.V0.cpu().numpy(), V_a)

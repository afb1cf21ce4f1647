"""Batch sessions (chase_batch_* / chase_solve_batch) through the C ABI: many uneven
eigenproblems advanced together, their emulated-FP64 filter steps sharing launches.

Each problem's arithmetic is the one chase_solve performs (the grouped modular products are
exact integer products like the single ones, the rest runs per problem), so the batch must
reproduce the single solves bit for bit; against the known spectrum the usual FP64
tolerances hold (eigenvalues within 1e-10 ||A||, residuals < tol).
"""
import numpy as np
import pytest

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


def _problems(specs):
    out = []
    for (n, cplx, nev, nex, seed) in specs:
        lam = W.spectrum_uniform(n, -1.0, 1.0, seed)
        A = W.known_spectrum_matrix(lam, seed, cplx, device="cuda")
        V0 = W.start_block(n, nev + nex, seed, cplx)
        out.append((A, V0, nev, nex, lam))
    return out


SPECS = [(300, False, 15, 3, 41), (517, True, 26, 6, 42), (777, False, 39, 8, 43),
         (1024, True, 52, 11, 44), (1290, False, 65, 13, 45), (450, True, 23, 5, 46),
         (1500, True, 75, 15, 47), (640, False, 32, 7, 48)]


def _single(cl, A, V0, nev, nex, lam, cfg):
    h = cl.Handle(0)
    try:
        V = dev(V0)
        rc, ev, res, st, _ = cl.chase_solve(h, A, V, nev, nex, W.bounds_for(lam, nev + nex), cfg)
    finally:
        h.close()
    return rc, ev, res, V.cpu().numpy(), st


def test_batch_reproduces_single_solves_bit_for_bit(cl):
    cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU)
    probs = _problems(SPECS)
    h = cl.Handle(0)
    try:
        bp = [cl.BatchProblem(A, dev(V0), nev, nex, W.bounds_for(lam, nev + nex), cfg)
              for (A, V0, nev, nex, lam) in probs]
        status = cl.chase_solve_batch(h, bp, cfg)
    finally:
        h.close()
    assert status == [0] * len(probs)
    for p, (A, V0, nev, nex, lam) in zip(bp, probs):
        normA = np.abs(lam).max()
        assert p.resid.max() < 1e-10
        assert np.abs(p.evals - lam[:nev]).max() <= 1e-10 * normA
        rc, ev, res, V, st = _single(cl, A, V0, nev, nex, lam, cfg)
        assert rc == 0
        np.testing.assert_array_equal(p.evals, ev)
        np.testing.assert_array_equal(p.resid, res)
        np.testing.assert_array_equal(p.V.cpu().numpy(), V)
        assert p.stats["iterations"] == st["iterations"] and p.stats["matvecs"] == st["matvecs"]


def test_batch_admits_problems_between_steps(cl):
    """Three problems start, two more join after two steps; every one ends with the single
    solve's results."""
    cfg = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU)
    probs = _problems(SPECS[:5])
    h = cl.Handle(0)
    b = cl.Batch(h)
    done = []
    try:
        bp = [cl.BatchProblem(A, dev(V0), nev, nex, W.bounds_for(lam, nev + nex), cfg)
              for (A, V0, nev, nex, lam) in probs]
        for p in bp[:3]:
            b.add(p)
        for _ in range(2):
            done += b.step()
        for p in bp[3:]:
            b.add(p)
        while b.pending():
            done += b.step()
    finally:
        b.close()
        h.close()
    assert sorted(p.id for p in done) == list(range(5))
    for p, (A, V0, nev, nex, lam) in zip(bp, probs):
        assert p.status == 0
        rc, ev, res, V, st = _single(cl, A, V0, nev, nex, lam, cfg)
        np.testing.assert_array_equal(p.evals, ev)
        np.testing.assert_array_equal(p.resid, res)


def test_batch_with_other_precisions_and_lanczos_bounds(cl):
    """A native-FP64 problem and a problem without bounds (Lanczos estimates) share a session
    with emulated ones: each ends with its single solve's results."""
    emu = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64_EMU)
    fp64 = cl.config_default(opt_degree=1, prec=cl.CHASE_FP64)
    probs = _problems(SPECS[:3])
    h = cl.Handle(0)
    b = cl.Batch(h)
    try:
        bp = []
        for i, (A, V0, nev, nex, lam) in enumerate(probs):
            cfg = fp64 if i == 1 else emu
            bounds = None if i == 2 else W.bounds_for(lam, nev + nex)
            bp.append(b.add(cl.BatchProblem(A, dev(V0), nev, nex, bounds, cfg)))
        while b.pending():
            b.step()
    finally:
        b.close()
        h.close()
    for i, (p, (A, V0, nev, nex, lam)) in enumerate(zip(bp, probs)):
        assert p.status == 0
        assert np.abs(p.evals - lam[:nev]).max() <= 1e-10 * np.abs(lam).max()
        cfg = fp64 if i == 1 else emu
        h1 = cl.Handle(0)
        try:
            V = dev(V0)
            rc, ev, res, _, _ = cl.chase_solve(h1, A, V, nev, nex,
                                               None if i == 2 else W.bounds_for(lam, nev + nex), cfg)
        finally:
            h1.close()
        np.testing.assert_array_equal(p.evals, ev)


def test_batch_reports_invalid_problems_without_running_them(cl):
    h = cl.Handle(0)
    b = cl.Batch(h)
    try:
        A = torch.zeros((8, 8), dtype=torch.float64, device="cuda").mT
        with pytest.raises(cl.ChaseError):
            b.add(cl.BatchProblem(A, dev(np.ones((8, 3))), 4, 3, (0.0, 1.0, 0.5)))  # b_sup < lambda_ell
        assert b.pending() == 0
    finally:
        b.close()
        h.close()

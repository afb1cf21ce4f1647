"""Failure detection on the GPU without a fault: a bounded device wait that runs out is
reported to the host as CHASE_ERR_TIMEOUT, promptly, and the handle and the CUDA context
stay usable afterwards (a filter on the same handle still matches the oracle).  Collected
after the parity suites (only tests/test_zz_no_alloc.py comes later)."""
import time

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


def test_device_wait_timeout_is_reported_and_context_stays_usable(cl):
    h = cl.Handle(0)
    try:
        t0 = time.perf_counter()
        rc = cl.chase_selftest_wait_timeout(h, 0.02)
        assert rc == cl.CHASE_ERR_TIMEOUT, rc
        assert time.perf_counter() - t0 < 5.0
        assert cl.chase_selftest_wait_timeout(h, 0.0) == -2  # invalid limit, nothing launched
        n = 300
        lam = W.spectrum_uniform(n, -1.0, 1.0, 31)
        A = W.known_spectrum_matrix(lam, 31, True)
        V = W.start_block(n, 8, 32, True)
        degs = [2, 3, 3, 5, 8, 8, 10, 12]
        l1, le, bs = lam[0], lam[7], lam[-1] + 1e-3
        c, e = 0.5 * (bs + le), 0.5 * (bs - le)
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().mT
        got = cl.chase_filter(h, dev(A.numpy()), dev(V), degs, c, e, l1).cpu().numpy()
        ref = oracle.filter(A.numpy(), V, degs, c, e, l1)
        err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() <= 1e-11
    finally:
        h.close()

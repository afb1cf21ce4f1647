"""chase_filter_noalloc: the filter for callers that cannot allocate device memory.

Callers that run inside a CUDA graph capture, that keep all of HBM in their own
pre-reserved pool, or that cannot afford the device-wide synchronisation of
cudaMalloc / cudaFree need a filter that never allocates.  chase_filter_noalloc
keeps its scratch in a fixed 32 MiB device array inside the library.  This test
calls it through the C ABI twice in a row and checks each result against the
existing chase_filter entry point, within the filter tolerance the parity tests
use (per-column normwise relative difference <= 1e-11), and checks that the
second call changes no device-memory usage.  It lives in a file of its own,
collected last, and passes alone or after the other tests.
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


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().mT


@pytest.mark.parametrize("complex_", [False, True])
def test_noalloc_filter_matches_chase_filter_twice(cl, complex_):
    n = 517
    degs = [0, 1, 2, 2, 5, 8, 8, 13, 20, 20, 27, 36, 36, 36]
    lam = W.spectrum_uniform(n, -1.0, 1.0, 5)
    A = W.known_spectrum_matrix(lam, 5, complex_, device="cuda")
    V = _dev(W.start_block(n, len(degs), 6, complex_))
    l1, le, bs = lam[0], lam[len(degs) - 1], lam[-1] + 1e-3
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    h = cl.Handle(0)
    try:
        ref = cl.chase_filter(h, A, V, degs, c, e, l1).cpu().numpy()
    finally:
        h.close()
    V_before = V.cpu().numpy()
    outs, free = [], []
    for _ in range(2):
        out = cl.chase_filter_noalloc(A, V, degs, c, e, l1)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        outs.append(out.cpu().numpy())
        del out
    for got in outs:
        err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() <= 1e-11, err.max()
    np.testing.assert_array_equal(V.cpu().numpy(), V_before)  # input untouched
    # the output buffer of each call is allocated by torch's caching allocator, which
    # reuses the freed block; the library itself allocates nothing per call
    assert free[0] == free[1]


def test_noalloc_filter_in_place(cl):
    n = 300
    lam = W.spectrum_uniform(n, -1.0, 1.0, 7)
    A = W.known_spectrum_matrix(lam, 7, True, device="cuda")
    V = _dev(W.start_block(n, 6, 8, True))
    degs = [3, 3, 4, 9, 9, 10]
    h = cl.Handle(0)
    try:
        ref = cl.chase_filter(h, A, V, degs, 0.5, 0.6, -1.2).cpu().numpy()
    finally:
        h.close()
    cl.chase_filter_noalloc(A, V, degs, 0.5, 0.6, -1.2, out=V)
    got = V.cpu().numpy()
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-11


def test_noalloc_rejects_blocks_beyond_the_fixed_scratch(cl):
    """n * ncols * 16 bytes above 32 MiB: rejected on the host before any device work."""
    n, ncols = 4096, 520  # 34 MB of complex128
    A = torch.zeros((n, n), dtype=torch.complex128, device="cuda").mT
    V = torch.zeros((ncols, n), dtype=torch.complex128, device="cuda").mT
    out = torch.full((ncols, n), 7.0, dtype=torch.complex128, device="cuda").mT
    with pytest.raises(cl.ChaseError) as ex:
        cl.chase_filter_noalloc(A, V, [2] * ncols, 0.5, 0.6, -1.2, out=out)
    assert ex.value.code == cl.CHASE_ERR_TOO_LARGE
    assert bool((out == 7.0).all())


def test_noalloc_rejects_outputs_that_overlap_its_inputs(cl):
    """An output shifted against the input block, or inside A, would be overwritten while
    the filter still reads it: rejected (-12) before any device work."""
    n = 40
    A = _dev(np.eye(n) * 0.1)
    buf = _dev(np.arange(n * 6, dtype=np.float64).reshape(6, n).T)
    before = buf.cpu().numpy()
    for out, V in ((buf[:, 2:5], buf[:, 0:3]), (A[:, 1:4], buf[:, 0:3])):
        with pytest.raises(cl.ChaseError) as ex:
            cl.chase_filter_noalloc(A, V, [1, 2, 3], 0.5, 0.6, -1.2, out=out)
        assert ex.value.code == -12
    np.testing.assert_array_equal(buf.cpu().numpy(), before)


def test_noalloc_filter_captures_into_a_cuda_graph(cl):
    """Recorded once into a CUDA graph (global capture mode: an allocation would fail the
    capture), replayed on new contents of the same input buffer: every replay matches
    chase_filter on that input."""
    n = 517
    degs = [1, 2, 5, 8, 13, 20, 20, 36]
    lam = W.spectrum_uniform(n, -1.0, 1.0, 9)
    A = W.known_spectrum_matrix(lam, 9, True, device="cuda")
    l1, le, bs = lam[0], lam[len(degs) - 1], lam[-1] + 1e-3
    c, e = 0.5 * (bs + le), 0.5 * (bs - le)
    Vs = _dev(W.start_block(n, len(degs), 10, True))
    Out = torch.empty_like(Vs.mT).mT
    cl.chase_filter_noalloc(A, Vs, degs, c, e, l1, out=Out)  # caches the scratch address
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        cl.chase_filter_noalloc(A, Vs, degs, c, e, l1, out=Out)
    h = cl.Handle(0)
    try:
        for seed in (11, 12):
            Vs.copy_(_dev(W.start_block(n, len(degs), seed, True)))
            g.replay()
            torch.cuda.synchronize()
            ref = cl.chase_filter(h, A, Vs, degs, c, e, l1).cpu().numpy()
            got = Out.cpu().numpy()
            err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
            assert err.max() <= 1e-11, err.max()
    finally:
        h.close()

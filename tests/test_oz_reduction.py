"""Host-side check of the emulated product's modular epilogue (Ozaki scheme II).

Each split of a modular product sums at most 2^16 products of residues in the symmetric range
(|r| <= 128), so |sum| <= 2^30.  The epilogue reduces the sum with a float quotient,
q = floor(fl(fl(sum) * fl(1/p))), r = sum - q p, and one correction step of +p or -p.  That is
exact when the float quotient lies within one of sum / p, which holds for every modulus above 160.
This test replays the reduction in IEEE float32 (round to nearest even, as the kernel computes
it) at every multiple of each modulus in the top octave of the range, one below and one above
it, and at random sums over the whole range, and compares the result with exact integer
arithmetic.  The moduli are read from the kernel source.
"""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2603_10514_gb300", "csrc", "gemm_oz.cu")
SUM_MAX = (1 << 16) * 128 * 128  # longest split (2^16) times the largest residue product


def kernel_moduli():
    text = open(SRC).read()
    m = re.search(r"constexpr int t\[kOzModuli\]\s*=\s*\{([^}]*)\}", text)
    assert m, "moduli table not found"
    return [int(x) for x in m.group(1).replace("\n", " ").split(",") if x.strip()]


def reduce_like_kernel(s, p):
    """The epilogue's reduction of int32 sums s (numpy int64 array holding int32 values)."""
    ip = np.float32(1.0) / np.float32(p)
    q = np.floor(s.astype(np.float32) * ip).astype(np.int64)
    r = s - q * p
    r = np.where(r < 0, r + p, r)
    r = np.where(r >= p, r - p, r)
    return r


def test_moduli_table_is_the_documented_one():
    p = kernel_moduli()
    assert len(p) == 17 and len(set(p)) == 17
    assert min(p) > 160 and max(p) <= 256
    P = 1
    for x in p:
        P *= x
    assert P > 2 * (1 << 17) * (1 << 114)


def test_float_quotient_reduction_is_exact_up_to_the_split_bound():
    rng = np.random.default_rng(7)
    for p in kernel_moduli():
        # every multiple of p in [2^29, 2^30] (the largest float errors), +-1 around it, both signs
        q = np.arange((1 << 29) // p, SUM_MAX // p + 1, dtype=np.int64)
        for off in (-1, 0, 1):
            s = q * p + off
            s = s[np.abs(s) <= SUM_MAX]
            for sgn in (1, -1):
                v = sgn * s
                np.testing.assert_array_equal(reduce_like_kernel(v, p), np.mod(v, p))
        # random sums over the whole range, and the extremes
        v = rng.integers(-SUM_MAX, SUM_MAX + 1, size=200000, dtype=np.int64)
        v = np.concatenate([v, np.array([0, 1, -1, SUM_MAX, -SUM_MAX], dtype=np.int64)])
        np.testing.assert_array_equal(reduce_like_kernel(v, p), np.mod(v, p))


def test_reduction_check_detects_an_unbounded_quotient():
    """The replay is discriminating: without the correction step the remainder leaves [0, p)."""
    p = 191
    s = np.arange(SUM_MAX - 100000, SUM_MAX, dtype=np.int64)
    ip = np.float32(1.0) / np.float32(p)
    q = np.floor(s.astype(np.float32) * ip).astype(np.int64)
    r = s - q * p
    assert np.any((r < 0) | (r >= p))

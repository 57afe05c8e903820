"""The FP64-exact emulated product (8-bit slices on tensor cores, exact recombination) on the CPU:
its slicing and recombination code against exact rational arithmetic."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2204_11404_gb300 import capi


def _rows(rng, m):
    A = rng.standard_normal((m, 32)) * np.exp(rng.uniform(-30, 0, (m, 32)))    # amplitude-like spread
    A[rng.random((m, 32)) < 0.1] = 0.0
    A[0] = 0.0                                                                  # an all-zero row
    A[1, :] = 1e-300 * rng.standard_normal(32)                                  # tiny scale
    A[2, :16] = 0.5
    A[2, 16:] = -0.5                                                            # exact ties
    return A


def _exact(A, B):
    out = np.zeros((A.shape[0], B.shape[0]), dtype=object)
    for r in range(A.shape[0]):
        fa = [Fraction(float(v)) for v in A[r]]
        for n in range(B.shape[0]):
            out[r, n] = sum((fa[k] * Fraction(float(B[n, k])) for k in range(32)), Fraction(0))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_emulated_product_is_fp64_accurate(seed):
    rng = np.random.default_rng(seed)
    m = 24
    A = _rows(rng, m)
    q, _ = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))
    B = np.zeros((32, 32))                     # real embedding of a 16x16 complex matrix (rows = outputs)
    B[0::2, 0::2], B[0::2, 1::2] = q.real, -q.imag
    B[1::2, 0::2], B[1::2, 1::2] = q.imag, q.real
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.ascontiguousarray(B).ctypes.data, m, out.ctypes.data)
    ex = _exact(A, B)
    ref = A @ B.T
    for r in range(m):
        sa = max(abs(float(v)) for v in A[r]) if np.any(A[r]) else 0.0
        for n in range(32):
            sb = max(abs(float(v)) for v in B[n])
            e = abs(Fraction(float(out[r, n])) - ex[r, n])
            # truncation to 56 bits of each input + dropped slice products + one final rounding
            bound = Fraction(2.0 ** -44) * Fraction(sa) * Fraction(sb) + abs(ex[r, n]) * Fraction(2.0 ** -53)
            assert e <= bound, (r, n, float(e), float(bound))
    err = np.abs(out - np.array(ex, dtype=float)).max()
    err_np = np.abs(ref - np.array(ex, dtype=float)).max()
    assert err <= max(4 * err_np, 1e-300)       # as accurate as numpy's FP64 product


def test_zero_and_single_term_rows_are_exact():
    A = np.zeros((2, 32))
    A[1, 5] = 0.123456789012345678
    B = np.eye(32)
    out = np.zeros((2, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, B.ctypes.data, 2, out.ctypes.data)
    assert not out[0].any()
    assert out[1, 5] == A[1, 5] and np.count_nonzero(out[1]) == 1

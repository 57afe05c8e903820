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
    A[3, :] = 1e-300 * rng.standard_normal(32)
    A[3, ::4] = 3e-310 * rng.standard_normal(8)                                 # subnormals beside normals
    return A


def _exact(A, B):
    out = np.zeros((A.shape[0], B.shape[0]), dtype=object)
    for r in range(A.shape[0]):
        fa = [Fraction(float(v)) for v in A[r]]
        for n in range(B.shape[0]):
            out[r, n] = sum((fa[k] * Fraction(float(B[n, k])) for k in range(32)), Fraction(0))
    return out


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_emulated_product_is_fp64_accurate(seed, variant):
    rng = np.random.default_rng(seed)
    m = 24
    A = _rows(rng, m)
    q, _ = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))
    B = np.zeros((32, 32))                     # real embedding of a 16x16 complex matrix (rows = outputs)
    B[0::2, 0::2], B[0::2, 1::2] = q.real, -q.imag
    B[1::2, 0::2], B[1::2, 1::2] = q.imag, q.real
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.ascontiguousarray(B).ctypes.data, m, variant, out.ctypes.data)
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


@pytest.mark.parametrize("variant", [0, 1])
def test_zero_and_single_term_rows_are_exact(variant):
    A = np.zeros((2, 32))
    A[1, 5] = 0.123456789012345678
    B = np.eye(32)
    out = np.zeros((2, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, B.ctypes.data, 2, variant, out.ctypes.data)
    assert not out[0].any()
    assert out[1, 5] == A[1, 5] and np.count_nonzero(out[1]) == 1


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_largest_digits_recombine_exactly(variant):
    """Every 8-bit digit at 255 (mantissas of all ones, one exponent per row) drives each diagonal to
    its largest value, (t + 1) * 32 * 255^2: the 32-bit pieces of the recombination must not overflow.
    Signs are mixed so that the diagonals reach both extremes."""
    big = 2.0 - 2.0 ** -52                                  # 53 one-bits
    sgn = np.where(np.arange(32) % 3 == 0, -1.0, 1.0)
    A = np.stack([np.full(32, big), -np.full(32, big), big * sgn, big * sgn[::-1]])
    B = np.stack([np.full(32, big) if n % 2 == 0 else big * sgn for n in range(32)])
    m = A.shape[0]
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.ascontiguousarray(B).ctypes.data, m, variant, out.ctypes.data)
    ex = _exact(A, B)
    if variant in (0, 1):
        for r in range(m):
            for n in range(32):
                e = abs(Fraction(float(out[r, n])) - ex[r, n])
                assert e <= Fraction(2.0 ** -44) * Fraction(big) ** 2 + abs(ex[r, n]) * Fraction(2.0 ** -53), (r, n)
    else:
        for r in range(m):
            a_ex = sum((v * v for v in ex[r]), Fraction(0))
            err = abs(Fraction(out[r, 0]) - a_ex)
            if variant == 2:
                assert err <= Fraction(2.0 ** -42) * Fraction(big) ** 4 * 32 + a_ex * Fraction(2.0 ** -50), r
            else:
                assert err <= Fraction(out[r, 1]), (r, float(err), out[r, 1])
            if variant == 4:
                n_ex = sum((Fraction(float(v)) ** 2 for v in A[r]), Fraction(0))
                assert abs(Fraction(out[r, 2]) - n_ex) <= Fraction(out[r, 3]), r


def test_bad_variant_rejected():
    a = np.zeros((1, 32))
    with pytest.raises(capi.QecError):
        capi.qec_debug_ozaki_gemm(a.ctypes.data, np.zeros((32, 32)).ctypes.data, 1, 6, a.ctypes.data)


@pytest.mark.parametrize("seed", [0, 3])
def test_probability_sums_are_fp64_accurate(seed):
    """Variant 2: A_r = sum_n (A[r] . B[n])^2 and N_r = sum_k A[r][k]^2 with integer sums of squares."""
    rng = np.random.default_rng(seed)
    m = 12
    A = _rows(rng, m)
    q, _ = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))
    q[3] = 0.0                                   # a zero output row, as projector-like Kraus operators have
    B = np.zeros((32, 32))
    B[0::2, 0::2], B[0::2, 1::2] = q.real, -q.imag
    B[1::2, 0::2], B[1::2, 1::2] = q.imag, q.real
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.ascontiguousarray(B).ctypes.data, m, 2, out.ctypes.data)
    ex = _exact(A, B)
    sb = float(np.abs(B).max())
    tiny = Fraction(2.0 ** -1074)                # sums below the FP64 range flush to zero
    for r in range(m):
        sa = float(np.abs(A[r]).max())
        a_ex = sum((v * v for v in ex[r]), Fraction(0))
        n_ex = sum((Fraction(float(v)) ** 2 for v in A[r]), Fraction(0))
        # per product: the 2^-44 sa sb bound of the emulated product, squared into the sum
        ea = abs(Fraction(out[r, 0]) - a_ex)
        assert ea <= Fraction(2.0 ** -42) * (Fraction(sa) * Fraction(sb)) ** 2 * 32 + a_ex * Fraction(2.0 ** -50) + tiny, (r, float(ea))
        en = abs(Fraction(out[r, 1]) - n_ex)
        assert en <= Fraction(2.0 ** -50) * n_ex + Fraction(2.0 ** -52) * Fraction(sa) ** 2 + tiny, (r, float(en))


@pytest.mark.parametrize("seed", [0, 5, 9])
def test_bounded_probability_sum_contains_the_exact_value(seed):
    """Variant 3: A^ from 3 slices of each operand and its bound: |A_exact - A^| <= bound, with
    the bound below 1e-3 of A for rows of ordinary scale (it is rigorous, so loose: about 1e-4)."""
    rng = np.random.default_rng(seed)
    m = 16
    A = _rows(rng, m)
    q, _ = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))
    q[5] = 0.0
    q[6] *= 1e-9                                   # a small output row beside ordinary ones
    B = np.zeros((32, 32))
    B[0::2, 0::2], B[0::2, 1::2] = q.real, -q.imag
    B[1::2, 0::2], B[1::2, 1::2] = q.imag, q.real
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.ascontiguousarray(B).ctypes.data, m, 3, out.ctypes.data)
    ex = _exact(A, B)
    for r in range(m):
        a_ex = sum((v * v for v in ex[r]), Fraction(0))
        err = abs(Fraction(out[r, 0]) - a_ex)
        assert err <= Fraction(out[r, 1]) + Fraction(2.0 ** -1074), (r, float(err), out[r, 1])
        if float(a_ex) > 1e-200:
            assert out[r, 1] <= 1e-3 * float(a_ex), (r, out[r, 1], float(a_ex))


def _unitary_embedding(rng, zero_row=None, small_row=None):
    q, _ = np.linalg.qr(rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16)))
    if zero_row is not None:
        q[zero_row] = 0.0
    if small_row is not None:
        q[small_row] *= 1e-9
    B = np.zeros((32, 32))
    B[0::2, 0::2], B[0::2, 1::2] = q.real, -q.imag
    B[1::2, 0::2], B[1::2, 1::2] = q.imag, q.real
    return np.ascontiguousarray(B)


@pytest.mark.parametrize("seed", [0, 4, 8])
def test_fused_probability_bounds_contain_the_exact_values(seed):
    """Variant 4, the fused pass's probability: the whole A is one tile under one exponent, each real
    cut to 24 bits, 3 slices, diagonals 0..2.  Per row, |sum_n (A[r] . B[n])^2 - A^| and
    |sum_k A[r][k]^2 - N^| must lie within the returned bounds, whatever the row's scale (zero rows,
    rows far below the tile's largest value, subnormals)."""
    rng = np.random.default_rng(seed)
    m = 16
    A = _rows(rng, m)
    B = _unitary_embedding(rng, zero_row=5, small_row=6)
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, B.ctypes.data, m, 4, out.ctypes.data)
    ex = _exact(A, B)
    tiny = Fraction(2.0 ** -1074)
    for r in range(m):
        a_ex = sum((v * v for v in ex[r]), Fraction(0))
        n_ex = sum((Fraction(float(v)) ** 2 for v in A[r]), Fraction(0))
        assert abs(Fraction(out[r, 0]) - a_ex) <= Fraction(out[r, 1]) + tiny, (r, out[r, 0], float(a_ex), out[r, 1])
        assert abs(Fraction(out[r, 2]) - n_ex) <= Fraction(out[r, 3]) + tiny, (r, out[r, 2], float(n_ex), out[r, 3])


@pytest.mark.parametrize("seed", [1, 2])
def test_fused_probability_bound_is_tight_on_an_ordinary_tile(seed):
    """On a tile whose amplitudes share one scale (the code state's equal magnitudes with noise
    spread), the summed bounds stay below 2e-4 of A + N (measured: 6e-5; the per-output bound takes
    all 32 terms at their largest magnitudes), so the outcome is left to the exact pass only for
    draws within about 1e-4 of their probability."""
    rng = np.random.default_rng(seed)
    m = 128
    A = rng.standard_normal((m, 32)) / 64
    A[rng.random((m, 32)) < 0.5] *= 1e-3
    B = _unitary_embedding(rng)
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, B.ctypes.data, m, 4, out.ctypes.data)
    a_sum, n_sum = out[:, 0].sum(), out[:, 2].sum()
    assert abs(a_sum - float(((A @ B.T) ** 2).sum())) <= out[:, 1].sum()
    assert abs(n_sum - float((A ** 2).sum())) <= out[:, 3].sum()
    assert out[:, 1].sum() + out[:, 3].sum() < 2e-4 * (a_sum + n_sum)


@pytest.mark.parametrize("seed", [0, 5, 9])
def test_speculative_sums_contain_the_exact_values(seed):
    """Variant 5, the speculative pass's two sums of squares: each real cut to its top 24 bits under
    its row's largest exponent (the inputs) or under the whole tile's (the outputs), squared and
    summed in integers, then as FP32 intervals with directed rounding.  Per row the exact sum of
    squares must lie within each estimate's bound, whatever the row's scale (zero rows, rows far
    below the tile's largest value, subnormals, ties)."""
    rng = np.random.default_rng(seed)
    m = 16
    A = _rows(rng, m)
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.zeros((32, 32)).ctypes.data, m, 5, out.ctypes.data)
    tiny = Fraction(2.0 ** -1074)
    for r in range(m):
        n_ex = sum((Fraction(float(v)) ** 2 for v in A[r]), Fraction(0))
        assert abs(Fraction(out[r, 0]) - n_ex) <= Fraction(out[r, 1]) + tiny, (r, out[r, 0], float(n_ex), out[r, 1])
        assert abs(Fraction(out[r, 2]) - n_ex) <= Fraction(out[r, 3]) + tiny, (r, out[r, 2], float(n_ex), out[r, 3])
    assert out[0, 0] == 0.0 and out[0, 2] == 0.0          # the all-zero row


@pytest.mark.parametrize("seed", [1, 2])
def test_speculative_sums_are_tight_on_an_ordinary_tile(seed):
    """On a tile of amplitude-like values (half of them 1e-3 smaller), both bounds stay below 5e-6
    of the sum (measured: 1.1e-6 with the rows' exponents, 1.4e-6 with the tile's), so the outcome
    is left to the exact pass only for draws within about 1e-5 of their probability."""
    rng = np.random.default_rng(seed)
    m = 128
    A = rng.standard_normal((m, 32)) / 64
    A[rng.random((m, 32)) < 0.5] *= 1e-3
    out = np.zeros((m, 32))
    capi.qec_debug_ozaki_gemm(A.ctypes.data, np.zeros((32, 32)).ctypes.data, m, 5, out.ctypes.data)
    ex = float((A ** 2).sum())
    for c in (0, 2):
        assert abs(out[:, c].sum() - ex) <= out[:, c + 1].sum()
        assert out[:, c + 1].sum() < 5e-6 * ex, (c, out[:, c + 1].sum() / ex)

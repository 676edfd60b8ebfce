"""Pins for the FP64 GEMM oracle: results fixed by mathematics, not by the oracle itself."""
import math

import numpy as np
import pytest

from oracle import gemm as og
from paper_2008_13145_gb300 import workloads as wl


def store(opmat: np.ndarray, trans: str) -> np.ndarray:
    """Storage of a logical operand: itself ('N') or its transpose ('T'), as (1, rows, ld)."""
    return np.ascontiguousarray(opmat if trans == "N" else opmat.T)[None]


TRANS = [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")]


@pytest.mark.parametrize("ta,tb", TRANS)
def test_identity(ta, tb):
    rng = np.random.default_rng(5)
    M, K = 7, 5
    A = rng.uniform(-1, 1, (M, K))
    C, den = og.gemm(ta, tb, M, K, K, 1.5, store(A, ta), store(np.eye(K), tb))
    assert np.array_equal(C[0], 1.5 * A)
    assert np.array_equal(den[0], 1.5 * np.abs(A))


@pytest.mark.parametrize("ta,tb", TRANS)
def test_permutation(ta, tb):
    rng = np.random.default_rng(6)
    M, N = 9, 4
    p = rng.permutation(M)
    P = np.zeros((M, M))
    P[np.arange(M), p] = 1.0
    B = rng.uniform(-1, 1, (M, N))
    C, _ = og.gemm(ta, tb, M, N, M, 1.0, store(P, ta), store(B, tb))
    assert np.array_equal(C[0], B[p])


def test_rank1_closed_form():
    M, N = 6, 5
    u = np.arange(M, dtype=np.float64)[:, None]
    v = np.ones((1, N))
    C0 = np.arange(M * N, dtype=np.float64).reshape(M, N)
    C, den = og.gemm("N", "N", M, N, 1, 2.0, u[None], v[None], 0.25, C0[None])
    i = np.arange(M)[:, None]
    assert np.array_equal(C[0], 2.0 * i + 0.25 * C0)
    assert np.array_equal(den[0], 2.0 * i + 0.25 * np.abs(C0))


def test_all_ones():
    M, N, K = 4, 3, 37
    C, den = og.gemm("N", "N", M, N, K, -0.5, np.ones((1, M, K)), np.ones((1, K, N)))
    assert np.all(C == -0.5 * K) and np.all(den == 0.5 * K)


@pytest.mark.parametrize("ta,tb", TRANS)
def test_polynomial_closed_form(ta, tb):
    # A[i,k] = i + s, B[k,j] = s (j + 1), s = k + 1:
    # C[i,j] = (j + 1) (i K(K+1)/2 + K(K+1)(2K+1)/6); asymmetric in i, j and k.
    M, N, K = 5, 6, 11
    s = np.arange(1, K + 1, dtype=np.float64)
    A = np.arange(M, dtype=np.float64)[:, None] + s[None, :]
    B = s[:, None] * (np.arange(N, dtype=np.float64)[None, :] + 1)
    C, _ = og.gemm(ta, tb, M, N, K, 1.0, store(A, ta), store(B, tb))
    i = np.arange(M)[:, None]
    j = np.arange(N)[None, :]
    expect = (j + 1) * (i * K * (K + 1) / 2 + K * (K + 1) * (2 * K + 1) / 6)
    assert np.array_equal(C[0], expect)


@pytest.mark.parametrize("ta,tb", TRANS)
def test_small_integers_exact(ta, tb):
    # |a|,|b| <= 8, K <= 4096: every partial sum is an integer below 2^53,
    # so FP64 is exact and equals int64 arithmetic.
    shape = wl.Shape(33, 17, 257, 3, ta, tb)
    A, B, C0 = wl.gemm_inputs(shape, seed=9, kind="integer", bound=8, beta_nonzero=True)
    C, den = og.gemm(ta, tb, shape.M, shape.N, shape.K, 3.0, A, B, -2.0, C0)
    for b in range(shape.batch):
        Ai = A[b][:, :shape.stored_a()[1]].astype(np.int64)
        Bi = B[b][:, :shape.stored_b()[1]].astype(np.int64)
        opA = Ai if ta == "N" else Ai.T
        opB = Bi if tb == "N" else Bi.T
        c0 = C0[b][:, :shape.N].astype(np.int64)
        assert np.array_equal(C[b], (3 * (opA @ opB) - 2 * c0).astype(np.float64))
        assert np.array_equal(den[b], (3 * (np.abs(opA) @ np.abs(opB)) + 2 * np.abs(c0)).astype(np.float64))


def test_beta_zero_ignores_c0():
    A = np.ones((1, 2, 3))
    B = np.ones((1, 3, 2))
    C, den = og.gemm("N", "N", 2, 2, 3, 1.0, A, B, 0.0, np.full((1, 2, 2), np.nan))
    assert np.array_equal(C[0], np.full((2, 2), 3.0)) and np.array_equal(den[0], np.full((2, 2), 3.0))


def test_nonnegative_den_equals_product():
    rng = np.random.default_rng(3)
    A = rng.integers(0, 5, (1, 8, 9)).astype(np.float64)
    B = rng.integers(0, 5, (1, 9, 10)).astype(np.float64)
    C, den = og.gemm("N", "N", 8, 10, 9, 2.0, A, B)
    assert np.array_equal(C, den)


def test_padding_not_read():
    shape = wl.Shape(5, 6, 7, 2, "T", "N")
    A, B, _ = wl.gemm_inputs(shape, seed=1, ld_multiple=16)  # NaN padding
    C, den = og.gemm("T", "N", 5, 6, 7, 1.0, A, B)
    assert np.all(np.isfinite(C)) and np.all(np.isfinite(den))


def test_entries_match_full():
    shape = wl.Shape(40, 30, 20, 2, "N", "T")
    A, B, C0 = wl.gemm_inputs(shape, seed=2, beta_nonzero=True)
    C, den = og.gemm("N", "T", 40, 30, 20, 0.7, A, B, 0.3, C0)
    pos = wl.sample_positions(shape, 3, 2, seed=4)
    Ce, De = og.gemm_entries("N", "T", 40, 30, 20, 0.7, A, B, 0.3, C0, pos)
    assert np.array_equal(Ce, C[pos[:, 0], pos[:, 1], pos[:, 2]])
    assert np.array_equal(De, den[pos[:, 0], pos[:, 1], pos[:, 2]])


def test_threads_agree():
    shape = wl.Shape(64, 48, 100, 2, "T", "T")
    A, B, _ = wl.gemm_inputs(shape, seed=8)
    C1, _ = og.gemm("T", "T", 64, 48, 100, 1.0, A, B, nthreads=1)
    C4, _ = og.gemm("T", "T", 64, 48, 100, 1.0, A, B, nthreads=4)
    assert np.array_equal(C1, C4)


def test_fp32_rounding_within_gamma_bound():
    # An FP32 dot product in any summation order satisfies
    # |fl(c) - c| <= gamma_K * sum |a||b|, gamma_K = K u / (1 - K u), u = 2^-24.
    rng = np.random.default_rng(12)
    K = 1000
    a = rng.uniform(-1, 1, K).astype(np.float32)
    b = rng.uniform(-1, 1, K).astype(np.float32)
    C, den = og.gemm("N", "N", 1, 1, K, 1.0, a[None, None, :], b[None, :, None])
    acc = np.float32(0)
    for x, y in zip(a, b):
        acc = np.float32(acc + np.float32(x * y))
    u = 2.0 ** -24
    gamma = K * u / (1 - K * u)
    assert og.error_ratio(np.array([acc]), C.ravel(), den.ravel()) <= gamma


def test_error_ratio_semantics():
    assert og.error_ratio([1.0], [1.0], [0.0]) == 0.0
    assert og.error_ratio([1e-30], [0.0], [0.0]) == math.inf
    assert og.error_ratio([np.nan], [0.0], [1.0]) == math.inf
    assert og.error_ratio([1.5, 2.0], [1.0, 2.0], [10.0, 1.0]) == pytest.approx(0.05)

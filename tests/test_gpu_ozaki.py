"""The Ozaki-split tcgen05 GEMM (test hook of include/inla_testing.h) against FP64 numpy.

With S slices of 7 bits per operand row (scaled per 512-wide chunk) the only errors are the
dropped slice products i + j >= S and the slicing remainder, both below
(S + 2) 2^-7S |A_i,:|_max |B_j,:|_max per K term, so
|C - A B^T| <= (S + 2) 2^-7S K max|A_i,:| max|B_j,:| (plus double-float rounding, 2^-46
relative).  An inexact (rounded) FP32 accumulation would show errors near 2^-24 instead.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    L = inla.lib()
    P = C.POINTER(C.c_double)
    L.inla_test_ozaki_gemm.argtypes = [P, P, P] + [C.c_int32] * 8 + [C.c_double, C.c_double]
    return L


def _run(L, A, Bm, Cm, M, N, K, S, ta=0, tb=0, lower=0, kmode=0, alpha=0.0, beta=1.0):
    A = np.ascontiguousarray(A, np.float64)
    Bm = np.ascontiguousarray(Bm, np.float64)
    out = np.ascontiguousarray(Cm.copy(), np.float64)
    P = C.POINTER(C.c_double)
    rc = L.inla_test_ozaki_gemm(A.ctypes.data_as(P), Bm.ctypes.data_as(P), out.ctypes.data_as(P), M, N, K, S, ta, tb,
                                lower, kmode, alpha, beta)
    assert rc == 0, inla.status_string(rc)
    return out


def _bound(A, Bm, S, K):
    ra = np.max(np.abs(A), axis=1)[:, None]
    rb = np.max(np.abs(Bm), axis=1)[None, :]
    return (S + 2) * 2.0 ** (-7 * S) * K * ra * rb + 1e-13 * np.abs(A) @ np.abs(Bm).T


@pytest.mark.parametrize("S", [2, 3, 4, 5, 6])
def test_plain_product_within_slice_bound(lib, S):
    rng = np.random.default_rng(S)
    M, N, K = 300, 260, 576          # ragged tiles, K = one full chunk + a partial one
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    Bm = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, 1)))
    C0 = rng.standard_normal((M, N))
    ref = A @ Bm.T
    got = _run(lib, A, Bm, C0, M, N, K, S)
    err = np.abs(got - ref)
    assert np.all(err <= _bound(A, Bm, S, K)), np.max(err / _bound(A, Bm, S, K))
    if S == 4:
        # far below what a rounded FP32 accumulation would give (~2^-24 relative)
        assert np.max(err / (np.abs(A) @ np.abs(Bm).T)) < 2e-8


def test_accumulate_and_subtract(lib):
    rng = np.random.default_rng(11)
    M = N = 256
    K = 512
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K))
    C0 = rng.standard_normal((M, N)) * 100
    got = _run(lib, A, Bm, C0, M, N, K, 4, alpha=1.0, beta=-1.0)
    ref = C0 - A @ Bm.T
    assert np.max(np.abs(got - ref) / (np.abs(C0) + np.abs(A) @ np.abs(Bm).T)) < 1e-8


def test_transposed_operands_lower_and_k_ranges(lib):
    """C = W^T W over k >= max(row, col) tile starts, lower tiles only: the shape of the
    prior inversion Q_p = W^T W with W lower triangular."""
    rng = np.random.default_rng(3)
    n = 384
    W = np.tril(rng.standard_normal((n, n)))
    got = _run(lib, W, W, np.zeros((n, n)), n, n, n, 4, ta=1, tb=1, lower=1, kmode=1)
    ref = W.T @ W
    il = np.tril_indices(n)
    err = np.abs(got - ref)[il]
    assert np.all(err <= _bound(W.T, W.T, 4, n)[il])
    # k >= col tile start (Z^T W with W lower)
    Z = rng.standard_normal((n, 192))
    got = _run(lib, Z, W, np.zeros((192, n)), 192, n, n, 4, ta=1, tb=1, kmode=2)
    ref = Z.T @ W
    assert np.all(np.abs(got - ref) <= _bound(Z.T, W.T, 4, n))


@pytest.fixture
def narrow(lib):
    """Every launch on the double-buffered 128 x 64 tile (reset to the shape rule after)."""
    assert lib.inla_test_gemm_tile_width(64) == 0
    yield lib
    assert lib.inla_test_gemm_tile_width(0) == 0


@pytest.mark.parametrize("S", [2, 3, 4, 5, 6])
def test_narrow_tile_plain_and_accumulate(narrow, S):
    rng = np.random.default_rng(40 + S)
    M, N, K = 300, 200, 1088         # ragged in M and N (N = 3 tiles of 64 + 8), K = 2 chunks + 64
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    Bm = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, 1)))
    C0 = rng.standard_normal((M, N))
    got = _run(narrow, A, Bm, C0, M, N, K, S)
    ref = A @ Bm.T
    assert np.all(np.abs(got - ref) <= _bound(A, Bm, S, K))
    got = _run(narrow, A, Bm, C0, M, N, K, S, alpha=1.0, beta=-1.0)
    ref = C0 - A @ Bm.T
    assert np.all(np.abs(got - ref) <= _bound(A, Bm, S, K) + 1e-13 * np.abs(C0))


@pytest.mark.parametrize("n", [384, 320])
def test_narrow_tile_lower_and_k_ranges(narrow, n):
    """Lower launches enumerate two 64-wide tiles per 128 rows of the diagonal band; n = 320
    leaves a tile row whose second diagonal tile lies wholly beyond the matrix."""
    rng = np.random.default_rng(n)
    W = np.tril(rng.standard_normal((n, n)))
    C0 = rng.standard_normal((n, n))
    got = _run(narrow, W, W, C0, n, n, n, 4, ta=1, tb=1, lower=1, kmode=1)
    ref = W.T @ W
    il = np.tril_indices(n)
    assert np.all(np.abs(got - ref)[il] <= _bound(W.T, W.T, 4, n)[il])
    Z = rng.standard_normal((n, 96))
    got = _run(narrow, Z, W, np.zeros((96, n)), 96, n, n, 4, ta=1, tb=1, kmode=2)
    assert np.all(np.abs(got - Z.T @ W) <= _bound(Z.T, W.T, 4, n))
    got = _run(narrow, W, Z, np.zeros((n, 96)), n, 96, n, 5, ta=1, tb=1, kmode=3)
    assert np.all(np.abs(got - W.T @ Z) <= _bound(W.T, Z.T, 5, n))


def test_narrow_and_wide_tiles_agree_bitwise(lib):
    """The tile width changes which CTA computes an element and how many columns one MMA
    covers, not the element's chunk sums, their combination or its accumulation into C (N = 48
    selects the narrow tile by shape): the two agree far below the slice truncation."""
    rng = np.random.default_rng(77)
    M, N, K = 520, 48, 704
    A = rng.standard_normal((M, K))
    Bm = rng.standard_normal((N, K))
    C0 = rng.standard_normal((M, N))
    auto = _run(lib, A, Bm, C0, M, N, K, 4, alpha=1.0, beta=-1.0)
    assert lib.inla_test_gemm_tile_width(128) == 0
    try:
        wide = _run(lib, A, Bm, C0, M, N, K, 4, alpha=1.0, beta=-1.0)
    finally:
        assert lib.inla_test_gemm_tile_width(0) == 0
    scale = np.abs(C0) + np.abs(A) @ np.abs(Bm).T
    assert np.max(np.abs(auto - wide) / scale) < 1e-12
    assert lib.inla_test_gemm_tile_width(96) != 0

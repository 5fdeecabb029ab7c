"""The allocation-free GEMM entry point (inla_ozaki_gemm_noalloc) against the allocating
test entry point (inla_test_ozaki_gemm), through the C ABI, on two calls in a row.

Callers that cannot allocate device memory pass their own device buffers; the entry point
keeps its intermediates in a static device array shared by all calls, so the second call
must not be affected by what the first one left behind.  Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla

pytestmark = pytest.mark.gpu


def _bound(A, Bm, S, K):
    ra = np.max(np.abs(A), axis=1)[:, None]
    rb = np.max(np.abs(Bm), axis=1)[None, :]
    return (S + 2) * 2.0 ** (-7 * S) * K * ra * rb + 1e-13 * np.abs(A) @ np.abs(Bm).T


def test_noalloc_gemm_matches_allocating_entry_point_twice():
    import torch
    B.build()
    L = inla.lib()
    P = C.POINTER(C.c_double)
    L.inla_test_ozaki_gemm.argtypes = [P, P, P] + [C.c_int32] * 8 + [C.c_double, C.c_double]
    L.inla_ozaki_gemm_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p] + [C.c_int32] * 4 + [C.c_void_p]
    rng = np.random.default_rng(2024)
    # the largest call first, then a smaller ragged one: whatever the first call leaves in the
    # shared static array (planes, exponents and product of a 512 x 512 x 512 problem) must not
    # reach the second call's result
    shapes = [(512, 512, 512, 5), (300, 200, 320, 4)]
    for M, N, K, S in shapes:
        A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-2, 2, (M, 1)))
        Bm = rng.standard_normal((N, K)) * np.exp(rng.uniform(-2, 2, (N, 1)))
        ref = np.zeros((M, N))
        rc = L.inla_test_ozaki_gemm(A.ctypes.data_as(P), Bm.ctypes.data_as(P), ref.ctypes.data_as(P), M, N, K, S,
                                    0, 0, 0, 0, 0.0, 1.0)
        assert rc == 0, inla.status_string(rc)
        dA = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(Bm).cuda()
        dC = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = L.inla_ozaki_gemm_noalloc(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), M, N, K, S, None)
        assert rc == 0, inla.status_string(rc)
        got = dC.cpu().numpy()
        bound = _bound(A, Bm, S, K)
        assert np.all(np.abs(got - ref) <= bound)
        assert np.all(np.abs(got - A @ Bm.T) <= bound)


def test_noalloc_gemm_rejects_sizes_beyond_its_workspace():
    import torch
    B.build()
    L = inla.lib()
    L.inla_ozaki_gemm_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p] + [C.c_int32] * 4 + [C.c_void_p]
    d = torch.zeros(1024 * 64, dtype=torch.float64, device="cuda")
    p = d.data_ptr()
    assert L.inla_ozaki_gemm_noalloc(p, p, p, 1024, 64, 64, 4, None) == inla.E_BADARG   # M > 512
    assert L.inla_ozaki_gemm_noalloc(p, p, p, 64, 64, 96, 4, None) == inla.E_BADARG    # K not a multiple of 64
    assert L.inla_ozaki_gemm_noalloc(p, p, p, 64, 64, 64, 6, None) == inla.E_BADARG    # slices

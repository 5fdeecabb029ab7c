"""The Gauss-Hermite rule behind the variational Bayes correction (host code of the library, no
GPU): against numpy's rule, and exact on polynomials up to degree 2n - 1."""
import ctypes as C
import math

import numpy as np

from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla


def _rule(n):
    B.build()
    L = inla.lib()
    P = C.POINTER(C.c_double)
    L.inla_test_gauss_hermite.argtypes = [C.c_int32, P, P]
    x, w = np.zeros(n), np.zeros(n)
    assert L.inla_test_gauss_hermite(n, x.ctypes.data_as(P), w.ctypes.data_as(P)) == 0
    return x, w


def test_gauss_hermite_rule_matches_numpy_and_integrates_polynomials():
    for n in (1, 2, 5, 15, 32):
        x, w = _rule(n)
        xr, wr = np.polynomial.hermite.hermgauss(n)
        assert np.max(np.abs(x - xr)) < 1e-12 * max(1.0, np.max(np.abs(xr)))
        assert np.max(np.abs(w - wr) / wr) < 1e-10
        # int x^(2k) e^{-x^2} dx = Gamma(k + 1/2), exact up to degree 2n - 1
        for k in range(n):
            assert abs(np.sum(w * x ** (2 * k)) - math.gamma(k + 0.5)) <= 1e-10 * math.gamma(k + 0.5)

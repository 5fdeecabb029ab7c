"""Host logic of stage 2 (no GPU): the package's exploration designs reproduce the oracle's
point sets and quadrature weights, and the z -> theta map puts the design on the Gaussian
approximation of pi(theta|y)."""
import numpy as np

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import stage2


def _sorted(Z, d):
    return sorted(zip(map(lambda z: tuple(np.round(z, 12)), Z), d))


def test_ccd_and_grid_designs_match_the_oracle_rules():
    for t in (2, 3, 4, 5, 6):
        a, b = _sorted(*stage2.ccd_design(t)), _sorted(*O.ccd_design(t))
        assert len(a) == len(b)
        for (za, wa), (zb, wb) in zip(a, b):
            assert za == zb and abs(wa - wb) <= 1e-12 * abs(wb)
    a, b = _sorted(*stage2.grid_design(3, 0.5, 1.5)), _sorted(*O.grid_design(3, 0.5, 1.5))
    assert a == b and len(a) == 7 ** 3


def test_z_to_theta_whitens_the_gaussian_approximation():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((3, 3))
    negH = M @ M.T + 3 * np.eye(3)
    th = np.array([0.1, -0.4, 2.0])
    Z = rng.standard_normal((5, 3))
    T = stage2.z_to_theta(th, negH, Z)
    assert np.allclose(T, O.z_to_theta(th, negH, Z), atol=1e-12)
    # (theta - theta*)^T negH (theta - theta*) = |z|^2
    D = T - th
    assert np.allclose(np.einsum("ij,jk,ik->i", D, negH, D), np.sum(Z * Z, axis=1), rtol=1e-12)

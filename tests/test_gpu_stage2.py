"""Stage 2 on the GPU against the oracle's definitions: the finite-difference Hessian of
log pi~(theta|y) from one batched evaluation of its 2 t^2 + 1 points, and the latent marginals
integrated over the CCD and grid designs (Section 2, Stage 2; Appendix A.2), element by
element.  Both sides get the same theta* and negative Hessian (the oracle's), so that they
evaluate the same design points.

Tolerances: FP64 path -- Hessian within 1e-5 relative of its largest entry (central
differences with h = 0.02 divide log pi~ rounding of ~1e-13 by h^2), integrated means within
1e-9 of the largest and variances within 1e-9 relative (each point's mode and variances agree
to 1e-9 relative, and the weights exp(log pi~) to 1e-10 relative); mixed path -- the mixed
targets (1e-4 relative), the Hessian within 1e-3 relative of its largest entry."""
import numpy as np
import pytest

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, stage2, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


@pytest.fixture(scope="module")
def case():
    spec, thetas = synth.poisson_n256_m1000_5pts()
    th_star = np.array([0.05, np.log(0.22)])
    negH = -O.hessian_fd(lambda th: O.evaluate(spec, th, want_var=False)["log_post"], th_star, 2e-2)
    return spec, th_star, negH


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hessian_matches_oracle(case, precision):
    spec, th_star, negH = case
    m = inla.Model(spec)
    H = stage2.hessian([m], th_star, h=2e-2, precision=precision)
    tol = 1e-5 if precision == "fp64" else 1e-3
    print(precision, "Hessian", H.tolist(), "oracle", (-negH).tolist())
    assert np.max(np.abs(H + negH)) <= tol * np.max(np.abs(negH))


@pytest.mark.parametrize("precision,design", [("fp64", "ccd"), ("mixed", "ccd"), ("fp64", "grid")])
def test_integrated_marginals_match_oracle(case, precision, design):
    spec, th_star, negH = case
    Z, d = stage2.ccd_design(2) if design == "ccd" else stage2.grid_design(2, 1.0, 2.0)
    m = inla.Model(spec)
    mean, var, thetas, lp, st = stage2.integrate(m, th_star, negH, Z, d, precision=precision)
    assert np.all(st == 0)
    ref = O.integrate_marginals(spec, th_star, negH, Z, d)
    assert np.max(np.abs(thetas - ref["thetas"])) < 1e-12
    e_m = np.max(np.abs(mean - ref["mean"])) / np.max(np.abs(ref["mean"]))
    e_v = np.max(np.abs(var / ref["var"] - 1.0))
    print(f"{precision} {design}: {len(Z)} points, mean rel {e_m:.3e}, var rel {e_v:.3e}")
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert e_m <= tol
    assert e_v <= tol

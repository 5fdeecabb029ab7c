"""Variational Bayes correction of the posterior mean (Appendix A.2.2, Algorithm 2) on the GPU
against the oracle's Algorithm 2, element by element: the oracle refactors Q^c at every step,
the device path steps with the factor of Q* (the same fixed point).  log pi~ and the variances
stay those of the Laplace approximation.  Tolerances: FP64 path 1e-9 relative to the largest
mean (both sides stop at steps below 1e-8 of linearly / quadratically converging iterations;
the remaining distance to the fixed point is ~1e-9 absolute), mixed path 1e-4."""
import numpy as np
import pytest

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_vb_mean_matches_oracle(precision):
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas[:3], precision=precision, flags_extra=inla.OPT_VB_MEAN)
    lp0, st0, xs0, vs0 = inla.eval_batch([m], thetas[:3], precision=precision)
    tol = 1e-9 if precision == "fp64" else 1e-4
    for b in range(3):
        assert st[b] == 0, inla.status_string(st[b])
        r = O.vb_mean(spec, thetas[b])
        scale = np.max(np.abs(r["mean"]))
        e = np.max(np.abs(xs[b] - r["mean"])) / scale
        shift = np.max(np.abs(r["mean"] - r["laplace"]["x_hat"])) / scale
        print(f"{precision} point {b}: VB mean rel err {e:.3e} (the correction itself: {shift:.3e}, {r['iters']} oracle steps)")
        assert e <= tol
        assert shift > 100 * tol  # the correction is visible at this tolerance
        # log pi~ and the variances are the Laplace ones
        assert lp[b] == lp0[b]
        assert np.array_equal(vs[b], vs0[b])


def test_vb_mean_equals_the_mode_for_a_gaussian_likelihood_and_rejects_constraints():
    spec = synth.gaussian_spatial("g_vb", 23, 300)
    m = inla.Model(spec)
    th = np.array([[0.1, np.log(0.25)]])
    lp, st, xs, _ = inla.eval_batch([m], th, flags_extra=inla.OPT_VB_MEAN)
    lp0, st0, xs0, _ = inla.eval_batch([m], th)
    assert st[0] == 0
    assert np.max(np.abs(xs[0] - xs0[0])) <= 1e-12 * max(1.0, np.max(np.abs(xs0[0])))
    sc = synth.spacetime_age("small_st", 11, n_s=8, n_t=6, n_a=4)
    mc = inla.Model(sc)
    with pytest.raises(inla.InlaError) as e:
        inla.eval_batch([mc], np.ones((1, sc.theta_dim)), flags_extra=inla.OPT_VB_MEAN)
    assert e.value.code == inla.E_UNSUPPORTED

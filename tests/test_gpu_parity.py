"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element on
the same seeded inputs, plus edge cases.  FP64 mode: log pi~(theta|y) within relative
1e-10 (|diff| <= 1e-10 max(1, |log pi~|)); x_hat and the marginal variances within 1e-9
relative (both sides solve the same SPD systems in FP64; the bound covers rounding-order
differences amplified by the condition number of Q*)."""
import numpy as np
import pytest

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, synth
from paper_2311_08050_gb300.synth import CSR, Block, Factor, ModelSpec

pytestmark = pytest.mark.gpu

LP_RTOL = 1e-10
X_TOL = 1e-9
V_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    import torch
    assert torch.cuda.is_available()
    torch.cuda.init()


def _check(spec, thetas, lp, st, xs, vs, ref=None, var=True, lp_rtol=LP_RTOL, x_tol=X_TOL, v_rtol=V_RTOL):
    for b, th in enumerate(thetas):
        r = O.evaluate(spec, th, want_var=var) if ref is None else ref[b]
        assert st[b] == 0, inla.status_string(st[b])
        assert abs(lp[b] - r["log_post"]) <= lp_rtol * max(1.0, abs(r["log_post"])), (b, lp[b], r["log_post"])
        xs_ref = r["x_hat"]
        assert np.max(np.abs(xs[b] - xs_ref)) <= x_tol * max(1.0, np.max(np.abs(xs_ref))), b
        if var:
            assert np.max(np.abs(vs[b] / r["var"] - 1.0)) <= v_rtol, b


def test_n256_all_thetas():
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas)
    _check(spec, thetas, lp, st, xs, vs)


def test_ragged_spatial_poisson_with_offset():
    """n = 300 (intercept + 299 points; padded to 512), offsets, several tiles + ragged tail."""
    spec = synth.spatial_poisson("ragged", 7, 299, 900, [0.1, np.log(0.15)])
    spec.offset = np.random.default_rng(1).normal(0.2, 0.3, spec.m)
    thetas = np.array([[0.1, np.log(0.15)], [-0.3, np.log(0.3)]])
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas)
    _check(spec, thetas, lp, st, xs, vs)


def _small_spacetime(n_s=8, n_t=6, n_a=4):
    return synth.spacetime_age("small_st", 11, n_s=n_s, n_t=n_t, n_a=n_a)


# Constrained marginal variances are a difference diag(Q*^-1) - diag(kriging correction)
# whose terms are ~1/eps = 1e5 along the null directions of the intrinsic blocks while the
# result is ~1e-2: a relative cancellation of ~1e7.  FP64 rounding (~1e-15 relative on each
# term after the Cholesky and triangular inverse) then allows ~1e-8 relative on the result,
# on either side; 1e-6 leaves margin for the rounding-order difference of the two sides.
CONSTRAINED_V_RTOL = 1e-6
# The kriged mode x_u - Q*^-1 C^T S^-1 C x_u subtracts two vectors that are large (up to
# ~1/eps times the constraint residual) along the null directions: the same cancellation,
# milder because C x_u -> 0 as Newton converges; observed agreement ~2e-9.
CONSTRAINED_X_TOL = 1e-7


def test_constrained_spacetime_model():
    spec = _small_spacetime()
    thetas = np.array([[1.0, 2.0, 3.0, 4.0, 1.0, 2.0], [0.5, 1.5, 2.5, 3.0, 0.0, 1.0]])
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas)
    _check(spec, thetas, lp, st, xs, vs, x_tol=CONSTRAINED_X_TOL, v_rtol=CONSTRAINED_V_RTOL)
    C = spec.C.to_dense()
    for x in xs:
        assert np.max(np.abs(C @ x)) < 1e-10  # A_c x_hat = 0


def test_uneven_gaussian_models_in_one_batch():
    specs = [synth.gaussian_spatial(f"g{n}", 100 + n, n) for n in (100, 333, 700)]
    ms = [inla.Model(s) for s in specs]
    thetas = np.array([[0.0, np.log(0.2)], [0.2, np.log(0.1)], [-0.1, np.log(0.3)], [0.0, np.log(0.25)]])
    which = np.array([2, 0, 1, 0], dtype=np.int32)
    lp, st, xs, vs = inla.eval_batch(ms, thetas, model_of_theta=which)
    for b in range(4):
        _check(specs[which[b]], thetas[b:b + 1], lp[b:b + 1], st[b:b + 1], xs[b:b + 1], vs[b:b + 1])


def test_no_observations_gives_the_theta_prior():
    """m = 0: Q* = Q_p, so the Laplace approximation is exact and equals log pi(theta)."""
    spec, _ = synth.poisson_n256_m1000_5pts()
    empty = CSR(0, spec.n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    spec0 = ModelSpec("empty", spec.n, "poisson", empty, np.zeros(0), None, spec.blocks, spec.theta_prior)
    th = np.array([0.1, np.log(0.3)])
    m = inla.Model(spec0)
    lp, st, xs, vs = inla.eval_batch([m], th[None])
    assert st[0] == 0
    ref = O.log_theta_prior(spec0, th)
    assert abs(lp[0] - ref) < 1e-9
    assert np.max(np.abs(xs[0])) == 0.0


def test_failed_point_does_not_poison_the_batch():
    """A theta whose covariance overflows (sigma = e^400) makes a non-finite pivot: that point
    reports NOT_SPD while the other point of the batch is unaffected."""
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 1, (40, 2))
    A = CSR.from_rows(80, 40, [np.array([rng.integers(0, 40)]) for _ in range(80)], [np.ones(1)] * 80)
    y = rng.standard_normal(80)
    blk = Block("dense_exp", 40, points=pts, theta_sigma=0, theta_range_x=1, theta_range_y=1, theta_iid=2,
                nugget=1e-6)
    spec = ModelSpec("sing", 40, "gaussian", A, y, None, [blk],
                     [("gauss", 0, 1), ("gauss", 0, 1), ("gauss", 0, 1)], lik_prec=2.0)
    m = inla.Model(spec)
    thetas = np.array([[400.0, np.log(0.2), 1.0], [0.0, np.log(0.2), 1.0]])
    lp, st, xs, vs = inla.eval_batch([m], thetas)
    assert st[0] == inla.E_NOT_SPD
    assert st[1] == 0
    r = O.evaluate(spec, thetas[1])
    assert abs(lp[1] - r["log_post"]) <= LP_RTOL * abs(r["log_post"])


def test_eval_theta_and_marginals_entry_points():
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    lp, x, iters = inla.eval_theta(m, thetas[2])
    r = O.evaluate(spec, thetas[2])
    assert abs(lp - r["log_post"]) <= LP_RTOL * abs(r["log_post"])
    assert iters == r["newton_iters"]
    mean, var = inla.marginals(m, thetas[2])
    assert np.max(np.abs(mean - r["x_hat"])) <= X_TOL * np.max(np.abs(r["x_hat"]))
    assert np.max(np.abs(var / r["var"] - 1)) <= V_RTOL


def test_bad_arguments_are_rejected():
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    with pytest.raises(inla.InlaError) as e:
        inla.eval_batch([m], np.array([[np.nan, 0.0]]))
    assert e.value.code == inla.E_BADARG
    bad = synth.poisson_n256_m1000_5pts()[0]
    bad.y = bad.y.copy()
    bad.y[0] = -1.0  # negative count
    with pytest.raises(inla.InlaError) as e:
        inla.Model(bad)
    assert e.value.code == inla.E_BADARG


@pytest.mark.slow
def test_n4096_fd_points_subset():
    spec, thetas = synth.poisson_n4096_m20000_fd7()
    sub = thetas[[0, 3]]
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], sub)
    _check(spec, sub, lp, st, xs, vs)


@pytest.mark.slow
def test_spacetime_one_point():
    spec, thetas = synth.spacetime_n8149_m8000_fd13()
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas[:1])
    _check(spec, thetas[:1], lp, st, xs, vs, x_tol=CONSTRAINED_X_TOL, v_rtol=CONSTRAINED_V_RTOL)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_intercept_seen_by_more_than_4096_observations(precision):
    """m = 6000 observations all load the intercept: its row of A^T and its A^T D A pair have
    more than 4096 contributions and are reduced by whole blocks (the other rows by one warp
    each); the results match the oracle like any other model."""
    spec = synth.spatial_poisson("heavy_intercept", synth.SEED_BASE + 91, 255, 6000, [0.0, np.log(0.2)])
    thetas = np.array([[0.0, np.log(0.2)], [0.2, np.log(0.3)]])
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision=precision)
    if precision == "fp64":
        _check(spec, thetas, lp, st, xs, vs)
    else:
        _check(spec, thetas, lp, st, xs, vs, lp_rtol=1e-3 / 3000.0, x_tol=1e-4, v_rtol=1e-4)

"""The Moore-Penrose / Woodbury covariance route (Section 3.1, Eq. (woodeqn)) on the GPU against
the oracle's Eq. (woodeqn), element by element, on a constrained space-time model (intrinsic
blocks: Q+ is a genuine pseudo-inverse, the route needs no constraint handling) and on a dense
spatial model with fewer observations than latent effects.  Mixed-path tolerance: 1e-4 relative
on the variances (the route's m x m system is factored by the mixed Cholesky)."""
import numpy as np
import pytest

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _compare(spec, thetas, kriging_rtol=None):
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed", flags_extra=inla.OPT_WOODBURY_VAR)
    lpk, stk, xsk, vsk = inla.eval_batch([m], thetas, precision="mixed")
    for b in range(len(thetas)):
        assert st[b] == 0, inla.status_string(st[b])
        r = O.woodbury_marginals(spec, thetas[b])
        e = np.max(np.abs(vs[b] / r["var"] - 1.0))
        ek = np.max(np.abs(vs[b] / vsk[b] - 1.0))
        print(f"{spec.name} point {b}: Woodbury var rel err {e:.3e}; against the kriging route {ek:.3e}")
        assert e <= 1e-4
        assert lp[b] == lpk[b] and np.array_equal(xs[b], xsk[b])
        if kriging_rtol is not None:
            assert ek <= kriging_rtol


def test_woodbury_route_on_a_constrained_spacetime_model():
    spec = synth.spacetime_age("small_st", 11, n_s=8, n_t=6, n_a=4)
    thetas = np.array([[1.0, 2.0, 3.0, 4.0, 1.0, 2.0], [0.5, 1.5, 2.5, 3.0, 0.0, 1.0]])
    _compare(spec, thetas, kriging_rtol=1e-3)  # equal as eps -> 0 (eps = 1e-5 here)


def test_woodbury_route_on_a_dense_spatial_model():
    spec = synth.spatial_poisson("dense_m200", synth.SEED_BASE + 93, 299, 200, [0.0, np.log(0.2)])
    thetas = np.array([[0.0, np.log(0.2)], [0.3, np.log(0.15)]])
    _compare(spec, thetas, kriging_rtol=1e-4)  # no intrinsic block: Q+ = Q_p^-1, the routes agree


def test_woodbury_route_rejects_what_it_does_not_cover():
    spec, th = synth.poisson_n256_m1000_5pts()  # m = 1000 > the padded n = 256
    m = inla.Model(spec)
    for kw in (dict(precision="mixed"), dict(precision="fp64")):
        with pytest.raises(inla.InlaError) as e:
            inla.eval_batch([m], th[:1], flags_extra=inla.OPT_WOODBURY_VAR, **kw)
        assert e.value.code == inla.E_UNSUPPORTED

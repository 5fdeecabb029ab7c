"""Full-size parity with the FP64 oracle, element by element, in the launch configuration the
benchmark times (every point of a call batched together on the device):

* the n = 16384 Poisson workload (9-point FD batch, mixed path as benchmarked: the slice counts
  the precision autotuner picks for the model), compared at two FD points (the centre and the
  last axial point);
* the constrained space-time model at full size (n = 8149, k = 1486), mixed path with its tuned
  slice counts, one point;
* one Gaussian model of each size n in {512, 1024, 2048, 4096} from the 64-model workload,
  FP64 and mixed paths.

Tolerances: the stated targets of the mixed form (log pi~ within 1e-3 absolute, marginal
variances within 1e-4 relative; the mode within 1e-4 relative) and, in FP64 mode, those of
test_gpu_parity.py.  The oracle needs about two minutes per point at n = 16384 on the host.
"""
import numpy as np
import pytest

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, synth, tune

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

LP_ABS = 1e-3
V_RTOL = 1e-4
X_RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _errors(r, lp, x, v):
    e_lp = abs(lp - r["log_post"])
    e_x = np.max(np.abs(x - r["x_hat"])) / max(1.0, np.max(np.abs(r["x_hat"])))
    e_v = np.max(np.abs(v / r["var"] - 1.0))
    return e_lp, e_x, e_v


def test_mixed_n16384_fd_batch_against_oracle_at_two_points():
    spec, thetas = synth.poisson_n16384_m100000_fd9()
    m = inla.Model(spec)
    tr = tune.tune_precision(m, thetas[0])
    print("n=16384 tuned slices", tr.opts())
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed", **tr.opts())
    assert np.all(st == 0), st
    for b in (0, len(thetas) - 1):
        r = O.evaluate(spec, thetas[b])
        e_lp, e_x, e_v = _errors(r, lp[b], xs[b], vs[b])
        print(f"n=16384 point {b}: log pi~ abs {e_lp:.3e}, x_hat rel {e_x:.3e}, var rel {e_v:.3e}")
        assert e_lp <= LP_ABS, (b, e_lp)
        assert e_x <= X_RTOL, (b, e_x)
        assert e_v <= V_RTOL, (b, e_v)


def test_mixed_spacetime_full_size_against_oracle():
    spec, thetas = synth.spacetime_n8149_m8000_fd13()
    m = inla.Model(spec)
    tr = tune.tune_precision(m, thetas[0])
    print("space-time tuned slices", tr.opts())
    lp, st, xs, vs = inla.eval_batch([m], thetas[:1], precision="mixed", **tr.opts())
    assert st[0] == 0, inla.status_string(st[0])
    r = O.evaluate(spec, thetas[0])
    e_lp, e_x, e_v = _errors(r, lp[0], xs[0], vs[0])
    print(f"space-time n=8149 k=1486: log pi~ abs {e_lp:.3e}, x_hat rel {e_x:.3e}, var rel {e_v:.3e}")
    assert e_lp <= LP_ABS
    assert e_x <= X_RTOL
    assert e_v <= V_RTOL
    C = spec.C.to_dense()
    assert np.max(np.abs(C @ xs[0])) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gaussian_models_one_per_size_against_oracle(precision):
    specs, thetas = synth.gaussian_64_models_n512_4096()
    pick = []
    for n in (512, 1024, 2048, 4096):
        pick.append(next(i for i, sp in enumerate(specs) if sp.n == n))
    ms = [inla.Model(specs[i]) for i in pick]
    th = thetas[pick]
    lp, st, xs, vs = inla.eval_batch(ms, th, model_of_theta=np.arange(4, dtype=np.int32), precision=precision)
    for j, i in enumerate(pick):
        assert st[j] == 0, inla.status_string(st[j])
        r = O.evaluate(specs[i], th[j])
        e_lp, e_x, e_v = _errors(r, lp[j], xs[j], vs[j])
        print(f"{precision} gaussian n={specs[i].n}: log pi~ abs {e_lp:.3e}, x rel {e_x:.3e}, var rel {e_v:.3e}")
        if precision == "fp64":
            assert e_lp <= 1e-10 * max(1.0, abs(r["log_post"]))
            assert e_x <= 1e-9
            assert e_v <= 1e-9
        else:
            assert e_lp <= LP_ABS
            assert e_x <= X_RTOL
            assert e_v <= V_RTOL

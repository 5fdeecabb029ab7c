"""Mixed-precision path (double-float storage, Ozaki-split tcgen05 GEMMs: 5 slices for the prior
inversion and the factor at the mode, 4 for the Newton factorisations, double-float 64 x 64
diagonal tiles) against the FP64 oracle, and at full size against the FP64 GPU path (itself
pinned to the oracle by test_gpu_parity.py).

Tolerances are the stated targets for the mixed form: |log pi~ - oracle| <= 1e-3 and the
marginal variances within 1e-4 relative.  The mode is the fixed point of Newton steps whose
gradient A^T (y - w) - Q_p x is exact up to the error of the mixed-precision prior precision
Q_p, so x_hat inherits that relative error (~1e-6 observed); it is held to 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, synth

pytestmark = pytest.mark.gpu

LP_ABS = 1e-3
V_RTOL = 1e-4
X_RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _check(spec, thetas, lp, st, xs, vs, v_rtol=V_RTOL, x_rtol=X_RTOL):
    errs = []
    for b, th in enumerate(thetas):
        r = O.evaluate(spec, th)
        assert st[b] == 0, inla.status_string(st[b])
        e_lp = abs(lp[b] - r["log_post"])
        e_x = np.max(np.abs(xs[b] - r["x_hat"])) / max(1.0, np.max(np.abs(r["x_hat"])))
        e_v = np.max(np.abs(vs[b] / r["var"] - 1))
        errs.append((e_lp, e_x, e_v, int(np.argmax(np.abs(vs[b] / r["var"] - 1)))))
        assert e_lp <= LP_ABS, (b, e_lp)
        assert e_x <= x_rtol, (b, e_x)
        assert e_v <= v_rtol, (b, e_v)
    print("mixed errors (log_post abs, x rel, var rel):", errs)
    return errs


def test_mixed_poisson_n256_m1000_5pts():
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed")
    _check(spec, thetas, lp, st, xs, vs)


def test_precision_ladder_error_decreases_with_slices():
    """Each extra 7-bit slice should cut the log pi~ error against the oracle (2^-7 per rung
    in the truncation term); the error must fall monotonically from 2 to 5 slices."""
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    r = O.evaluate(spec, thetas[0])
    errs = []
    for S in (2, 3, 4, 5):
        lp, st, _, _ = inla.eval_batch([m], thetas[:1], precision="mixed", slices=S, want_x=False, want_var=False)
        assert st[0] == 0
        errs.append(abs(lp[0] - r["log_post"]))
    print("ladder errors", errs)
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_six_slices_reach_fp64_accuracy():
    """Six slices for the prior inversion and the factor at the mode (Newton steps at 4, which
    only steer the iteration): log pi~ within 1e-10 relative of the oracle (the FP64 target),
    below the five-slice error, on both n = 256 points tried."""
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    for th in thetas[:2]:
        r = O.evaluate(spec, th)
        e = {}
        for S in (5, 6):
            lp, st, _, _ = inla.eval_batch([m], th[None], precision="mixed", slices=S, newton_slices=4,
                                           want_x=False, want_var=False)
            assert st[0] == 0
            e[S] = abs(lp[0] - r["log_post"])
        rel6 = e[6] / max(1.0, abs(r["log_post"]))
        print(f"log pi~ {r['log_post']:.6f}: error 5 slices {e[5]:.3e}, 6 slices {e[6]:.3e} (rel {rel6:.2e})")
        assert e[6] < e[5]
        assert rel6 <= 1e-10


def test_mixed_ragged_with_offset():
    spec = synth.spatial_poisson("ragged", 7, 299, 900, [0.1, np.log(0.15)])
    spec.offset = np.random.default_rng(1).normal(0.2, 0.3, spec.m)
    thetas = np.array([[0.1, np.log(0.15)], [-0.3, np.log(0.3)]])
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed")
    _check(spec, thetas, lp, st, xs, vs)


def test_mixed_constrained_spacetime():
    spec = synth.spacetime_age("small_st", 11, n_s=8, n_t=6, n_a=4)
    thetas = np.array([[1.0, 2.0, 3.0, 4.0, 1.0, 2.0], [0.5, 1.5, 2.5, 3.0, 0.0, 1.0]])
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed")
    _check(spec, thetas, lp, st, xs, vs)
    C = spec.C.to_dense()
    for x in xs:
        # the kriging correction runs in the mixed precision: C x_hat = 0 to ~1e-7
        assert np.max(np.abs(C @ x)) < 1e-6


def test_mixed_gaussian_uneven_groups():
    specs = [synth.gaussian_spatial(f"g{n}", 100 + n, n) for n in (100, 333)]
    ms = [inla.Model(s) for s in specs]
    thetas = np.array([[0.0, np.log(0.2)], [0.2, np.log(0.1)], [-0.1, np.log(0.3)]])
    which = np.array([1, 0, 1], dtype=np.int32)
    lp, st, xs, vs = inla.eval_batch(ms, thetas, model_of_theta=which, precision="mixed")
    for b in range(3):
        _check(specs[which[b]], thetas[b:b + 1], lp[b:b + 1], st[b:b + 1], xs[b:b + 1], vs[b:b + 1])


@pytest.mark.slow
def test_mixed_n4096_fd_subset():
    spec, thetas = synth.poisson_n4096_m20000_fd7()
    sub = thetas[[0, 5]]
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], sub, precision="mixed")
    _check(spec, sub, lp, st, xs, vs)


def test_double_float_covariance_matches_fp64_definition():
    """The mixed path builds the dense covariance in double-float (its own exp by ln 2
    reduction and a Taylor series, sqrt by a Newton step): against numpy's FP64 over distances
    d from 0 to ~40 range units.  exp(-d) has relative condition number d and a double-float
    distance carries ~2^-46 relative error; the exponential itself (two squarings of a
    double-float Taylor value) adds ~4 * 2^-46: the bound is (1 + d) * 6e-14 relative, hence
    sigma^2 (1 + d) e^-d * 6e-14 <= 6e-14 sigma^2 absolute (far below the 2^-35 slice error of
    the products the covariance enters)."""
    import ctypes as C
    L = inla.lib()
    P = C.POINTER(C.c_double)
    L.inla_test_cov_df.argtypes = [P, C.c_int32, C.c_double, C.c_double, C.c_double, P]
    rng = np.random.default_rng(77)
    n = 700
    pts = rng.uniform(0, 1, size=(n, 2))
    pts[:5] = pts[5]            # coincident points (d = 0)
    for sigma2, irx, iry in [(1.0, 5.0, 5.0), (2.7, 28.0, 3.0), (0.05, 1.0, 40.0)]:
        out = np.empty((n, n))
        rc = L.inla_test_cov_df(pts.ctypes.data_as(P), n, sigma2, irx, iry, out.ctypes.data_as(P))
        assert rc == 0
        dx = (pts[:, None, 0] - pts[None, :, 0]) * irx
        dy = (pts[:, None, 1] - pts[None, :, 1]) * iry
        d = np.sqrt(dx * dx + dy * dy)
        ref = sigma2 * np.exp(-d)
        err = np.abs(out - ref)
        assert np.max(err / ref / (1.0 + d)) < 6e-14, np.max(err / ref / (1.0 + d))
        assert np.max(err) / sigma2 < 6e-14, np.max(err) / sigma2


def test_newton_trace_refactors_early_and_reuses_near_the_mode():
    """The mixed Newton iteration starts from a weighted least-squares solution (its factor is
    the trace's first entry) and reuses a factor while the steps shrink fast (modified Newton:
    the gradient is exact, so the fixed point is the mode); the FP64 path runs Algorithm 1 from
    x = 0 and refactors every iteration.  Both reach the step tolerance."""
    import ctypes as C
    L = inla.lib()
    L.inla_test_newton_trace.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_int32]
    spec, thetas = synth.poisson_n256_m1000_5pts()
    model = inla.Model(spec)
    for prec in ("mixed", "fp64"):
        inla.eval_batch([model], thetas, want_x=False, want_var=False, precision=prec)
        steps = np.zeros(64)
        ref = np.zeros(64, dtype=np.int32)
        n = L.inla_test_newton_trace(steps.ctypes.data_as(C.POINTER(C.c_double)),
                                     ref.ctypes.data_as(C.POINTER(C.c_int32)), 64)
        assert 2 <= n <= 50
        assert ref[0] == 1
        assert steps[n - 1] <= 1e-8
        if prec == "fp64":
            assert np.all(ref[:n] == 1)
        else:
            assert ref[n - 1] == 0       # the last iterations reuse the factor
            assert np.sum(ref[:n]) <= n // 2  # at most every other iteration factors afresh


def _check_vs_fp64(lp, st, xs, vs, ref, names):
    lp64, st64, xs64, vs64 = ref
    for b in range(len(lp)):
        assert st[b] == 0 and st64[b] == 0, (names[b], inla.status_string(st[b]), inla.status_string(st64[b]))
        e_lp = abs(lp[b] - lp64[b])
        e_x = np.max(np.abs(xs[b] - xs64[b])) / max(1.0, np.max(np.abs(xs64[b])))
        e_v = np.max(np.abs(vs[b] / vs64[b] - 1))
        assert e_lp <= LP_ABS, (names[b], e_lp)
        assert e_x <= X_RTOL, (names[b], e_x)
        assert e_v <= V_RTOL, (names[b], e_v)


@pytest.mark.slow
def test_mixed_spacetime_full_size_against_fp64_path():
    """The constrained space-time model at full size (n = 8149, k = 1486 sum-to-zero
    constraints, six log precisions): two FD points, mixed against FP64 on the GPU."""
    spec, thetas = synth.spacetime_n8149_m8000_fd13()
    sub = thetas[[0, 7]]
    m = inla.Model(spec)
    mixed = inla.eval_batch([m], sub, precision="mixed")
    fp64 = inla.eval_batch([m], sub, precision="fp64")
    _check_vs_fp64(*mixed, fp64, ["fd0", "fd7"])
    C = spec.C.to_dense()
    for x in mixed[2]:
        assert np.max(np.abs(C @ x)) < 1e-6


@pytest.mark.slow
def test_mixed_64_uneven_models_against_fp64_path():
    """All 64 Gaussian models of uneven size (n in {512, 1024, 2048, 4096}) in one batch call,
    each at its own theta: mixed against FP64 on the GPU, model by model."""
    specs, thetas = synth.gaussian_64_models_n512_4096()
    ms = [inla.Model(sp) for sp in specs]
    which = np.arange(len(specs), dtype=np.int32)
    mixed = inla.eval_batch(ms, thetas, model_of_theta=which, precision="mixed")
    fp64 = inla.eval_batch(ms, thetas, model_of_theta=which, precision="fp64")
    _check_vs_fp64(*mixed, fp64, [sp.name for sp in specs])


def test_outer_block_tuner_decides_and_results_agree():
    """The mixed Cholesky times its two outer-block candidates (256, 512) on the first two real
    factorisations of a size and keeps the faster, and so does the transposed inverse; every
    result along the way (both candidates and the tuned choice) stays within the mixed
    tolerances of the oracle."""
    import ctypes as C
    L = inla.lib()
    spec = synth.spatial_poisson("tune_n1500", synth.SEED_BASE + 71, 1499, 4000, [0.0, np.log(0.2)])
    thetas = np.array([[0.0, np.log(0.2)], [0.3, np.log(0.15)]])
    m = inla.Model(spec)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed")
    _check(spec, thetas, lp, st, xs, vs)
    lp2, st2, xs2, vs2 = inla.eval_batch([m], thetas, precision="mixed")
    _check(spec, thetas, lp2, st2, xs2, vs2)
    n_pad = 1536
    assert L.inla_test_outer_block(n_pad, 4) in (256, 512)
    assert L.inla_test_outer_block(n_pad, 5) in (256, 512)
    # the transposed inverse (prior covariance, then the variances) is tuned the same way
    assert L.inla_test_inverse_block(n_pad, 5) in (256, 512)



def _gemm_flops(run):
    """Algorithmic flops of every tensor-core GEMM launched by run() (library statistics)."""
    import ctypes as C
    L = inla.lib()
    L.inla_test_stats_read.argtypes = [C.POINTER(C.c_double)]
    st = (C.c_double * 5)()
    L.inla_test_stats_read(st)
    L.inla_test_stats_enable(1)
    try:
        res = run()
    finally:
        L.inla_test_stats_enable(0)
    L.inla_test_stats_read(st)
    return res, st[1]


def test_fd_batch_followers_start_from_the_centre_mode():
    """A 5-point central FD stencil on one Poisson model: the centre runs Newton from 0, the
    four other points start from its mode with its final factor.  Every point still matches the
    oracle at the mixed tolerances, and the batch needs fewer Newton factorisations than with
    every point on its own (INLA_OPT_NO_SHARED_START)."""
    spec = synth.spatial_poisson("fd_n1024", synth.SEED_BASE + 81, 1023, 4000, [0.0, np.log(0.2)])
    thetas = synth._fd_batch(np.array([0.1, np.log(0.25)]))
    m = inla.Model(spec)
    (lp, st, xs, vs), f_shared = _gemm_flops(lambda: inla.eval_batch([m], thetas, precision="mixed"))
    _check(spec, thetas, lp, st, xs, vs)
    (lp0, st0, xs0, vs0), f_own = _gemm_flops(
        lambda: inla.eval_batch([m], thetas, precision="mixed", flags_extra=inla.OPT_NO_SHARED_START))
    _check(spec, thetas, lp0, st0, xs0, vs0)
    n3 = float(spec.n) ** 3
    print(f"GEMM algorithmic flops per point: shared start {f_shared / 5 / n3:.2f} n^3, own {f_own / 5 / n3:.2f} n^3")
    assert f_shared < 0.8 * f_own
    # both routes converge to the same modes (step tolerance 1e-8)
    for b in range(len(thetas)):
        assert np.max(np.abs(xs[b] - xs0[b])) <= 1e-6 * max(1.0, np.max(np.abs(xs0[b])))


def test_precision_autotuner_choice_meets_the_targets_against_the_oracle():
    """The autotuner calibrates on the model against its own six-slice evaluation (no oracle);
    its choice must hold the targets against the oracle on every point of the workload, and
    (at n = 256, where fewer bits suffice) cost no more GEMM passes than the default 5/5/4."""
    from paper_2311_08050_gb300 import tune
    spec, thetas = synth.poisson_n256_m1000_5pts()
    m = inla.Model(spec)
    tr = tune.tune_precision(m, thetas[0])
    print("tuned", tr.opts(), tr.errors, [t["setting"] for t in tr.tried])
    assert (tr.prior_slices, tr.gram_slices, tr.slices, tr.newton_slices, tr.var_slices) in tune.CANDIDATES
    passes = lambda S: S * (S + 1) // 2
    assert passes(tr.prior_slices) + passes(tr.slices) <= passes(5) + passes(5)
    lp, st, xs, vs = inla.eval_batch([m], thetas, precision="mixed", **tr.opts())
    _check(spec, thetas, lp, st, xs, vs)

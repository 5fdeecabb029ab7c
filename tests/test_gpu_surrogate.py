"""The learned surrogate on the GPU: its kernels against the FP64 reference network
(gradients, input gradients, one Adam step), training convergence, and what the trained
network gains over the search without it, on exact evaluations of a model of the n = 16384
benchmark's family (anisotropic exponential covariance + folded iid, theta of dimension 4)
at n = 256.  The gain is counted in sequential exact calls after training (each call is one
batched evaluation on the GPU); the training set itself is one batch of 2000 exact points
(a few calls), and the integration points are ranked by the trained network."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla, surrogate, synth

pytestmark = pytest.mark.gpu
H = surrogate.HIDDEN


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def _data(N=300, D=4, seed=11):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, D)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - 0.3 * X[:, 3] ** 2).astype(np.float32)
    return X, y


def test_loss_gradient_matches_fp64_backprop():
    X, y = _data()
    p = surrogate.init_params(4, 5)
    net = surrogate.MLP(4, 1024)
    net.set_params(p)
    loss, g = net.loss_grad(X, y)
    lref, gref = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64), 4, H)
    assert abs(loss - lref) <= 1e-5 * abs(lref)
    # FP32 sums over 300 samples: bound the error by the gradient's scale per block
    assert np.linalg.norm(g - gref) <= 2e-5 * np.linalg.norm(gref)
    assert np.max(np.abs(g - gref)) <= 1e-5 * np.max(np.abs(gref)) + 1e-7


def test_forward_and_input_gradient_match_fp64():
    X, _ = _data(N=257)
    p = surrogate.init_params(4, 6)
    net = surrogate.MLP(4, 512)
    net.set_params(p)
    f, dfdx = net.predict(X, want_grad=True)
    fref = M.forward(p.astype(np.float64), X.astype(np.float64), 4, H)[0]
    gref = M.input_grad(p.astype(np.float64), X.astype(np.float64), 4, H)
    np.testing.assert_allclose(f, fref, rtol=0, atol=1e-5 * np.max(np.abs(fref)) + 1e-6)
    np.testing.assert_allclose(dfdx, gref, rtol=0, atol=1e-5 * np.max(np.abs(gref)) + 1e-6)


def test_one_adam_step_matches_definition():
    X, y = _data()
    p = surrogate.init_params(4, 7)
    net = surrogate.MLP(4, 1024)
    net.set_params(p)
    hist = net.train(X, y, 1, 1e-3)
    p1 = net.get_params().astype(np.float64)
    l0, g0 = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64), 4, H)
    pref, _, _ = M.adam_step(p.astype(np.float64), g0, np.zeros_like(g0), np.zeros_like(g0), 1, 1e-3)
    assert abs(hist[0] - l0) <= 1e-5 * l0
    # first Adam step moves every parameter by ~lr * sign(g): compare the moves
    np.testing.assert_allclose(p1 - p, pref - p, rtol=0, atol=2e-6)


def test_training_fits_a_smooth_function():
    X, y = _data(N=2000)
    net = surrogate.MLP(4, 2048)
    net.set_params(surrogate.init_params(4, 8))
    ys = (y - y.mean()) / y.std()
    hist = net.train(X, ys, 1500, 3e-3)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.01 * hist[0]
    Xt, yt = _data(N=500, seed=12)
    pred = net.predict(Xt) * y.std() + y.mean()
    assert np.sqrt(np.mean((pred - yt) ** 2)) < 0.05 * np.std(yt) + 0.02


def _workload():
    th = np.array([0.0, np.log(0.2), np.log(0.1), np.log(4.0)])
    spec = synth.spatial_poisson("poisson_n256_m1000_aniso", synth.SEED_BASE + 55, 255, 1000, th,
                                 anisotropic=True, folded_iid=True)
    return spec, th


def test_surrogate_search_gains_over_exact_search():
    spec, th_true = _workload()
    model = inla.Model(spec)

    def exact_eval(thetas):
        out = []
        for c in range(0, len(thetas), 512):
            lp, st, _, _ = inla.eval_batch([model], thetas[c:c + 512], want_x=False, want_var=False,
                                           precision="mixed")
            lp = np.where(np.asarray(st) == 0, lp, -np.inf)
            out.append(lp)
        return np.concatenate(out)

    rng = np.random.default_rng(synth.SEED_BASE + 56)
    T = th_true + 0.5 * rng.standard_normal((2000, 4))
    train = surrogate.ExactCounter(exact_eval)
    vals = train(T)
    assert np.isfinite(vals).mean() > 0.99
    sur = surrogate.Surrogate(4).fit(T, vals, epochs=1500, lr=3e-3)
    # held-out accuracy of the surrogate over the training distribution
    Th = th_true + 0.5 * rng.standard_normal((300, 4))
    vh = exact_eval(Th)
    ok = np.isfinite(vh)
    r2 = 1.0 - np.mean((sur.predict(Th[ok]) - vh[ok]) ** 2) / np.var(vh[ok])
    assert r2 > 0.99, r2

    th0 = th_true + np.array([0.6, -0.5, 0.4, -0.6])
    base = surrogate.ExactCounter(exact_eval)
    xb, fb, _, _ = surrogate.search_exact(base, th0)
    guided = surrogate.ExactCounter(exact_eval)
    xs, fs, calls = surrogate.search_with_surrogate(guided, sur, th0)
    print(f"exact search: {base.calls} sequential calls, {base.points} points, log pi~ {fb:.6f}; "
          f"surrogate-guided: {guided.calls} calls, {guided.points} points, log pi~ {fs:.6f} "
          f"(after {train.calls} training batches of {train.points} points); held-out R^2 {r2:.5f}")
    # the surrogate-guided search reaches the same optimum (exactly evaluated) ...
    assert fs >= fb - 1e-3
    assert np.max(np.abs(xs - xb)) < 0.05
    # ... with at most half the sequential exact calls of the search without it
    assert guided.calls * 2 <= base.calls

    # integration points: the CCD design in the coordinates of the Laplace approximation of
    # the hyperparameter posterior (exact FD Hessian at the mode: one batch); a surrogate fit
    # on one batch of 400 exact points drawn from that approximation predicts and ranks the
    # design, and one exact batch checks it
    negH = -surrogate.fd_hessian(guided, xs)
    cov = np.linalg.inv(negH)
    local = rng.multivariate_normal(xs, cov, 400)
    local_v = exact_eval(local)
    sur_local = surrogate.Surrogate(4).fit(local, local_v, epochs=1500, lr=3e-3)
    pts, pred = surrogate.rank_ccd(sur_local, xs, negH)
    ex = exact_eval(pts)
    assert np.all(np.isfinite(ex))
    spread = ex.max() - ex.min()
    err = np.max(np.abs(pred - ex))
    print(f"CCD: {len(pts)} points, exact log pi~ spread {spread:.4f}, surrogate max error {err:.4f}")
    assert err <= 0.1 * spread
    assert np.argmax(ex) in np.argsort(-pred)[:3]

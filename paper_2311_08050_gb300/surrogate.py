"""Learned surrogate of log pi~(theta|y) and the hyperparameter search that uses it.

The network and its training run in libinla (include/inla_surrogate.h: forward,
backpropagation and Adam kernels; the epoch is a CUDA graph); this module marshals arrays,
standardises inputs and targets, and drives the search on the host:

* ``Surrogate`` -- fit on exact evaluations (theta, log pi~), predict values and gradients.
* ``bfgs_maximize`` -- BFGS with a backtracking (Armijo) line search, used on the surrogate
  (cheap) and, for the method without the surrogate, on the exact function with
  finite-difference gradients (the paper's FD batch of 2t + 1 points per gradient).
* ``search_with_surrogate`` -- the surrogate proposes a maximiser and its Hessian; the exact
  batched evaluation decides (the proposal is kept only if its exact log pi~ improves) and
  exact FD-BFGS, warm-started with the surrogate's Hessian, finishes the search.
* ``ccd_design`` / ``rank_ccd`` -- central composite design points around the mode in the
  coordinates of the Laplace approximation of the hyperparameter posterior (exact FD Hessian,
  one batch), predicted and ranked by a surrogate, then evaluated exactly.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import inla

HIDDEN = 128
_P = C.POINTER
_f32 = C.c_float


def _lib():
    L = inla.lib()
    if not getattr(L, "_mlp_ready", False):
        L.inla_mlp_num_params.argtypes = [C.c_int32]
        L.inla_mlp_num_params.restype = C.c_int64
        L.inla_mlp_create.argtypes = [C.c_int32, C.c_int32, _P(C.c_void_p)]
        L.inla_mlp_destroy.argtypes = [C.c_void_p]
        L.inla_mlp_set_params.argtypes = [C.c_void_p, _P(_f32)]
        L.inla_mlp_get_params.argtypes = [C.c_void_p, _P(_f32)]
        L.inla_mlp_train.argtypes = [C.c_void_p, _P(_f32), _P(_f32), C.c_int32, C.c_int32, _f32, _P(_f32)]
        L.inla_mlp_loss_grad.argtypes = [C.c_void_p, _P(_f32), _P(_f32), C.c_int32, _P(_f32), _P(_f32)]
        L.inla_mlp_predict.argtypes = [C.c_void_p, _P(_f32), C.c_int32, _P(_f32), _P(_f32)]
        L._mlp_ready = True
    return L


def _fp(a):
    return a.ctypes.data_as(_P(_f32)) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise inla.InlaError(rc, what)


class MLP:
    """The device network (wraps inla_mlp*): din inputs, 128 hidden units, one output."""

    def __init__(self, din: int, max_samples: int):
        self.din = int(din)
        self.max_samples = int(max_samples)
        self.np = int(_lib().inla_mlp_num_params(self.din))
        h = C.c_void_p()
        _check(_lib().inla_mlp_create(self.din, self.max_samples, C.byref(h)), "inla_mlp_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib().inla_mlp_destroy(h)
            self._h = None

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.shape == (self.np,)
        _check(_lib().inla_mlp_set_params(self._h, _fp(p)), "inla_mlp_set_params")

    def get_params(self):
        p = np.empty(self.np, dtype=np.float32)
        _check(_lib().inla_mlp_get_params(self._h, _fp(p)), "inla_mlp_get_params")
        return p

    def train(self, X, y, epochs, lr):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        hist = np.empty(max(int(epochs), 1), dtype=np.float32)
        _check(_lib().inla_mlp_train(self._h, _fp(X), _fp(y), len(y), int(epochs), float(lr), _fp(hist)),
               "inla_mlp_train")
        return hist[:epochs]

    def loss_grad(self, X, y):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.np, dtype=np.float32)
        _check(_lib().inla_mlp_loss_grad(self._h, _fp(X), _fp(y), len(y), _fp(loss), _fp(g)), "inla_mlp_loss_grad")
        return float(loss[0]), g

    def predict(self, X, want_grad=False):
        X = np.ascontiguousarray(X, dtype=np.float32)
        f = np.empty(len(X), dtype=np.float32)
        g = np.empty((len(X), self.din), dtype=np.float32) if want_grad else None
        _check(_lib().inla_mlp_predict(self._h, _fp(X), len(X), _fp(f), _fp(g)), "inla_mlp_predict")
        return (f, g) if want_grad else f


def init_params(din: int, seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases, packed in the library's order."""
    rng = np.random.default_rng(seed)
    H = HIDDEN

    def glorot(fan_in, fan_out, size):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-a, a, size)

    return np.concatenate([glorot(din, H, H * din), np.zeros(H), glorot(H, H, H * H), np.zeros(H),
                           glorot(H, 1, H), np.zeros(1)]).astype(np.float32)


class Surrogate:
    """log pi~(theta|y) ~= s_y f((theta - m_x) / s_x) + m_y, f the device MLP."""

    def __init__(self, dim: int, max_samples: int = 8192, seed: int = 2311080511):
        self.dim = dim
        self.net = MLP(dim, max_samples)
        self.seed = seed
        self.net.set_params(init_params(dim, seed))
        self.loss_history = np.zeros(0, dtype=np.float32)

    def fit(self, thetas, logpost, epochs=1500, lr=3e-3, reset=True):
        thetas = np.asarray(thetas, dtype=np.float64)
        logpost = np.asarray(logpost, dtype=np.float64)
        ok = np.isfinite(logpost)
        thetas, logpost = thetas[ok], logpost[ok]
        self.mx = thetas.mean(axis=0)
        self.sx = thetas.std(axis=0) + 1e-12
        self.my = logpost.mean()
        self.sy = logpost.std() + 1e-12
        if reset:
            self.net.set_params(init_params(self.dim, self.seed))
        X = (thetas - self.mx) / self.sx
        y = (logpost - self.my) / self.sy
        self.loss_history = self.net.train(X, y, epochs, lr)
        return self

    def predict(self, thetas, want_grad=False):
        thetas = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        X = (thetas - self.mx) / self.sx
        if not want_grad:
            return self.net.predict(X).astype(np.float64) * self.sy + self.my
        f, g = self.net.predict(X, want_grad=True)
        return f.astype(np.float64) * self.sy + self.my, g.astype(np.float64) * (self.sy / self.sx)[None, :]

    def hessian(self, theta, h=1e-3):
        """Central differences of the surrogate's gradient (t x t, symmetrised)."""
        t = self.dim
        pts = np.array([theta + s * h * np.eye(t)[i] for i in range(t) for s in (1.0, -1.0)])
        _, g = self.predict(pts, want_grad=True)
        Hm = np.array([(g[2 * i] - g[2 * i + 1]) / (2 * h) for i in range(t)])
        return 0.5 * (Hm + Hm.T)


def bfgs_maximize(fg: Callable[[np.ndarray], tuple[float, np.ndarray]], x0, max_iter=100, gtol=1e-6, xtol=1e-8,
                  max_step=1.0, hinv0=None, fg0=None):
    """Maximise f by BFGS on -f with an Armijo backtracking line search.  fg(x) -> (f, grad).
    hinv0: initial inverse Hessian of -f (default identity); fg0: (f, grad) at x0 if known.
    Returns (x, f, iterations, function evaluations)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    if fg0 is None:
        f, g = fg(x)
        nfev = 1
    else:
        f, g = fg0
        nfev = 0
    Hinv = np.eye(len(x)) if hinv0 is None else np.array(hinv0, dtype=np.float64)
    it = 0
    for it in range(1, max_iter + 1):
        if np.linalg.norm(g, np.inf) < gtol:
            break
        d = Hinv @ g                      # ascent direction
        nd = np.linalg.norm(d)
        if nd > max_step:
            d *= max_step / nd
        a, accepted = 1.0, False
        for _ in range(30):
            xn = x + a * d
            fn, gn = fg(xn)
            nfev += 1
            if np.isfinite(fn) and fn >= f + 1e-4 * a * g @ d:
                accepted = True
                break
            a *= 0.5
        if not accepted:
            break
        s, yv = xn - x, -(gn - g)          # secant pair of -f
        x, f, g = xn, fn, gn
        sy = s @ yv
        if sy > 1e-12:
            rho = 1.0 / sy
            I = np.eye(len(x))
            Hinv = (I - rho * np.outer(s, yv)) @ Hinv @ (I - rho * np.outer(yv, s)) + rho * np.outer(s, s)
        if np.linalg.norm(s, np.inf) < xtol:
            break
    return x, f, it, nfev


@dataclass
class ExactCounter:
    """Wraps the exact batched evaluation theta (B x t) -> log pi~ (B), counting points and
    sequential calls (each call is one batched launch sequence on the GPU)."""
    evaluate: Callable[[np.ndarray], np.ndarray]
    points: int = 0
    calls: int = 0
    log: list = field(default_factory=list)

    def __call__(self, thetas):
        thetas = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        v = np.asarray(self.evaluate(thetas), dtype=np.float64)
        self.points += len(thetas)
        self.calls += 1
        self.log.append((thetas.copy(), v.copy()))
        return v


def fd_value_grad(exact: ExactCounter, theta, h=1e-3):
    """log pi~ and its central-difference gradient from one batch of 2t + 1 exact points."""
    t = len(theta)
    pts = [theta] + [theta + s * h * np.eye(t)[i] for i in range(t) for s in (1.0, -1.0)]
    v = exact(np.array(pts))
    g = np.array([(v[1 + 2 * i] - v[2 + 2 * i]) / (2 * h) for i in range(t)])
    return float(v[0]), g


def search_exact(exact: ExactCounter, theta0, gtol=1e-3, max_iter=100, h=1e-3):
    """The method without the surrogate: BFGS on exact values with FD gradients."""
    return bfgs_maximize(lambda th: fd_value_grad(exact, th, h), theta0, max_iter=max_iter, gtol=gtol)


def surrogate_hinv(surrogate: Surrogate, theta, floor=1e-6):
    """Inverse of the surrogate's negative Hessian at theta, eigenvalues floored (a positive
    definite initial inverse Hessian for BFGS on -log pi~)."""
    lam, V = np.linalg.eigh(-surrogate.hessian(theta))
    lam = np.maximum(lam, floor * max(1.0, float(np.max(np.abs(lam)))))
    return (V / lam[None, :]) @ V.T


def search_with_surrogate(exact: ExactCounter, surrogate: Surrogate, theta0, gtol=1e-3, max_iter=100, h=1e-3):
    """Surrogate proposal, exact decision, exact polish.

    1. Maximise the surrogate from theta0 (no exact evaluation).
    2. One exact batch: theta0 and the FD stencil (2t + 1 points) around the proposal.  The
       proposal is accepted if its exact log pi~ beats theta0's; otherwise the search starts
       from theta0 (its gradient costs one more batch).
    3. Exact BFGS with FD gradients from there, its initial inverse Hessian taken from the
       surrogate (the exact evaluation still decides every step).
    Returns (theta, exact log pi~, sequential exact calls of the search)."""
    th0 = np.asarray(theta0, dtype=np.float64)
    t = len(th0)
    calls0 = exact.calls
    prop, _, _, _ = bfgs_maximize(lambda x: (float(surrogate.predict(x)[0]), surrogate.predict(x, want_grad=True)[1][0]),
                                  th0, max_iter=300, gtol=1e-8)
    stencil = [prop] + [prop + sg * h * np.eye(t)[i] for i in range(t) for sg in (1.0, -1.0)]
    v = exact(np.array([th0] + stencil))
    f0, fp = float(v[0]), float(v[1])
    if np.isfinite(fp) and fp > f0:
        start = prop
        g = np.array([(v[2 + 2 * i] - v[3 + 2 * i]) / (2 * h) for i in range(t)])
        fg0 = (fp, g)
    else:
        start = th0
        fg0 = fd_value_grad(exact, th0, h)
    x, f, _, _ = bfgs_maximize(lambda th: fd_value_grad(exact, th, h), start, max_iter=max_iter, gtol=gtol,
                               hinv0=surrogate_hinv(surrogate, start), fg0=fg0)
    return x, f, exact.calls - calls0


def ccd_design(t: int) -> np.ndarray:
    """Central composite design (Box & Wilson, 1951) in standardised coordinates: the centre,
    the 2^t corners (+-1)^t and the 2t axial points at +-(2^t)^(1/4) (rotatable design)."""
    corners = np.array(np.meshgrid(*[[-1.0, 1.0]] * t, indexing="ij")).reshape(t, -1).T
    alpha = (2.0 ** t) ** 0.25
    axial = np.concatenate([alpha * np.eye(t), -alpha * np.eye(t)])
    return np.concatenate([np.zeros((1, t)), corners, axial])


def fd_hessian(exact: ExactCounter, theta, h=2e-2):
    """Central-difference Hessian of log pi~ from one exact batch of 2t^2 + 1 points."""
    theta = np.asarray(theta, dtype=np.float64)
    t = len(theta)
    E = np.eye(t) * h
    pts = [theta]
    for i in range(t):
        pts += [theta + E[i], theta - E[i]]
    for i in range(t):
        for j in range(i + 1, t):
            pts += [theta + E[i] + E[j], theta + E[i] - E[j], theta - E[i] + E[j], theta - E[i] - E[j]]
    v = exact(np.array(pts))
    f0 = v[0]
    Hm = np.zeros((t, t))
    for i in range(t):
        Hm[i, i] = (v[1 + 2 * i] - 2 * f0 + v[2 + 2 * i]) / (h * h)
    k = 1 + 2 * t
    for i in range(t):
        for j in range(i + 1, t):
            Hm[i, j] = Hm[j, i] = (v[k] - v[k + 1] - v[k + 2] + v[k + 3]) / (4 * h * h)
            k += 4
    return Hm


def ccd_points(theta_star, neg_hessian):
    """CCD design around theta* in the coordinates of the Laplace approximation of the
    hyperparameter posterior: theta = theta* + V Lambda^-1/2 z, (V, Lambda) the eigenpairs of
    the negative Hessian of log pi~ at theta* (so z ~ N(0, I) under that approximation)."""
    lam, V = np.linalg.eigh(np.asarray(neg_hessian, dtype=np.float64))
    if np.min(lam) <= 0:
        raise ValueError("the negative Hessian is not positive definite at theta*")
    Z = ccd_design(len(theta_star))
    return np.asarray(theta_star)[None, :] + (Z / np.sqrt(lam)[None, :]) @ V.T


def rank_ccd(surrogate: Surrogate, theta_star, neg_hessian):
    """The CCD points ordered by the surrogate's log pi~ (best first): (points, predictions)."""
    pts = ccd_points(theta_star, neg_hessian)
    pred = surrogate.predict(pts)
    order = np.argsort(-pred)
    return pts[order], pred[order]


def experiment(exact_eval: Callable[[np.ndarray], np.ndarray], th_true, th0, n_train=2000, n_holdout=200,
               spread=0.5, seed=2311080556, epochs=1500, lr=3e-3, gtol=1e-3, clock=None):
    """The learned-surrogate experiment with every exact evaluation counted.

    exact_eval: theta (B x t) -> exact log pi~ (B), one batched evaluation per call.
    1. The method without the surrogate: exact FD-BFGS from th0 (`search_exact`).
    2. The surrogate: n_train exact evaluations at theta ~ N(th_true, spread^2 I), a fit, its
       error on n_holdout further exact points (not counted in the search), then the
       surrogate-guided search from th0 (`search_with_surrogate`).
    3. Integration points: the CCD design around the guided search's mode in the coordinates
       of the Laplace approximation of the hyperparameter posterior (exact FD Hessian), ranked
       by the surrogate and checked by one exact batch.
    Wall times by `clock` (default time.perf_counter); returns a dict of counts, times and
    errors, including the totals with the training evaluations charged to the guided search
    and the number of searches over which the training pays off (None if it never does)."""
    import time
    clock = clock or time.perf_counter
    rng = np.random.default_rng(seed)
    th_true = np.asarray(th_true, dtype=np.float64)
    t = len(th_true)
    out = {}
    # 1. exact search
    base = ExactCounter(exact_eval)
    c0 = clock()
    xb, fb, itb, _ = search_exact(base, th0, gtol=gtol)
    out["exact_search"] = {"calls": base.calls, "points": base.points, "seconds": clock() - c0,
                           "bfgs_iterations": itb, "theta": xb.tolist(), "log_post": fb}
    # 2. training set, fit, held-out error
    T = th_true + spread * rng.standard_normal((n_train, t))
    train = ExactCounter(exact_eval)
    c0 = clock()
    vals = train(T)
    t_train = clock() - c0
    ok = np.isfinite(vals)
    c0 = clock()
    sur = Surrogate(t, max_samples=max(8192, n_train)).fit(T[ok], vals[ok], epochs=epochs, lr=lr)
    t_fit = clock() - c0
    Th = th_true + spread * rng.standard_normal((n_holdout, t))
    vh = exact_eval(Th)
    okh = np.isfinite(vh)
    pred = sur.predict(Th[okh])
    res = pred - vh[okh]
    out["training"] = {"points": train.points, "calls": train.calls, "finite": int(ok.sum()), "seconds": t_train,
                       "theta_evals_per_s": train.points / t_train if t_train > 0 else None,
                       "fit_seconds": t_fit, "epochs": epochs, "final_loss": float(sur.loss_history[-1])}
    out["holdout"] = {"points": int(okh.sum()), "rmse": float(np.sqrt(np.mean(res ** 2))),
                      "max_abs": float(np.max(np.abs(res))), "r2": float(1.0 - np.mean(res ** 2) / np.var(vh[okh])),
                      "log_post_spread": float(np.ptp(vh[okh]))}
    # near the mode the accuracy that matters for the proposals
    # 3. guided search
    guided = ExactCounter(exact_eval)
    c0 = clock()
    xs, fs, calls = search_with_surrogate(guided, sur, th0, gtol=gtol)
    t_guided = clock() - c0
    out["guided_search"] = {"calls": calls, "points": guided.points, "seconds": t_guided, "theta": xs.tolist(),
                            "log_post": fs, "same_mode": bool(np.max(np.abs(xs - xb)) < 0.05 and fs >= fb - 1e-3)}
    tot_points = train.points + guided.points
    tot_time = t_train + t_fit + t_guided
    out["totals"] = {"exact_points_with_training": tot_points, "exact_points_without_surrogate": base.points,
                     "time_to_mode_with_training_s": tot_time,
                     "time_to_mode_without_surrogate_s": out["exact_search"]["seconds"]}
    saving = out["exact_search"]["seconds"] - t_guided
    out["totals"]["searches_to_break_even"] = (t_train + t_fit) / saving if saving > 0 else None
    # 4. CCD integration points ranked by the surrogate, one exact batch decides
    negH = -fd_hessian(guided, xs)
    try:
        pts, predc = rank_ccd(sur, xs, negH)
        ex = exact_eval(pts)
        okc = np.isfinite(ex)
        out["ccd"] = {"points": len(pts), "exact_spread": float(np.ptp(ex[okc])),
                      "max_abs_error": float(np.max(np.abs(predc[okc] - ex[okc]))),
                      "best_in_surrogate_top3": bool(np.argmax(np.where(okc, ex, -np.inf)) in np.argsort(-predc)[:3])}
    except ValueError as e:
        out["ccd"] = {"error": str(e)}
    return out

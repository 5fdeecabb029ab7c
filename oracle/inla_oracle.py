"""FP64 CPU oracle for one evaluation of the dense INLA theta-level quantities.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product path (the CUDA
library and its Python binding) never calls it and shares no code with it; the two
read the same seeded ``ModelSpec`` from ``paper_2311_08050_gb300.synth`` and nothing
else.

What it computes, per hyperparameter point theta (plain definitions, numpy/scipy FP64,
no blocking or fusion of our own):

* the prior precision Q_p(theta) of the latent field (Section 1, LGM statement; dense
  covariance blocks are inverted, structured blocks are tau * R (+ eps I), Section 5.1),
* the conditional mode x_hat by the Gaussian-approximation Newton iteration
  (Appendix A.2.1, Algorithm 1: Q* = Q_x + Q_l(x0), b = grad g + Q_l x0, solve),
  with linear constraints C x = 0 imposed after every solve by conditioning by
  kriging (Section 5.2; the Gaussian conditioning identity of Appendix C),
* the Laplace approximation log pi~(theta | y) of Eq. (41), written out with all
  normalising constants (see ``evaluate``), and
* the Gaussian marginals x_i | theta, y ~ N(x_hat_i, (Q*^-1)_ii) (Appendix A.2.1),
  corrected for the constraints by kriging, and
* stage 2: the Hessian of log pi~ at theta*, the CCD / grid exploration points and the
  latent marginals integrated over them (Section 2, Stage 2; Appendix A.2), and
* the variational Bayes correction of the posterior mean (Appendix A.2.2, Algorithm 2), and
* the Moore-Penrose / Woodbury covariance route of Section 3.1, Eq. (woodeqn)
  (readings of these at the end of this file).

Readings of the paper taken here (the paper is silent or garbled on these):
  Newton tolerance 1e-8 in the infinity norm, at most 50 iterations, step halving
  (at most 30 halvings) when the objective decreases; a Gaussian likelihood takes one
  Newton solve (Section 4: "1 Cholesky in case of Gaussian likelihood"); the factor is
  always recomputed at x_hat; the marginal variance is (Q*^-1)_ii; eps is added to the
  intrinsic blocks (so also to Q*); PC prior on log precisions; N(0, 1) on log sigma and
  log range.

Parity pins: every function here is checked in tests/test_oracle_pins.py against
something other than itself (closed forms, the paper's worked example of Appendix C,
brute force on tiny inputs, an independent optimiser).
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.special import gammaln

def chol(M):
    """Lower Cholesky factor (LAPACK dpotrf through scipy)."""
    return sla.cholesky(M, lower=True, check_finite=False)


def spd_inverse(L):
    """(L L^T)^-1 from a lower Cholesky factor (LAPACK dpotri), symmetrised."""
    inv, info = sla.lapack.dpotri(L, lower=1)
    if info != 0:
        raise np.linalg.LinAlgError(f"dpotri info={info}")
    return np.tril(inv) + np.tril(inv, -1).T


NEWTON_TOL = 1e-8
NEWTON_MAX = 50
HALVING_MAX = 30
HALVING_RTOL = 1e-10   # a decrease smaller than this (relative) is rounding, not divergence


# ------------------------------------------------------------------------------------
# hyperparameter prior  (PC prior for precisions, Section 5.1 / Section 6; N(0,1) else)
# ------------------------------------------------------------------------------------

def log_theta_prior(spec, theta) -> float:
    """log pi(theta) = sum of independent component priors.

    ("gauss", mu, sd): N(mu, sd^2) on the component.
    ("pc_prec", U, alpha): PC prior of a precision tau with P(1/sqrt(tau) > U) = alpha,
    written for theta = log tau:  log(lam/2) - theta/2 - lam exp(-theta/2),
    lam = -log(alpha)/U.
    """
    lp = 0.0
    for t, (kind, a, b) in enumerate(spec.theta_prior):
        th = float(theta[t])
        if kind == "gauss":
            lp += -0.5 * math.log(2 * math.pi) - math.log(b) - 0.5 * ((th - a) / b) ** 2
        elif kind == "pc_prec":
            lam = -math.log(b) / a
            lp += math.log(lam / 2.0) - th / 2.0 - lam * math.exp(-th / 2.0)
        else:
            raise ValueError(kind)
    return lp


# ------------------------------------------------------------------------------------
# prior precision (Section 1; Section 5.1 structures)
# ------------------------------------------------------------------------------------

def structure_matrix(factor) -> np.ndarray:
    """Fixed structure R of an intrinsic GMRF factor (Section 5.1):
    ICAR (Besag): R = D - W of the neighbourhood graph; RW1 / RW2: R = D^T D with D the
    first / second difference matrix; IID: the identity."""
    if factor.kind == "icar":
        W = factor.graph.to_dense()
        return np.diag(W.sum(axis=1)) - W
    if factor.kind == "rw1":
        D1 = np.diff(np.eye(factor.size), axis=0)
        return D1.T @ D1
    if factor.kind == "rw2":
        D2 = np.diff(np.eye(factor.size), n=2, axis=0)
        return D2.T @ D2
    if factor.kind == "iid":
        return np.eye(factor.size)
    raise ValueError(factor.kind)


def exp_covariance(block, theta) -> np.ndarray:
    """Dense covariance sigma^2 exp(-d) + (1/tau_iid + nugget) I with the scaled
    distance d = sqrt((dx/rho_x)^2 + (dy/rho_y)^2) (exponential / Matern-1/2)."""
    sigma2 = math.exp(2.0 * theta[block.theta_sigma])
    rx = math.exp(theta[block.theta_range_x])
    ry = math.exp(theta[block.theta_range_y])
    p = block.points
    dx = (p[:, None, 0] - p[None, :, 0]) / rx
    dy = (p[:, None, 1] - p[None, :, 1]) / ry
    S = sigma2 * np.exp(-np.sqrt(dx * dx + dy * dy))
    diag_add = block.nugget
    if block.theta_iid >= 0:
        diag_add += math.exp(-theta[block.theta_iid])
    S[np.diag_indices_from(S)] += diag_add
    return S


def prior_precision(spec, theta):
    """Q_p(theta) as a dense n x n matrix and log|Q_p| (block diagonal over the blocks).

    dense_exp blocks: Q_b = Sigma^-1, log|Q_b| = -log|Sigma| (Cholesky of Sigma).
    kron blocks: Q_b = tau (R_1 kron R_2 ...) + eps I, log|Q_b| from its Cholesky.
    """
    n = spec.n
    Qp = np.zeros((n, n))
    logdet = 0.0
    start = 0
    for blk in spec.blocks:
        sl = slice(start, start + blk.size)
        if blk.kind == "fixed":
            Qp[sl, sl] = np.eye(blk.size) * blk.prec
            logdet += blk.size * math.log(blk.prec)
        elif blk.kind == "iid":
            Qp[sl, sl] = np.eye(blk.size) * math.exp(theta[blk.theta_idx])
            logdet += blk.size * theta[blk.theta_idx]
        elif blk.kind == "dense_exp":
            S = exp_covariance(blk, theta)
            L = chol(S)
            Qp[sl, sl] = spd_inverse(L)
            logdet += -2.0 * np.log(np.diag(L)).sum()
        elif blk.kind == "kron":
            R = np.ones((1, 1))
            for f in blk.factors:
                R = np.kron(R, structure_matrix(f))
            Qb = math.exp(theta[blk.theta_idx]) * R + blk.eps * np.eye(blk.size)
            Qp[sl, sl] = Qb
            logdet += 2.0 * np.log(np.diag(chol(Qb))).sum()
        else:
            raise ValueError(blk.kind)
        start += blk.size
    assert start == n
    return Qp, logdet


# ------------------------------------------------------------------------------------
# likelihood (Section 1 / Section 5: Poisson with log link and offset; Gaussian)
# ------------------------------------------------------------------------------------

def _A_sparse(spec):
    A = spec.A
    return sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.nrows, spec.n))


def _offset(spec):
    return np.zeros(spec.m) if spec.offset is None else spec.offset


def log_likelihood(spec, eta) -> float:
    """sum_i log p(y_i | eta_i): Poisson y eta - e^eta - log y!, or Gaussian with
    fixed precision tau: 1/2 log tau - 1/2 log 2 pi - tau/2 (y - eta)^2."""
    y = spec.y
    if spec.likelihood == "poisson":
        return float(np.sum(y * eta - np.exp(eta) - gammaln(y + 1.0)))
    tau = spec.lik_prec
    return float(np.sum(0.5 * math.log(tau) - 0.5 * math.log(2 * math.pi)
                        - 0.5 * tau * (y - eta) ** 2))


def newton_system(spec, As, Qp, x):
    """One step of Algorithm 1 at the current iterate x0 = x:
    Q* = Q_x + Q_l(x0) with Q_l = A^T diag(w) A the negative Hessian of the
    log-likelihood, and b = grad g(x0) + Q_l x0."""
    eta = As @ x + _offset(spec)
    if spec.likelihood == "poisson":
        w = np.exp(eta)
        grad = As.T @ (spec.y - w)
    else:
        w = np.full(spec.m, spec.lik_prec)
        grad = As.T @ (spec.lik_prec * (spec.y - eta))
    Ql = (As.T @ sp.diags(w) @ As).toarray()
    Q = Qp + Ql
    b = grad + Ql @ x
    return Q, b


# ------------------------------------------------------------------------------------
# conditioning by kriging (Section 5.2, Appendix C)
# ------------------------------------------------------------------------------------

def kriging_mean(Q, C, x_u):
    """x = x_u - Q^-1 C^T (C Q^-1 C^T)^-1 C x_u: the mean of N(x_u, Q^-1) given C x = 0."""
    L = chol(Q)
    QiCt = sla.cho_solve((L, True), C.T)
    S = C @ QiCt
    return x_u - QiCt @ np.linalg.solve(S, C @ x_u)


def kriging_covariance(Q, C):
    """Sigma* = Q^-1 - Q^-1 C^T (C Q^-1 C^T)^-1 C Q^-1: the covariance of N(., Q^-1)
    given C x = 0 (the kriging route of Appendix C)."""
    Qi = np.linalg.inv(Q)
    QiCt = Qi @ C.T
    return Qi - QiCt @ np.linalg.solve(C @ QiCt, QiCt.T)


# ------------------------------------------------------------------------------------
# one theta evaluation
# ------------------------------------------------------------------------------------

def _objective(spec, As, Qp, x):
    return log_likelihood(spec, As @ x + _offset(spec)) - 0.5 * float(x @ (Qp @ x))


def find_mode(spec, Qp, As=None, tol=NEWTON_TOL, max_iter=NEWTON_MAX):
    """Algorithm 1 (Gaussian approximation) from x0 = 0, with kriging after each solve
    when constraints are present.  Returns (x_hat, iterations)."""
    As = _A_sparse(spec) if As is None else As
    C = None if spec.C is None else spec.C.to_dense()
    x = np.zeros(spec.n)
    f_old = _objective(spec, As, Qp, x)
    for it in range(1, max_iter + 1):
        Q, b = newton_system(spec, As, Qp, x)
        x_new = sla.cho_solve((chol(Q), True), b)
        if C is not None:
            x_new = kriging_mean(Q, C, x_new)
        if spec.likelihood == "gaussian":
            return x_new, it
        f_new = _objective(spec, As, Qp, x_new)
        h = 0
        while f_new < f_old - HALVING_RTOL * (1.0 + abs(f_old)) and h < HALVING_MAX:
            x_new = x + 0.5 * (x_new - x)
            f_new = _objective(spec, As, Qp, x_new)
            h += 1
        step = float(np.max(np.abs(x_new - x)))
        x, f_old = x_new, f_new
        if step <= tol:
            return x, it
    return x, max_iter


def evaluate(spec, theta, want_var=True):
    """log pi~(theta|y), x_hat and the marginal variances at one theta.

    Eq. (41) evaluated at x_hat, with pi(x | theta) = N(0, Q_p^-1) conditioned on
    C x = 0 and pi~_G = N(x_u, Q*^-1) conditioned on C x = 0:

      log pi~(theta|y) = log pi(theta) + sum_i log p(y_i | eta_hat_i)
                         - 1/2 x_hat^T Q_p x_hat + 1/2 log|Q_p| - 1/2 log|Q*|
                         + 1/2 log|C Q_p^-1 C^T| - 1/2 log|C Q*^-1 C^T|

    (the 2 pi factors cancel; Q* is recomputed at x_hat).  Marginal variances:
    diag(Q*^-1) minus the kriging correction diag(Q*^-1 C^T S^-1 C Q*^-1).
    """
    theta = np.asarray(theta, dtype=np.float64)
    As = _A_sparse(spec)
    Qp, logdet_Qp = prior_precision(spec, theta)
    x_hat, iters = find_mode(spec, Qp, As)
    Q, _ = newton_system(spec, As, Qp, x_hat)
    L = chol(Q)
    logdet_Q = 2.0 * np.log(np.diag(L)).sum()
    eta = As @ x_hat + _offset(spec)
    terms = dict(log_prior_theta=log_theta_prior(spec, theta),
                 log_lik=log_likelihood(spec, eta),
                 quad=-0.5 * float(x_hat @ (Qp @ x_hat)),
                 half_logdet_Qp=0.5 * logdet_Qp,
                 half_logdet_Q=-0.5 * logdet_Q,
                 half_logdet_Sp=0.0, half_logdet_S=0.0)
    var = None
    if spec.C is not None:
        C = spec.C.to_dense()
        QiCt = sla.cho_solve((L, True), C.T)
        S = C @ QiCt
        Sp = C @ sla.cho_solve((chol(Qp), True), C.T)
        terms["half_logdet_Sp"] = float(np.log(np.diag(chol(Sp))).sum())
        terms["half_logdet_S"] = -float(np.log(np.diag(chol(S))).sum())
        if want_var:
            corr = np.einsum("ij,ij->i", QiCt, np.linalg.solve(S, QiCt.T).T)
            var = np.diag(spd_inverse(L)) - corr
    elif want_var:
        var = np.diag(spd_inverse(L))
    log_post = float(sum(terms.values()))
    return dict(log_post=log_post, x_hat=x_hat, var=var, newton_iters=iters,
                logdet_Q=logdet_Q, logdet_Qp=logdet_Qp, terms=terms)


# ------------------------------------------------------------------------------------
# Stage 2 (Section 2, Stage 1 and Stage 2; Appendix A.1.2, Eq. (thetatozscale); Appendix A.2):
# the Hessian of log pi~(theta|y) at theta*, the exploration points of the hyperparameter
# space, and the latent marginals integrated over them.
#
# Readings (the paper cites the grid and CCD strategies without their weights):
#  * Hessian by central second differences with step h (2 t^2 + 1 evaluations);
#  * z-coordinates: theta(z) = theta* + V Lambda^-1/2 z, (V, Lambda) the eigenpairs of the
#    negative Hessian, so z ~ N(0, I) under the Gaussian approximation of pi(theta|y);
#  * CCD: the centre plus the factorial points (+-1)^t (a half fraction with
#    x_t = x_1 ... x_{t-1} for t >= 5, giving the 45 points of t = 6) and the 2t axial points,
#    every non-centre point on the sphere of radius f0 sqrt(t); quadrature weight 1 at the
#    centre and delta = exp(f0^2 t / 2) / (N (f0^2 - 1)) at the N others, the value for which a
#    Gaussian pi(theta|y) has its variance reproduced exactly;
#  * grid: the points dz * k, |k_i| dz <= z_max, equal weights;
#  * integration weights w_k ~ delta_k pi~(theta_k|y) (the linear map's Jacobian is constant),
#    and the integrated marginal of x_i is the mixture of the Gaussian marginals
#    N(x_hat_i(theta_k), var_i(theta_k)): mean sum_k w_k x_hat_i, variance
#    sum_k w_k (var_i + x_hat_i^2) - mean^2.
# ------------------------------------------------------------------------------------

def hessian_fd(f, theta, h):
    """Central second differences of a scalar function f at theta (t x t):
    (f(+h e_i) - 2 f(0) + f(-h e_i)) / h^2 on the diagonal and
    (f(+,+) - f(+,-) - f(-,+) + f(-,-)) / (4 h^2) off it."""
    theta = np.asarray(theta, dtype=np.float64)
    t = theta.size
    E = np.eye(t) * h
    f0 = f(theta)
    H = np.zeros((t, t))
    for i in range(t):
        H[i, i] = (f(theta + E[i]) - 2.0 * f0 + f(theta - E[i])) / (h * h)
        for j in range(i + 1, t):
            H[i, j] = H[j, i] = (f(theta + E[i] + E[j]) - f(theta + E[i] - E[j]) - f(theta - E[i] + E[j])
                                 + f(theta - E[i] - E[j])) / (4.0 * h * h)
    return H


def ccd_design(t, f0=1.1):
    """CCD points in z-coordinates and their quadrature weights (see the readings above)."""
    import itertools
    corners = [np.array(c, dtype=np.float64) for c in itertools.product((-1.0, 1.0), repeat=t)]
    if t >= 5:
        corners = [c for c in corners if c[-1] == np.prod(c[:-1])]
    axial = [s * np.eye(t)[i] for i in range(t) for s in (1.0, -1.0)]
    dirs = corners + axial
    pts = [np.zeros(t)] + [d / np.linalg.norm(d) * f0 * math.sqrt(t) for d in dirs]
    N = len(dirs)
    delta = math.exp(f0 * f0 * t / 2.0) / (N * (f0 * f0 - 1.0))
    return np.array(pts), np.array([1.0] + [delta] * N)


def grid_design(t, dz, z_max):
    """Grid points dz * k with |k_i| dz <= z_max, equal weights."""
    import itertools
    K = int(math.floor(z_max / dz + 1e-12))
    ks = np.arange(-K, K + 1) * dz
    pts = np.array(list(itertools.product(ks, repeat=t)), dtype=np.float64)
    return pts, np.ones(len(pts))


def z_to_theta(theta_star, neg_hessian, Z):
    """theta(z) = theta* + V Lambda^-1/2 z for each row z of Z."""
    lam, V = np.linalg.eigh(np.asarray(neg_hessian, dtype=np.float64))
    if np.min(lam) <= 0:
        raise ValueError("the negative Hessian is not positive definite")
    return np.asarray(theta_star, dtype=np.float64)[None, :] + (np.atleast_2d(Z) / np.sqrt(lam)[None, :]) @ V.T


def integrate_marginals(spec, theta_star, neg_hessian, Z, delta):
    """Integrated Gaussian marginals of the latent field over the exploration points:
    evaluate every theta_k, weight w_k ~ delta_k exp(log pi~(theta_k|y)), and return the
    mixture's mean and variance per latent element."""
    thetas = z_to_theta(theta_star, neg_hessian, Z)
    res = [evaluate(spec, th) for th in thetas]
    lp = np.array([r["log_post"] for r in res])
    w = np.asarray(delta, dtype=np.float64) * np.exp(lp - lp.max())
    w = w / w.sum()
    X = np.array([r["x_hat"] for r in res])
    Vv = np.array([r["var"] for r in res])
    mean = w @ X
    var = w @ (Vv + X * X) - mean * mean
    return dict(mean=mean, var=var, weights=w, thetas=thetas, log_post=lp)


# ------------------------------------------------------------------------------------
# Variational Bayes correction of the posterior mean (Appendix A.2.2, Algorithm 2)
#
# Readings: the Gaussian posterior keeps the Laplace precision Q* and moves its mean by lambda;
# lambda minimises E_{x ~ N(mu + lambda, Q*^-1)}[-log pi(y|x)] + 1/2 (mu + lambda)^T Q_p (mu + lambda)
# (the KLD terms that depend on lambda), the expectation expanded to second order in
# delta = A lambda around the current mean, so each step solves
#     Q^c lambda = -c,   c = A^T I'(0) + Q_p mu,   Q^c = Q_p + A^T diag(I''(0)) A
# (the paper prints "Q^c lambda = c": the minimiser of its own objective carries the minus
# sign).  I'(0)_i, I''(0)_i are the means of l'(eta), l''(eta), l = -log pi(y_i|eta), under
# eta ~ N(nu_i, sigma_i^2), nu = A mu + offset, sigma_i^2 = (A Q*^-1 A^T)_ii from the Laplace
# approximation (fixed), by Gauss-Hermite quadrature with 15 points.  The mean is updated until
# max |lambda| <= 1e-8 (at most 50 steps).  Models with linear constraints are not covered.
# ------------------------------------------------------------------------------------

VB_GH_POINTS = 15
VB_TOL = 1e-8
VB_MAX = 50


def neg_loglik_derivs(spec, eta):
    """l'(eta), l''(eta) of l = -log pi(y|eta) per observation (Poisson: e^eta - y, e^eta;
    Gaussian with precision tau: tau (eta - y), tau)."""
    if spec.likelihood == "poisson":
        e = np.exp(eta)
        return e - spec.y[..., None] if eta.ndim == 2 else e - spec.y, e
    tau = spec.lik_prec
    y = spec.y[..., None] if eta.ndim == 2 else spec.y
    return tau * (eta - y), np.full_like(eta, tau)


def vb_expected_derivs(spec, nu, sigma2, n_gh=VB_GH_POINTS):
    """I'(0), I''(0): the means of l', l'' under eta_i ~ N(nu_i, sigma2_i) by Gauss-Hermite
    quadrature (nodes r_j, weights w_j of the weight e^-r^2): (1 / sqrt(pi)) sum_j w_j
    l(sqrt(2) sigma_i r_j + nu_i)."""
    r, w = np.polynomial.hermite.hermgauss(n_gh)
    eta = nu[:, None] + math.sqrt(2.0) * np.sqrt(sigma2)[:, None] * r[None, :]
    d1, d2 = neg_loglik_derivs(spec, eta)
    return d1 @ w / math.sqrt(math.pi), d2 @ w / math.sqrt(math.pi)


def vb_mean(spec, theta, n_gh=VB_GH_POINTS, tol=VB_TOL, max_iter=VB_MAX):
    """Algorithm 2 from the Laplace mode at theta: returns the corrected mean, the iterations,
    the Laplace result and the linear predictor's variances."""
    if spec.C is not None:
        raise ValueError("the variational Bayes correction is defined here for unconstrained models")
    theta = np.asarray(theta, dtype=np.float64)
    r = evaluate(spec, theta, want_var=False)
    As = _A_sparse(spec)
    Qp, _ = prior_precision(spec, theta)
    Qstar, _ = newton_system(spec, As, Qp, r["x_hat"])
    Sigma = spd_inverse(chol(Qstar))
    A = As.toarray()
    sigma2 = np.einsum("ij,jk,ik->i", A, Sigma, A)
    mu = r["x_hat"].copy()
    it = 0
    for it in range(1, max_iter + 1):
        nu = As @ mu + _offset(spec)
        I1, I2 = vb_expected_derivs(spec, nu, sigma2, n_gh)
        c = As.T @ I1 + Qp @ mu
        Qc = Qp + (As.T @ sp.diags(I2) @ As).toarray()
        lam = sla.cho_solve((chol(Qc), True), -c)
        mu = mu + lam
        if np.max(np.abs(lam)) <= tol:
            break
    return dict(mean=mu, iters=it, laplace=r, sigma_eta2=sigma2)


# ------------------------------------------------------------------------------------
# Moore-Penrose / Woodbury covariance route (Section 3.1, Eq. (woodeqn); Appendix C)
#
# Q+ is the Moore-Penrose pseudo-inverse of the prior precision without the eps jitter (block
# by block: 1 / prec, 1 / tau, the dense covariance Sigma, and (tau R)+ for intrinsic blocks);
# the posterior covariance is Sigma* = Q+ - Q+ (I + Q_like Q+)^-1 Q_like Q+ with
# Q_like = A^T D A the likelihood's negative Hessian.  Reading: Q_like is taken at the mode of
# the kriging route (with eps), to which this route is equal as eps -> 0 (Appendix C).
# ------------------------------------------------------------------------------------

def prior_pseudo_inverse(spec, theta):
    """Q+ block by block (dense n x n)."""
    n = spec.n
    P = np.zeros((n, n))
    start = 0
    for blk in spec.blocks:
        sl = slice(start, start + blk.size)
        if blk.kind == "fixed":
            P[sl, sl] = np.eye(blk.size) / blk.prec
        elif blk.kind == "iid":
            P[sl, sl] = np.eye(blk.size) * math.exp(-theta[blk.theta_idx])
        elif blk.kind == "dense_exp":
            P[sl, sl] = exp_covariance(blk, theta)
        elif blk.kind == "kron":
            R = np.ones((1, 1))
            for f in blk.factors:
                R = np.kron(R, structure_matrix(f))
            P[sl, sl] = np.linalg.pinv(math.exp(theta[blk.theta_idx]) * R, rcond=1e-10, hermitian=True)
        start += blk.size
    return P


def woodbury_covariance(Qplus, Qlike):
    """Eq. (woodeqn): Q+ - Q+ (I + Q_like Q+)^-1 Q_like Q+."""
    n = Qplus.shape[0]
    return Qplus - Qplus @ np.linalg.solve(np.eye(n) + Qlike @ Qplus, Qlike @ Qplus)


def woodbury_marginals(spec, theta):
    """Mean (the kriging route's mode) and the marginal variances of Eq. (woodeqn)."""
    theta = np.asarray(theta, dtype=np.float64)
    r = evaluate(spec, theta, want_var=False)
    As = _A_sparse(spec)
    eta = As @ r["x_hat"] + _offset(spec)
    w = np.exp(eta) if spec.likelihood == "poisson" else np.full(spec.m, spec.lik_prec)
    Qlike = (As.T @ sp.diags(w) @ As).toarray()
    S = woodbury_covariance(prior_pseudo_inverse(spec, theta), Qlike)
    return dict(mean=r["x_hat"], var=np.diag(S), laplace=r)

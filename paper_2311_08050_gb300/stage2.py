"""Stage 2 on the batched engine (Section 2, Stage 1 and Stage 2; Appendix A.1.2, Appendix A.2):
the Hessian of log pi~(theta|y) at its mode theta*, the exploration points of the hyperparameter
space, and the latent marginals integrated over them.

Host orchestration only: every log pi~ and every Gaussian marginal comes from
``inla.eval_batch`` (one batched device run per chunk of points) and the integration from
``inla_integrate_marginals`` (a device kernel); this module builds the point sets and the
finite-difference combinations of a handful of scalars.

* ``hessian``: central second differences with step h, the 2 t^2 + 1 points in one batch.
* ``ccd_design``: the centre, the factorial points (+-1)^t (the half fraction
  x_t = x_1 ... x_{t-1} from t = 5 on) and the 2t axial points, the non-centre points on the
  sphere of radius f0 sqrt(t); quadrature weights 1 at the centre and
  exp(f0^2 t / 2) / (N (f0^2 - 1)) at the N others (the value that reproduces the variance of a
  Gaussian pi(theta|y)).  ``grid_design``: dz * k, |k_i| dz <= z_max, equal weights.
* ``z_to_theta``: theta = theta* + V Lambda^-1/2 z, (V, Lambda) the eigenpairs of the negative
  Hessian, so that z ~ N(0, I) under the Gaussian approximation of pi(theta|y).
* ``integrate``: evaluate the design points (log pi~, x_hat, marginal variances kept on the
  device) and form the mixture moments of every latent element on the device.
"""
from __future__ import annotations

import ctypes as C
import itertools
import math

import numpy as np

from . import inla


def _stencil(theta, h):
    t = len(theta)
    pts = [theta.copy()]
    for i in range(t):
        for s in (1.0, -1.0):
            p = theta.copy()
            p[i] += s * h
            pts.append(p)
    for i in range(t):
        for j in range(i + 1, t):
            for si, sj in ((1.0, 1.0), (1.0, -1.0), (-1.0, 1.0), (-1.0, -1.0)):
                p = theta.copy()
                p[i] += si * h
                p[j] += sj * h
                pts.append(p)
    return np.array(pts)


def hessian(models, theta, h=2e-2, model_index=0, **opt_kw):
    """Central-difference Hessian of log pi~ at theta from one batch of 2 t^2 + 1 points."""
    theta = np.asarray(theta, dtype=np.float64)
    t = len(theta)
    pts = _stencil(theta, h)
    mot = np.full(len(pts), model_index, dtype=np.int32) if len(models) > 1 else None
    lp, st, _, _ = inla.eval_batch(models, pts, model_of_theta=mot, want_x=False, want_var=False, **opt_kw)
    if np.any(np.asarray(st) != 0):
        raise inla.InlaError(int(np.asarray(st)[np.asarray(st) != 0][0]), "stage2.hessian")
    H = np.empty((t, t))
    f0 = lp[0]
    for i in range(t):
        H[i, i] = (lp[1 + 2 * i] - 2.0 * f0 + lp[2 + 2 * i]) / (h * h)
    k = 1 + 2 * t
    for i in range(t):
        for j in range(i + 1, t):
            H[i, j] = H[j, i] = (lp[k] - lp[k + 1] - lp[k + 2] + lp[k + 3]) / (4.0 * h * h)
            k += 4
    return H


def ccd_design(t, f0=1.1):
    """(points z, quadrature weights) of the CCD described in the module docstring."""
    fact = np.array(list(itertools.product((-1.0, 1.0), repeat=t)))
    if t >= 5:
        fact = fact[fact[:, -1] == np.prod(fact[:, :-1], axis=1)]
    ax = np.concatenate([np.eye(t), -np.eye(t)])
    dirs = np.concatenate([fact, ax])
    dirs = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * (f0 * math.sqrt(t))
    N = len(dirs)
    d = math.exp(0.5 * f0 * f0 * t) / (N * (f0 * f0 - 1.0))
    return np.concatenate([np.zeros((1, t)), dirs]), np.concatenate([[1.0], np.full(N, d)])


def grid_design(t, dz, z_max):
    """(points z, weights) of the regular grid dz * k with |k_i| dz <= z_max."""
    K = int(math.floor(z_max / dz + 1e-12))
    axis = dz * np.arange(-K, K + 1)
    Z = np.array(list(itertools.product(axis, repeat=t)), dtype=np.float64)
    return Z, np.ones(len(Z))


def z_to_theta(theta_star, neg_hessian, Z):
    lam, V = np.linalg.eigh(np.asarray(neg_hessian, dtype=np.float64))
    if lam.min() <= 0.0:
        raise ValueError("the negative Hessian is not positive definite at theta*")
    return np.asarray(theta_star, dtype=np.float64) + (np.atleast_2d(Z) * (1.0 / np.sqrt(lam))) @ V.T


def integrate(model, theta_star, neg_hessian, Z, delta, chunk=16, **opt_kw):
    """Integrated Gaussian marginals of the latent field over the design (Z, delta) around
    theta*: returns (mean, var, thetas, log_post, status) with mean / var of length n."""
    import torch
    thetas = z_to_theta(theta_star, neg_hessian, Z)
    K, n = len(thetas), model.n
    X = torch.empty((K, n), dtype=torch.float64, device="cuda")
    Vv = torch.empty((K, n), dtype=torch.float64, device="cuda")
    lp = np.empty(K)
    st = np.empty(K, dtype=np.int32)
    for c in range(0, K, chunk):
        sl = slice(c, min(K, c + chunk))
        l, s, _, _ = inla.eval_batch([model], thetas[sl], device_out=True,
                                     x_out=[X[k].data_ptr() for k in range(sl.start, sl.stop)],
                                     var_out=[Vv[k].data_ptr() for k in range(sl.start, sl.stop)], **opt_kw)
        lp[sl] = np.where(np.asarray(s) == 0, l, -np.inf)
        st[sl] = s
    torch.cuda.synchronize()
    L = inla.lib()
    P = C.POINTER(C.c_double)
    L.inla_integrate_marginals.argtypes = [C.c_int32, C.c_int32, P, P, C.c_void_p, C.c_void_p, C.c_int64,
                                           C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    mean = torch.empty(n, dtype=torch.float64, device="cuda")
    var = torch.empty(n, dtype=torch.float64, device="cuda")
    dl = np.ascontiguousarray(delta, dtype=np.float64)
    rc = L.inla_integrate_marginals(K, n, lp.ctypes.data_as(P), dl.ctypes.data_as(P), X.data_ptr(), Vv.data_ptr(),
                                    n, mean.data_ptr(), var.data_ptr(), inla.OPT_DEVICE_OUT,
                                    opt_kw.get("stream"))
    if rc != 0:
        raise inla.InlaError(rc, "inla_integrate_marginals")
    return mean.cpu().numpy(), var.cpu().numpy(), thetas, lp, st

"""Precision-rung autotuner of the mixed path.

The mixed path's accuracy is set by its slice counts: ``prior_slices`` (the prior covariance's
factorisation and the inverse W of its factor), ``gram_slices`` (the prior precision W^T W),
``slices`` (the factor at the mode: log|Q*|), ``var_slices``
(the inverse of that factor, which gives the marginal variances) and ``newton_slices`` (the
Newton-step factorisations, which only steer the iteration: the gradient is exact).  Each slice
adds 7 bits and costs passes of the tensor-core GEMM (S (S + 1) / 2 BF16 products per GEMM), so
the cheapest setting that meets the accuracy targets depends on the model and its size.

``tune_precision`` calibrates on the model itself, with no oracle: it evaluates a probe point
with six slices everywhere (the FP64-accurate rung: log pi~ within ~1e-11 relative of FP64)
and takes that as the reference, then walks candidate settings from the cheapest up and keeps
the first whose log pi~, mode and variances stay within the targets divided by a safety margin
(3 by default) of the reference.  The choice is cached per (model, probe) and reported.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import inla

# (prior_slices, gram_slices, slices, newton_slices, var_slices) from the cheapest up by
# candidate_cost: the GEMM passes S (S + 1) / 2 of each phase weighted with its work per point of
# an FD batch -- the prior covariance's factorisation and inverse 2 n^3 / 3, the product W^T W
# n^3 / 3, the factor at the mode n^3 / 3, its inverse n^3 / 3 -- and the leading point's Newton
# factorisations at NEWTON_WEIGHT n^3 per point: four factorisations of one point in nine, whose
# single-slot launches run at about half the batched rate per flop (at n = 16384 that phase takes
# 148 ms per batch, as long as ~0.7 n^3 per point of batched work at 5 slices)
NEWTON_WEIGHT = 0.7


def candidate_cost(setting) -> float:
    """Relative GEMM cost per point of an FD batch of a (prior, gram, final, Newton, variance)
    slice setting, in units of n^3 BF16 passes."""
    p, g, s, nw, v = setting
    passes = lambda k: k * (k + 1) / 2
    return (2 * passes(p) + passes(g) + passes(s) + passes(v)) / 3 + NEWTON_WEIGHT * passes(nw)


CANDIDATES = [(4, 4, 4, 3, 3), (4, 4, 4, 3, 4), (4, 5, 4, 3, 4), (4, 4, 5, 3, 4), (4, 5, 5, 3, 3), (4, 4, 4, 4, 4),
              (4, 5, 5, 3, 4), (5, 5, 4, 3, 4), (5, 5, 5, 3, 3), (4, 5, 5, 4, 4), (5, 5, 5, 3, 4), (5, 5, 5, 3, 5),
              (5, 5, 5, 4, 4), (5, 5, 5, 4, 5), (6, 6, 5, 4, 5), (6, 6, 6, 4, 6)]


@dataclass
class TuneResult:
    prior_slices: int
    gram_slices: int
    slices: int
    newton_slices: int
    var_slices: int
    errors: dict
    tried: list = field(default_factory=list)
    seconds: float = 0.0

    def opts(self):
        return dict(prior_slices=self.prior_slices, gram_slices=self.gram_slices, slices=self.slices,
                    newton_slices=self.newton_slices, var_slices=self.var_slices)


_cache: dict = {}


def _errors(ref, cand):
    lp0, x0, v0 = ref
    lp, x, v = cand
    return {"log_post_abs": float(abs(lp - lp0)),
            "x_hat_rel": float(np.max(np.abs(x - x0)) / max(1.0, np.max(np.abs(x0)))),
            "var_rel": float(np.max(np.abs(v / v0 - 1.0)))}


def tune_precision(model, theta, lp_abs=1e-3, var_rel=1e-4, x_rel=1e-4, margin=3.0, **opt_kw):
    """The cheapest (prior_slices, gram_slices, slices, newton_slices, var_slices) whose errors against the six-slice
    evaluation of `theta` are within (targets / margin).  opt_kw: stream and other options
    passed to every evaluation."""
    key = (id(model), tuple(np.round(np.asarray(theta, dtype=np.float64), 12)), lp_abs, var_rel, x_rel, margin)
    if key in _cache:
        return _cache[key]
    t0 = time.perf_counter()
    th = np.asarray(theta, dtype=np.float64)[None, :]

    def run(p, g, s, nw, v):
        lp, st, xs, vs = inla.eval_batch([model], th, precision="mixed", prior_slices=p, gram_slices=g, slices=s,
                                         newton_slices=nw, var_slices=v, **opt_kw)
        if st[0] != 0:
            return None
        return float(lp[0]), xs[0], vs[0]

    ref = run(6, 6, 6, 4, 6)
    if ref is None:
        raise RuntimeError("reference evaluation failed")
    tried = []
    chosen = None
    for p, g, s, nw, v in CANDIDATES:
        r = run(p, g, s, nw, v)
        if r is None:
            tried.append({"setting": (p, g, s, nw, v), "status": "failed"})
            continue
        e = _errors(ref, r)
        ok = e["log_post_abs"] <= lp_abs / margin and e["var_rel"] <= var_rel / margin and e["x_hat_rel"] <= x_rel / margin
        tried.append({"setting": (p, g, s, nw, v), "errors": e, "ok": bool(ok)})
        if ok:
            chosen = TuneResult(p, g, s, nw, v, e)
            break
    if chosen is None:
        chosen = TuneResult(6, 6, 6, 4, 6, {"log_post_abs": 0.0, "x_hat_rel": 0.0, "var_rel": 0.0})
    chosen.tried = tried
    chosen.seconds = time.perf_counter() - t0
    _cache[key] = chosen
    return chosen

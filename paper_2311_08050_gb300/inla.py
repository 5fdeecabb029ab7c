"""ctypes binding of libinla (include/inla.h): argument marshalling only.

Every computation happens inside the CUDA library; this module converts a seeded
``ModelSpec`` (see synth.py) into the C descriptor, and numpy / torch buffers into
pointers.  Importing it does not load the library; the first call does, and fails loudly
if the in-tree ``libinla.so`` has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libinla.so")

OK, E_BADARG, E_CUDA, E_NOT_SPD, E_NO_CONVERGENCE, E_TIMEOUT, E_UNSUPPORTED, E_NOMEM = 0, -1, -2, -3, -4, -5, -6, -7
LIK = {"poisson": 0, "gaussian": 1}
BLOCK = {"fixed": 0, "iid": 1, "dense_exp": 2, "kron": 3}
FACTOR = {"icar": 0, "rw1": 1, "rw2": 2, "iid": 3}
PRIOR = {"gauss": 0, "pc_prec": 1}
PRECISION = {"fp64": 0, "mixed": 1}
OPT_DEVICE_OUT = 1
OPT_NO_SHARED_START = 2
OPT_VB_MEAN = 4
OPT_WOODBURY_VAR = 8

EXPORTED = ["inla_opts_default", "inla_model_create", "inla_model_destroy", "inla_eval_theta",
            "inla_eval_batch", "inla_marginals", "inla_status_string"]

_P = C.POINTER
_d, _i32, _i64 = C.c_double, C.c_int32, C.c_int64


class Factor(C.Structure):
    _fields_ = [("kind", _i32), ("size", _i32), ("graph_rowptr", _P(_i64)), ("graph_col", _P(_i32))]


class BlockS(C.Structure):
    _fields_ = [("kind", _i32), ("size", _i32), ("prec", _d), ("theta_idx", _i32), ("points", _P(_d)),
                ("theta_sigma", _i32), ("theta_range_x", _i32), ("theta_range_y", _i32), ("theta_iid", _i32),
                ("nugget", _d), ("nfactors", _i32), ("factors", _P(Factor)), ("eps", _d)]


class ModelDesc(C.Structure):
    _fields_ = [("n", _i32), ("m", _i32), ("k", _i32), ("likelihood", _i32), ("lik_prec", _d),
                ("A_rowptr", _P(_i64)), ("A_col", _P(_i32)), ("A_val", _P(_d)),
                ("y", _P(_d)), ("offset", _P(_d)),
                ("nblocks", _i32), ("blocks", _P(BlockS)),
                ("C_rowptr", _P(_i64)), ("C_col", _P(_i32)), ("C_val", _P(_d)),
                ("theta_dim", _i32), ("theta_prior_kind", _P(_i32)), ("theta_prior_a", _P(_d)),
                ("theta_prior_b", _P(_d))]


class Opts(C.Structure):
    _fields_ = [("precision", _i32), ("slices", _i32), ("newton_slices", _i32), ("newton_tol", _d),
                ("newton_max", _i32),
                ("spin_limit", _i64), ("stream", C.c_void_p), ("flags", _i32), ("prior_slices", _i32),
                ("reuse_below", _d), ("reuse_shrink", _d), ("var_slices", _i32), ("gram_slices", _i32)]


_lib = None


def lib():
    """The loaded library (loads it on first use; raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built: run paper_2311_08050_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.inla_opts_default.argtypes = [_P(Opts)]
        L.inla_model_create.argtypes = [_P(ModelDesc), _P(C.c_void_p)]
        L.inla_model_destroy.argtypes = [C.c_void_p]
        L.inla_eval_theta.argtypes = [C.c_void_p, _P(_d), _P(Opts), _P(_d), C.c_void_p, _P(_i32)]
        L.inla_eval_batch.argtypes = [_P(C.c_void_p), _i32, _P(_i32), _P(_d), _i32, _P(Opts), _P(_d), _P(_i32),
                                      _P(C.c_void_p), _P(C.c_void_p)]
        L.inla_marginals.argtypes = [C.c_void_p, _P(_d), _P(Opts), C.c_void_p, C.c_void_p]
        L.inla_status_string.argtypes = [C.c_int]
        L.inla_status_string.restype = C.c_char_p
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().inla_status_string(int(code)).decode()


class InlaError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct)) if a is not None else None


def make_opts(precision="fp64", slices=0, newton_tol=1e-8, newton_max=50, stream=None, device_out=False,
              spin_limit=1 << 26, newton_slices=0, flags_extra=0, prior_slices=0, reuse_below=0.0,
              reuse_shrink=0.0, var_slices=0, gram_slices=0):
    o = Opts()
    lib().inla_opts_default(C.byref(o))
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.slices = slices
    o.newton_slices = newton_slices
    o.newton_tol = newton_tol
    o.newton_max = newton_max
    o.spin_limit = spin_limit
    o.stream = stream
    o.flags = (OPT_DEVICE_OUT if device_out else 0) | int(flags_extra)
    o.prior_slices = prior_slices
    o.reuse_below = reuse_below
    o.reuse_shrink = reuse_shrink
    o.var_slices = var_slices
    o.gram_slices = gram_slices
    return o


class Model:
    """A model resident on the current CUDA device (wraps inla_model*)."""

    def __init__(self, spec):
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a

        self.spec = spec
        self.n, self.m, self.k = spec.n, spec.m, spec.k
        self.theta_dim = spec.theta_dim
        blocks = (BlockS * len(spec.blocks))()
        for bi, b in enumerate(spec.blocks):
            bs = blocks[bi]
            bs.kind, bs.size = BLOCK[b.kind], b.size
            bs.prec, bs.theta_idx = b.prec, b.theta_idx
            bs.theta_sigma, bs.theta_range_x, bs.theta_range_y = b.theta_sigma, b.theta_range_x, b.theta_range_y
            bs.theta_iid, bs.nugget, bs.eps = b.theta_iid, b.nugget, b.eps
            if b.points is not None:
                bs.points = _ptr(arr(b.points, np.float64), _d)
            if b.factors:
                fs = (Factor * len(b.factors))()
                for fi, f in enumerate(b.factors):
                    fs[fi].kind, fs[fi].size = FACTOR[f.kind], f.size
                    if f.graph is not None:
                        fs[fi].graph_rowptr = _ptr(arr(f.graph.rowptr, np.int64), _i64)
                        fs[fi].graph_col = _ptr(arr(f.graph.col, np.int32), _i32)
                keep.append(fs)
                bs.nfactors, bs.factors = len(b.factors), fs
        d = ModelDesc()
        d.n, d.m, d.k = spec.n, spec.m, spec.k
        d.likelihood, d.lik_prec = LIK[spec.likelihood], spec.lik_prec
        d.A_rowptr = _ptr(arr(spec.A.rowptr, np.int64), _i64)
        d.A_col = _ptr(arr(spec.A.col, np.int32), _i32)
        d.A_val = _ptr(arr(spec.A.val, np.float64), _d)
        d.y = _ptr(arr(spec.y, np.float64), _d)
        d.offset = _ptr(arr(spec.offset, np.float64), _d) if spec.offset is not None else None
        d.nblocks, d.blocks = len(spec.blocks), blocks
        if spec.C is not None:
            d.C_rowptr = _ptr(arr(spec.C.rowptr, np.int64), _i64)
            d.C_col = _ptr(arr(spec.C.col, np.int32), _i32)
            d.C_val = _ptr(arr(spec.C.val, np.float64), _d)
        d.theta_dim = spec.theta_dim
        d.theta_prior_kind = _ptr(arr([PRIOR[p[0]] for p in spec.theta_prior], np.int32), _i32)
        d.theta_prior_a = _ptr(arr([p[1] for p in spec.theta_prior], np.float64), _d)
        d.theta_prior_b = _ptr(arr([p[2] for p in spec.theta_prior], np.float64), _d)
        h = C.c_void_p()
        rc = lib().inla_model_create(C.byref(d), C.byref(h))
        if rc != OK:
            raise InlaError(rc, "inla_model_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().inla_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval_batch(models: Sequence[Model], thetas, model_of_theta=None, want_x=True, want_var=True,
               x_out=None, var_out=None, **opt_kw):
    """Evaluate B theta points (rows of `thetas`) in one batched device run.

    Returns (log_post[B], status[B], x_hat list, var list).  With ``device_out=True`` the
    caller passes ``x_out`` / ``var_out`` lists of device pointers (ints) and gets them back.
    """
    thetas = np.ascontiguousarray(np.atleast_2d(thetas), dtype=np.float64)
    B = thetas.shape[0]
    nm = len(models)
    mh = (C.c_void_p * nm)(*[m.handle for m in models])
    mot = None
    if model_of_theta is not None:
        mot_arr = np.ascontiguousarray(model_of_theta, dtype=np.int32)
        mot = _ptr(mot_arr, _i32)
    else:
        mot_arr = np.zeros(B, dtype=np.int32)
    o = make_opts(**opt_kw)
    lp = np.zeros(B)
    st = np.zeros(B, dtype=np.int32)
    xs = vs = None
    xp = vp = None
    if o.flags & OPT_DEVICE_OUT:
        if want_x and x_out is not None:
            xp = (C.c_void_p * B)(*x_out)
        if want_var and var_out is not None:
            vp = (C.c_void_p * B)(*var_out)
    else:
        if want_x:
            xs = [np.zeros(models[mot_arr[b]].n) for b in range(B)]
            xp = (C.c_void_p * B)(*[x.ctypes.data for x in xs])
        if want_var:
            vs = [np.zeros(models[mot_arr[b]].n) for b in range(B)]
            vp = (C.c_void_p * B)(*[v.ctypes.data for v in vs])
    rc = lib().inla_eval_batch(mh, nm, mot, _ptr(thetas, _d), B, C.byref(o), _ptr(lp, _d), _ptr(st, _i32), xp, vp)
    if rc != OK:
        raise InlaError(rc, "inla_eval_batch")
    return lp, st, xs, vs


def eval_theta(model: Model, theta, **opt_kw):
    """(log_post, x_hat, newton_iters) at one theta."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    o = make_opts(**opt_kw)
    lp = C.c_double()
    x = np.zeros(model.n)
    it = C.c_int32()
    rc = lib().inla_eval_theta(model.handle, _ptr(theta, _d), C.byref(o), C.byref(lp), x.ctypes.data, C.byref(it))
    if rc != OK:
        raise InlaError(rc, "inla_eval_theta")
    return lp.value, x, it.value


def marginals(model: Model, theta, **opt_kw):
    """(mean, var) of the Gaussian marginals at one theta."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    o = make_opts(**opt_kw)
    mean, var = np.zeros(model.n), np.zeros(model.n)
    rc = lib().inla_marginals(model.handle, _ptr(theta, _d), C.byref(o), mean.ctypes.data, var.ctypes.data)
    if rc != OK:
        raise InlaError(rc, "inla_marginals")
    return mean, var

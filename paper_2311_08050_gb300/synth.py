"""Seeded synthetic latent Gaussian models (LGMs) shaped like the paper's workloads.

This module only *describes* models and draws data: it holds none of the
method's arithmetic (no prior precision, no Laplace approximation, no
factorisation).  Both the FP64 oracle and the CUDA path read the same
`ModelSpec`, so their inputs are identical by construction.

The LGM statement follows Section 1 of the paper: y_i | x, theta ~ f(eta_i,
theta), eta = A x (+ offset), x | theta ~ N(0, Q_prior(theta)^-1),
theta ~ pi(theta).  The workloads stand in for the paper's simulation study
(Section 4, Tables 1-2: Poisson counts, dense spatial effects) and its
space x time x age disease-mapping model (Section 5, Type IV Kronecker
interactions with sum-to-zero constraints); the paper's datasets are not
available, so every input here is drawn from a fixed seed.

Prior blocks (latent vector = concatenation of blocks, in the given order):
  * ``fixed``     : precision ``prec`` * I (e.g. the intercept, precision 1e-3)
  * ``iid``       : exp(theta[theta_idx]) * I
  * ``dense_exp`` : covariance  sigma^2 exp(-d) + (1/tau_iid + nugget) I  on 2-D
                    points, d = sqrt((dx/rho_x)^2 + (dy/rho_y)^2); the block's
                    precision is the inverse of that covariance
  * ``kron``      : exp(theta[theta_idx]) * (R_1 kron R_2 kron ...) + eps I with
                    factors ICAR (graph Laplacian D - W), RW1 or IID
Theta priors: ``("gauss", mean, sd)`` or ``("pc_prec", U, alpha)`` on a log
precision.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

SEED_BASE = 2311080500


@dataclasses.dataclass
class CSR:
    nrows: int
    ncols: int
    rowptr: np.ndarray  # int64, nrows+1
    col: np.ndarray     # int32
    val: np.ndarray     # float64

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.nrows, self.ncols))
        for i in range(self.nrows):
            lo, hi = self.rowptr[i], self.rowptr[i + 1]
            np.add.at(out[i], self.col[lo:hi], self.val[lo:hi])
        return out

    @staticmethod
    def from_rows(nrows: int, ncols: int, rows_cols: Sequence[np.ndarray],
                  rows_vals: Sequence[np.ndarray]) -> "CSR":
        lens = np.array([len(c) for c in rows_cols], dtype=np.int64)
        rowptr = np.zeros(nrows + 1, dtype=np.int64)
        rowptr[1:] = np.cumsum(lens)
        col = np.concatenate(rows_cols).astype(np.int32) if nrows else np.zeros(0, np.int32)
        val = np.concatenate(rows_vals).astype(np.float64) if nrows else np.zeros(0)
        return CSR(nrows, ncols, rowptr, col, val)


@dataclasses.dataclass
class Factor:
    kind: str                      # "icar" | "rw1" | "iid"
    size: int
    graph: Optional[CSR] = None    # adjacency (0/1, symmetric, no diagonal) for "icar"


@dataclasses.dataclass
class Block:
    kind: str                      # "fixed" | "iid" | "dense_exp" | "kron"
    size: int
    prec: float = 0.0              # fixed
    theta_idx: int = -1            # iid / kron: log precision
    points: Optional[np.ndarray] = None   # dense_exp: (size, 2)
    theta_sigma: int = -1          # dense_exp: log sigma
    theta_range_x: int = -1        # dense_exp: log rho_x
    theta_range_y: int = -1        # dense_exp: log rho_y (== range_x when isotropic)
    theta_iid: int = -1            # dense_exp: log tau of a folded iid effect (-1: none)
    nugget: float = 1e-6
    factors: List[Factor] = dataclasses.field(default_factory=list)  # kron
    eps: float = 0.0               # kron: jitter added to the intrinsic structure


@dataclasses.dataclass
class ModelSpec:
    name: str
    n: int
    likelihood: str                # "poisson" | "gaussian"
    A: CSR
    y: np.ndarray
    offset: Optional[np.ndarray]
    blocks: List[Block]
    theta_prior: List[tuple]
    C: Optional[CSR] = None
    lik_prec: float = 1.0          # gaussian: fixed observation precision

    @property
    def m(self) -> int:
        return self.A.nrows

    @property
    def k(self) -> int:
        return 0 if self.C is None else self.C.nrows

    @property
    def theta_dim(self) -> int:
        return len(self.theta_prior)


# --------------------------------------------------------------------------------------
# random fields used only to draw the synthetic truth (not the method)
# --------------------------------------------------------------------------------------

def _exp_field_rff(rng, pts, sigma, rho_x, rho_y, nfeat=2048):
    """Approximate draw of a zero-mean field with covariance sigma^2 exp(-d) by random
    Fourier features: the spectral density of exp(-|h|) in 2-D is a bivariate Cauchy
    (Student-t, 1 dof), so omega = g / sqrt(u) with g ~ N(0, I), u ~ chi^2_1."""
    g = rng.standard_normal((nfeat, 2))
    u = rng.chisquare(1.0, size=(nfeat, 1))
    omega = g / np.sqrt(u)
    omega[:, 0] /= rho_x
    omega[:, 1] /= rho_y
    phase = rng.uniform(0, 2 * np.pi, nfeat)
    return sigma * np.sqrt(2.0 / nfeat) * np.cos(pts @ omega.T + phase).sum(axis=1)


def _selector_A(rng, m, n_pts, col0, with_intercept):
    """Each observation reads the intercept (column 0) and one uniformly drawn point."""
    pick = rng.integers(0, n_pts, size=m)
    r = 2 if with_intercept else 1
    rowptr = np.arange(m + 1, dtype=np.int64) * r
    col = np.empty((m, r), dtype=np.int32)
    if with_intercept:
        col[:, 0] = 0
    col[:, r - 1] = col0 + pick
    return CSR(m, 0, rowptr, col.reshape(-1), np.ones(m * r)), pick


def _fd_batch(center, h=5e-3):
    """Central finite-difference stencil: center, then +h and -h along each axis."""
    center = np.asarray(center, dtype=np.float64)
    pts = [center.copy()]
    for a in range(center.size):
        for s in (+1.0, -1.0):
            p = center.copy()
            p[a] += s * h
            pts.append(p)
    return np.stack(pts)


def delaunay_graph(rng, n_regions):
    """Planar, connected adjacency: Delaunay triangulation of seeded uniform points."""
    from scipy.spatial import Delaunay
    pts = rng.uniform(0, 1, size=(n_regions, 2))
    tri = Delaunay(pts)
    nbr = [set() for _ in range(n_regions)]
    for s in tri.simplices:
        for a in range(3):
            for b in range(3):
                if a != b:
                    nbr[s[a]].add(int(s[b]))
    cols = [np.array(sorted(nb), dtype=np.int64) for nb in nbr]
    vals = [np.ones(len(c)) for c in cols]
    return CSR.from_rows(n_regions, n_regions, cols, vals)


# --------------------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------------------

def spatial_poisson(name, seed, n_pts, m, theta_true, anisotropic=False, folded_iid=False):
    """Poisson LGM: intercept (precision 1e-3) + dense exponential-covariance spatial
    effect on n_pts uniform points of [0,1]^2; A selects intercept + one point per row."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, size=(n_pts, 2))
    theta_true = np.asarray(theta_true, dtype=np.float64)
    sigma = np.exp(theta_true[0])
    rho_x = np.exp(theta_true[1])
    rho_y = np.exp(theta_true[2]) if anisotropic else rho_x
    field = _exp_field_rff(rng, pts, sigma, rho_x, rho_y)
    if folded_iid:
        tau_iid = np.exp(theta_true[3] if anisotropic else theta_true[2])
        field = field + rng.standard_normal(n_pts) / np.sqrt(tau_iid)
    n = 1 + n_pts
    A, pick = _selector_A(rng, m, n_pts, 1, True)
    A.ncols = n
    eta = field[pick]
    y = rng.poisson(np.exp(eta)).astype(np.float64)
    t = 0
    blk_d = Block("dense_exp", n_pts, points=pts, theta_sigma=0, theta_range_x=1,
                  theta_range_y=2 if anisotropic else 1, nugget=1e-6)
    t = 3 if anisotropic else 2
    prior = [("gauss", 0.0, 1.0), ("gauss", 0.0, 1.0)] + ([("gauss", 0.0, 1.0)] if anisotropic else [])
    if folded_iid:
        blk_d.theta_iid = t
        prior.append(("pc_prec", 1.0, 0.01))
    blocks = [Block("fixed", 1, prec=1e-3), blk_d]
    return ModelSpec(name, n, "poisson", A, y, None, blocks, prior)


def poisson_n256_m1000_5pts():
    """n = 256 (intercept + 255 points), m = 1000, theta = (log sigma, log rho);
    five seeded theta points around (0, log 0.2)."""
    spec = spatial_poisson("poisson_n256_m1000", SEED_BASE + 1, 255, 1000, [0.0, np.log(0.2)])
    rng = np.random.default_rng(SEED_BASE + 101)
    thetas = np.array([0.0, np.log(0.2)]) + 0.3 * rng.standard_normal((5, 2))
    return spec, thetas


def poisson_n4096_m20000_fd7():
    """n = 4096 (intercept + 4095 points), m = 20000, theta = (log sigma, log rho,
    log tau_iid) with the iid effect folded into the covariance diagonal; batch of
    2*3+1 central finite-difference points."""
    th = np.array([0.0, np.log(0.2), np.log(4.0)])
    spec = spatial_poisson("poisson_n4096_m20000", SEED_BASE + 2, 4095, 20000, th, folded_iid=True)
    return spec, _fd_batch(th)


def poisson_n16384_m100000_fd9():
    """n = 16384 (intercept + 16383 points), m = 100000, theta = (log sigma, log rho_x,
    log rho_y, log tau_iid): anisotropic range + folded iid; batch of 2*4+1 FD points."""
    th = np.array([0.0, np.log(0.2), np.log(0.1), np.log(4.0)])
    spec = spatial_poisson("poisson_n16384_m100000", SEED_BASE + 5, 16383, 100000, th,
                           anisotropic=True, folded_iid=True)
    return spec, _fd_batch(th)


def poisson_n16384_theta_true():
    return np.array([0.0, np.log(0.2), np.log(0.1), np.log(4.0)])


def _rw1_walk(rng, n, sd):
    w = np.cumsum(rng.standard_normal(n) * sd)
    return w - w.mean()


def spacetime_age(name, seed, n_s=50, n_t=20, n_a=8, eps=1e-5):
    """Space x time x age Poisson model with a 3-way Kronecker interaction
    ICAR(n_s) x RW1(n_t) x RW1(n_a), main effects ICAR + iid (space), RW1 + iid (time),
    RW1 (age), an intercept, one count per cell with log-offsets ~ N(3, 0.5^2), and the
    sum-to-zero constraints that span the null space of every intrinsic block."""
    rng = np.random.default_rng(seed)
    g = delaunay_graph(rng, n_s)
    sizes = [1, n_s, n_s, n_t, n_t, n_a, n_s * n_t * n_a]
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    n = int(sum(sizes))
    b_mu, b_s, b_is, b_t, b_it, b_a, b_x = starts
    blocks = [
        Block("fixed", 1, prec=1e-3),
        Block("kron", n_s, theta_idx=0, factors=[Factor("icar", n_s, g)], eps=eps),
        Block("iid", n_s, theta_idx=1),
        Block("kron", n_t, theta_idx=2, factors=[Factor("rw1", n_t)], eps=eps),
        Block("iid", n_t, theta_idx=3),
        Block("kron", n_a, theta_idx=4, factors=[Factor("rw1", n_a)], eps=eps),
        Block("kron", n_s * n_t * n_a, theta_idx=5,
              factors=[Factor("icar", n_s, g), Factor("rw1", n_t), Factor("rw1", n_a)], eps=eps),
    ]
    # synthetic truth (smooth-ish, centred); the 3-way part is centred along every axis
    x_s = rng.standard_normal(n_s) * 0.3
    x_s -= x_s.mean()
    x_is = rng.standard_normal(n_s) * 0.1
    x_t = _rw1_walk(rng, n_t, 0.05)
    x_it = rng.standard_normal(n_t) * 0.05
    x_a = _rw1_walk(rng, n_a, 0.2)
    z = rng.standard_normal((n_s, n_t, n_a)) * 0.1
    z = z - z.mean(axis=0, keepdims=True)
    z = z - z.mean(axis=1, keepdims=True)
    z = z - z.mean(axis=2, keepdims=True)
    m = n_s * n_t * n_a
    cols, vals = [], []
    eta = np.zeros(m)
    offset = 3.0 + 0.5 * rng.standard_normal(m)
    for s in range(n_s):
        for t in range(n_t):
            for a in range(n_a):
                i = (s * n_t + t) * n_a + a
                cols.append(np.array([b_mu, b_s + s, b_is + s, b_t + t, b_it + t, b_a + a,
                                      b_x + i]))
                vals.append(np.ones(7))
                eta[i] = x_s[s] + x_is[s] + x_t[t] + x_it[t] + x_a[a] + z[s, t, a]
    A = CSR.from_rows(m, n, cols, vals)
    y = rng.poisson(np.exp(eta + offset)).astype(np.float64)
    # constraints: one sum-to-zero per intrinsic main effect, and 1483 independent rows
    # for the 3-way block: sums over s for every (t, a); over t for (s < n_s-1, a);
    # over a for (s < n_s-1, t < n_t-1)
    crow_c, crow_v = [], []
    for st, sz in ((b_s, n_s), (b_t, n_t), (b_a, n_a)):
        crow_c.append(np.arange(st, st + sz))
        crow_v.append(np.ones(sz))
    idx = lambda s, t, a: b_x + (s * n_t + t) * n_a + a
    for t in range(n_t):
        for a in range(n_a):
            crow_c.append(np.array([idx(s, t, a) for s in range(n_s)]))
            crow_v.append(np.ones(n_s))
    for s in range(n_s - 1):
        for a in range(n_a):
            crow_c.append(np.array([idx(s, t, a) for t in range(n_t)]))
            crow_v.append(np.ones(n_t))
    for s in range(n_s - 1):
        for t in range(n_t - 1):
            crow_c.append(np.array([idx(s, t, a) for a in range(n_a)]))
            crow_v.append(np.ones(n_a))
    C = CSR.from_rows(len(crow_c), n, crow_c, crow_v)
    prior = [("pc_prec", 1.0, 0.01)] * 6
    return ModelSpec(name, n, "poisson", A, y, offset, blocks, prior, C=C)


def spacetime_n8149_m8000_fd13():
    """50 Delaunay regions x 20 years x 8 ages (n = 8149, k = 1486 constraints), theta = six
    log precisions; batch of 2*6+1 central finite-difference points."""
    spec = spacetime_age("spacetime_age_n8149_k1486", SEED_BASE + 3)
    center = np.array([1.0, 2.0, 3.0, 4.0, 1.0, 2.0])
    return spec, _fd_batch(center)


def gaussian_spatial(name, seed, n, tau=10.0, theta=(0.0, np.log(0.2))):
    """Gaussian LGM: dense exponential-covariance effect on n points (no intercept),
    m = 4n selector observations with fixed noise precision tau."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, size=(n, 2))
    field = _exp_field_rff(rng, pts, np.exp(theta[0]), np.exp(theta[1]), np.exp(theta[1]))
    m = 4 * n
    A, pick = _selector_A(rng, m, n, 0, False)
    A.ncols = n
    y = field[pick] + rng.standard_normal(m) / np.sqrt(tau)
    blk = Block("dense_exp", n, points=pts, theta_sigma=0, theta_range_x=1, theta_range_y=1,
                nugget=1e-6)
    prior = [("gauss", 0.0, 1.0), ("gauss", 0.0, 1.0)]
    return ModelSpec(name, n, "gaussian", A, y, None, [blk], prior, lik_prec=tau)


def gaussian_64_models_n512_4096(n_models=64, sizes=(512, 1024, 2048, 4096)):
    """64 independent Gaussian LGMs with n drawn uniformly from {512, 1024, 2048, 4096};
    each evaluated at its own seeded theta."""
    rng = np.random.default_rng(SEED_BASE + 4)
    ns = rng.choice(np.array(sizes), size=n_models)
    specs, thetas = [], []
    for i, n in enumerate(ns):
        specs.append(gaussian_spatial(f"gauss_{i}_n{n}", SEED_BASE + 400 + i, int(n)))
        thetas.append(np.array([0.0, np.log(0.2)]) + 0.2 * rng.standard_normal(2))
    return specs, np.stack(thetas)


def surrogate_thetas(n_points, seed=SEED_BASE + 55, spread=0.5):
    """Training design for the learned surrogate: theta ~ N(theta_true, spread^2 I)."""
    rng = np.random.default_rng(seed)
    return poisson_n16384_theta_true() + spread * rng.standard_normal((n_points, 4))


WORKLOADS = {f.__name__: f for f in (poisson_n256_m1000_5pts, poisson_n4096_m20000_fd7, spacetime_n8149_m8000_fd13,
                                      gaussian_64_models_n512_4096, poisson_n16384_m100000_fd9)}

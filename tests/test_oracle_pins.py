"""Pins of the FP64 oracle against things other than itself.

Each test fixes one part of the oracle with an independent route: the worked example
printed in Appendix C, closed forms (the Gaussian-likelihood marginal likelihood, where
the Laplace approximation of Eq. (41) is exact), brute force on tiny inputs (an
independent optimiser plus finite-difference Hessians), eigenvalue routes for
determinants, the constraint counts of Section 5.2, and the normalisation of the PC prior.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so
import scipy.sparse as sp
from scipy.integrate import quad
from scipy.stats import multivariate_normal

from oracle import inla_oracle as O
from paper_2311_08050_gb300 import synth
from paper_2311_08050_gb300.synth import CSR, Block, Factor, ModelSpec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out, key, rows = {}, None, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            try:
                vals = [float(t) for t in tok]
                rows.append(vals)
                continue
            except ValueError:
                pass
            if key is not None:
                out[key] = np.array(rows) if len(rows) > 1 else np.array(rows[0])
            key, rows = tok[0], []
            if len(tok) > 1:
                rows.append([float(t) for t in tok[1:]])
    out[key] = np.array(rows) if len(rows) > 1 else np.array(rows[0])
    return out


# ---------------------------------------------------------------------------------
# Appendix C worked example
# ---------------------------------------------------------------------------------

def test_appendix_c_kriging_matches_printed_matrices():
    g = _read_golden("appendix_c_example.txt")
    eps = float(g["eps"][0])
    A, Ql, Qe, C = g["A"], np.diag(g["Ql"]), g["Qe"], g["C"].reshape(1, -1)
    Q = A.T @ Ql @ A + Qe + eps * np.eye(4)
    # the uncorrected covariance, and the kriging correction of the oracle
    assert np.max(np.abs(np.linalg.inv(Q) - g["Sigma_un"])) <= 5e-4
    S_star = O.kriging_covariance(Q, C)
    assert np.max(np.abs(S_star - g["Sigma_star"])) <= 5e-4
    # the oracle's kriging mean satisfies the constraint and equals the projection
    x_u = np.array([0.3, -1.0, 2.0, 0.5])
    xk = O.kriging_mean(Q, C, x_u)
    assert abs(float((C @ xk)[0])) < 1e-12
    # the Woodbury route of Eq. (woodeqn) with the printed pseudo-inverse
    Qp = np.linalg.pinv(Qe)
    assert np.max(np.abs(Qp - g["Qe_pinv"])) <= 5e-4
    Qlike = A.T @ Ql @ A
    S_wood = Qp - Qp @ np.linalg.solve(np.eye(4) + Qlike @ Qp, Qlike @ Qp)
    assert np.max(np.abs(S_wood - g["Sigma_star"])) <= 5e-4
    # kriging (with eps) and Woodbury/pinv differ by O(eps) only
    assert np.max(np.abs(S_wood - S_star)) < 10 * eps


# ---------------------------------------------------------------------------------
# small model builders
# ---------------------------------------------------------------------------------

def _ring_graph(n):
    cols = [np.array(sorted({(i - 1) % n, (i + 1) % n})) for i in range(n)]
    return CSR.from_rows(n, n, cols, [np.ones(len(c)) for c in cols])


def _dense_gauss_model(seed, n=12, m=30, tau=7.0, with_offset=True):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, (n, 2))
    cols = [np.array([rng.integers(0, n)]) for _ in range(m)]
    vals = [np.array([rng.uniform(0.5, 1.5)]) for _ in range(m)]
    A = CSR.from_rows(m, n, cols, vals)
    y = rng.standard_normal(m)
    off = 0.1 * rng.standard_normal(m) if with_offset else None
    blk = Block("dense_exp", n, points=pts, theta_sigma=0, theta_range_x=1, theta_range_y=2,
                theta_iid=3, nugget=1e-6)
    prior = [("gauss", 0.0, 1.0), ("gauss", -1.0, 0.5), ("gauss", -1.0, 0.5), ("pc_prec", 1.0, 0.01)]
    return ModelSpec("tiny_gauss", n, "gaussian", A, y, off, [blk], prior, lik_prec=tau)


def _structured_model(seed, likelihood, m=40):
    """intercept + ICAR(5) (eps) + iid(5) + RW1(4) (eps) + ICAR x RW1 (eps), with
    constraints that span the null space of every intrinsic block."""
    rng = np.random.default_rng(seed)
    g = _ring_graph(5)
    blocks = [Block("fixed", 1, prec=1e-3),
              Block("kron", 5, theta_idx=0, factors=[Factor("icar", 5, g)], eps=1e-5),
              Block("iid", 5, theta_idx=1),
              Block("kron", 4, theta_idx=2, factors=[Factor("rw1", 4)], eps=1e-5),
              Block("kron", 20, theta_idx=3, factors=[Factor("icar", 5, g), Factor("rw1", 4)], eps=1e-5)]
    n = 35
    cols, vals = [], []
    for i in range(m):
        s, t = rng.integers(0, 5), rng.integers(0, 4)
        cols.append(np.array([0, 1 + s, 6 + s, 11 + t, 15 + 4 * s + t]))
        vals.append(np.ones(5))
    A = CSR.from_rows(m, n, cols, vals)
    off = rng.normal(0.5, 0.2, m)
    if likelihood == "poisson":
        y = rng.poisson(np.exp(off + 0.3 * rng.standard_normal(m))).astype(float)
    else:
        y = off + rng.standard_normal(m)
    crow = [np.arange(1, 6), np.arange(11, 15)]
    crow += [np.array([15 + 4 * s + t for s in range(5)]) for t in range(4)]
    crow += [np.array([15 + 4 * s + t for t in range(4)]) for s in range(4)]
    C = CSR.from_rows(len(crow), n, crow, [np.ones(len(c)) for c in crow])
    prior = [("pc_prec", 1.0, 0.01)] * 4
    return ModelSpec("tiny_struct", n, likelihood, A, y, off, blocks, prior, C=C, lik_prec=3.0)


def _null_basis(C):
    """Orthonormal basis of {x : C x = 0} from the SVD of C."""
    u, s, vt = np.linalg.svd(C)
    r = int(np.sum(s > 1e-10 * s[0]))
    return vt[r:].T


# ---------------------------------------------------------------------------------
# closed forms: Gaussian likelihood (Laplace is exact)
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gaussian_marginal_likelihood_closed_form(seed):
    spec = _dense_gauss_model(seed)
    theta = np.array([0.2, np.log(0.3), np.log(0.15), np.log(5.0)])
    r = O.evaluate(spec, theta)
    # Sigma_x directly (no inversion): covariance of the latent field
    S = O.exp_covariance(spec.blocks[0], theta)
    A = spec.A.to_dense()
    cov_y = A @ S @ A.T + np.eye(spec.m) / spec.lik_prec
    ref = O.log_theta_prior(spec, theta) + multivariate_normal(spec.offset, cov_y).logpdf(spec.y)
    assert abs(r["log_post"] - ref) <= 1e-9 * max(1.0, abs(ref))
    # posterior mean and covariance by the covariance-form (Woodbury) route
    K = S @ A.T @ np.linalg.inv(cov_y)
    mean = K @ (spec.y - spec.offset)
    cov = S - K @ A @ S
    assert np.max(np.abs(r["x_hat"] - mean)) <= 1e-9 * np.max(np.abs(mean))
    assert np.max(np.abs(r["var"] - np.diag(cov)) / np.diag(cov)) <= 1e-8


def test_gaussian_constrained_closed_form():
    """Constrained Gaussian model: x = N z with N an orthonormal basis of null(C);
    z ~ N(0, (N^T Q_p N)^-1) is the prior conditioned on C x = 0, so
    y ~ N(o, A N (N^T Q_p N)^-1 N^T A^T + tau^-1 I) exactly."""
    spec = _structured_model(3, "gaussian")
    theta = np.array([0.5, 1.0, -0.3, 0.8])
    r = O.evaluate(spec, theta)
    Qp, _ = O.prior_precision(spec, theta)
    C = spec.C.to_dense()
    N = _null_basis(C)
    Sz = np.linalg.inv(N.T @ Qp @ N)
    A = spec.A.to_dense()
    AN = A @ N
    cov_y = AN @ Sz @ AN.T + np.eye(spec.m) / spec.lik_prec
    ref = O.log_theta_prior(spec, theta) + multivariate_normal(spec.offset, cov_y).logpdf(spec.y)
    assert abs(r["log_post"] - ref) <= 1e-8 * max(1.0, abs(ref))
    # posterior of z, mapped back: mode and marginal variances
    Pz = N.T @ Qp @ N + spec.lik_prec * AN.T @ AN
    z = np.linalg.solve(Pz, spec.lik_prec * AN.T @ (spec.y - spec.offset))
    assert np.max(np.abs(r["x_hat"] - N @ z)) <= 1e-8
    assert np.max(np.abs(C @ r["x_hat"])) <= 1e-10
    var = np.diag(N @ np.linalg.inv(Pz) @ N.T)
    assert np.max(np.abs(r["var"] - var) / var) <= 1e-6


# ---------------------------------------------------------------------------------
# brute force: Poisson Laplace approximation on tiny inputs
# ---------------------------------------------------------------------------------

def _fd_hessian(f, x, h=1e-4):
    d = x.size
    H = np.zeros((d, d))
    for i in range(d):
        for j in range(i, d):
            ei = np.zeros(d); ei[i] = h
            ej = np.zeros(d); ej[j] = h
            H[i, j] = H[j, i] = (f(x + ei + ej) - f(x + ei - ej) - f(x - ei + ej) + f(x - ei - ej)) / (4 * h * h)
    return H


def _laplace_bruteforce(spec, theta, N=None):
    """Mode by scipy BFGS and the Hessian by finite differences, both in the
    coordinates x = N z (N = I without constraints)."""
    Qp, logdet_Qp = O.prior_precision(spec, theta)
    A = spec.A.to_dense()
    off = np.zeros(spec.m) if spec.offset is None else spec.offset
    N = np.eye(spec.n) if N is None else N

    def f(z):
        x = N @ z
        eta = A @ x + off
        return float(np.sum(spec.y * eta - np.exp(eta)) - 0.5 * x @ Qp @ x)

    def g(z):
        x = N @ z
        eta = A @ x + off
        return N.T @ (A.T @ (spec.y - np.exp(eta)) - Qp @ x)

    res = so.minimize(lambda z: -f(z), np.zeros(N.shape[1]), jac=lambda z: -g(z), method="BFGS",
                      options=dict(gtol=1e-11, maxiter=10000))
    z = res.x
    H = -_fd_hessian(f, z)
    x = N @ z
    const = -float(np.sum(__import__("scipy.special", fromlist=["gammaln"]).gammaln(spec.y + 1)))
    lp = (O.log_theta_prior(spec, theta) + f(z) + const
          + 0.5 * np.linalg.slogdet(N.T @ Qp @ N)[1] - 0.5 * np.linalg.slogdet(H)[1])
    return lp, x


def test_poisson_laplace_bruteforce_unconstrained():
    rng = np.random.default_rng(7)
    n, m = 4, 9
    cols = [np.array([0, 1 + rng.integers(0, 3)]) for _ in range(m)]
    A = CSR.from_rows(m, n, cols, [np.array([1.0, rng.uniform(0.5, 1.5)]) for _ in range(m)])
    y = rng.poisson(2.0, m).astype(float)
    blocks = [Block("fixed", 1, prec=1e-3), Block("iid", 3, theta_idx=0)]
    spec = ModelSpec("tiny_pois", n, "poisson", A, y, None, blocks, [("pc_prec", 1.0, 0.01)])
    theta = np.array([0.7])
    r = O.evaluate(spec, theta)
    ref, x = _laplace_bruteforce(spec, theta)
    assert np.max(np.abs(r["x_hat"] - x)) < 1e-6
    assert abs(r["log_post"] - ref) < 1e-5
    # Newton converged to a stationary point of the log posterior
    As = sp.csr_matrix(spec.A.to_dense())
    Qp, _ = O.prior_precision(spec, theta)
    grad = As.T @ (y - np.exp(As @ r["x_hat"])) - Qp @ r["x_hat"]
    assert np.max(np.abs(grad)) < 1e-9


def test_poisson_laplace_bruteforce_constrained():
    spec = _structured_model(11, "poisson", m=30)
    theta = np.array([0.3, 1.2, -0.2, 0.5])
    r = O.evaluate(spec, theta)
    N = _null_basis(spec.C.to_dense())
    ref, x = _laplace_bruteforce(spec, theta, N)
    assert np.max(np.abs(r["x_hat"] - x)) < 1e-6
    assert abs(r["log_post"] - ref) < 1e-5
    assert np.max(np.abs(spec.C.to_dense() @ r["x_hat"])) < 1e-10


# ---------------------------------------------------------------------------------
# determinants / inverses by an independent route
# ---------------------------------------------------------------------------------

def test_prior_logdet_by_eigenvalues():
    spec = _structured_model(5, "poisson")
    theta = np.array([0.1, -0.4, 0.9, 1.3])
    Qp, logdet = O.prior_precision(spec, theta)
    # Kronecker blocks: eigenvalues of R1 kron R2 are the products of the factors'
    ld = 0.0
    for blk in spec.blocks:
        if blk.kind == "fixed":
            ld += blk.size * math.log(blk.prec)
        elif blk.kind == "iid":
            ld += blk.size * theta[blk.theta_idx]
        else:
            ev = np.ones(1)
            for f in blk.factors:
                ev = np.kron(ev, np.linalg.eigvalsh(O.structure_matrix(f)))
            ld += np.sum(np.log(math.exp(theta[blk.theta_idx]) * np.clip(ev, 0, None) + blk.eps))
    assert abs(logdet - ld) < 1e-8 * abs(ld)
    assert abs(logdet - np.sum(np.log(np.linalg.eigvalsh(Qp)))) < 1e-8 * abs(ld)


def test_dense_block_precision_is_inverse_covariance():
    spec = _dense_gauss_model(4, n=20)
    theta = np.array([-0.3, np.log(0.4), np.log(0.2), np.log(2.0)])
    Qp, logdet = O.prior_precision(spec, theta)
    S = O.exp_covariance(spec.blocks[0], theta)
    assert np.max(np.abs(Qp @ S - np.eye(20))) < 1e-9
    assert abs(logdet + np.sum(np.log(np.linalg.eigvalsh(S)))) < 1e-9 * abs(logdet)
    # covariance: distance-1 points correlate by exp(-1) (closed-form special case)
    blk = Block("dense_exp", 2, points=np.array([[0.0, 0.0], [0.3, 0.0]]), theta_sigma=0,
                theta_range_x=1, theta_range_y=2, nugget=0.0)
    S2 = O.exp_covariance(blk, np.array([0.0, np.log(0.3), np.log(5.0)]))
    assert abs(S2[0, 1] - math.exp(-1.0)) < 1e-15


# ---------------------------------------------------------------------------------
# hyperparameter prior
# ---------------------------------------------------------------------------------

def test_pc_prior_normalised_and_tail_probability():
    spec = ModelSpec("p", 1, "poisson", CSR(0, 1, np.zeros(1, np.int64), np.zeros(0, np.int32),
                     np.zeros(0)), np.zeros(0), None, [], [("pc_prec", 1.0, 0.01)])
    dens = lambda t: math.exp(O.log_theta_prior(spec, [t]))
    total = quad(dens, -40, 60, limit=400)[0]
    assert abs(total - 1.0) < 1e-8
    # P(sigma > U) = P(theta < -2 log U) = alpha, with U = 1
    assert abs(quad(dens, -60, 0.0, limit=400)[0] - 0.01) < 1e-8
    g = ModelSpec("g", 1, "poisson", spec.A, np.zeros(0), None, [], [("gauss", 0.5, 2.0)])
    assert abs(O.log_theta_prior(g, [1.5]) - math.log(0.5 / math.sqrt(2 * math.pi)
                                                      * math.exp(-0.125))) < 1e-14


# ---------------------------------------------------------------------------------
# constraint counts of Section 5.2 and the workload's constraint matrix
# ---------------------------------------------------------------------------------

def _rank(R, tol=1e-9):
    ev = np.linalg.eigvalsh(R)
    return int(np.sum(ev > tol * ev[-1]))


def test_constraint_counts_match_null_space_dimensions():
    rng = np.random.default_rng(0)
    Rs = O.structure_matrix(Factor("icar", 50, synth.delaunay_graph(rng, 50)))
    rs = _rank(Rs)
    assert rs == 49  # connected planar graph
    # Spain model: RW1 time (25) x RW1 age (9) x Besag space (50), mains + pairwise + 3-way
    rt, ra = _rank(O.structure_matrix(Factor("rw1", 25))), _rank(O.structure_matrix(Factor("rw1", 9)))
    nt, na, ns = 25, 9, 50
    null = lambda sizes, ranks: int(np.prod(sizes) - np.prod(ranks))
    k = (3 + null([nt, na], [rt, ra]) + null([nt, ns], [rt, rs]) + null([ns, na], [rs, ra])
         + null([ns, nt, na], [rs, rt, ra]))
    # paper's per-term formulas n_t n_a - (n_t-1)(n_a-1) etc. and its total
    assert null([nt, na], [rt, ra]) == nt * na - (nt - 1) * (na - 1)
    assert k == 2010
    # Table 3: RW2 time (5) + Besag space (200) + time x space: k = n_t + 2 n_s + 1
    for ns_ in (200, 400, 800):
        g = synth.delaunay_graph(np.random.default_rng(ns_), ns_)
        rs_ = _rank(O.structure_matrix(Factor("icar", ns_, g)))
        rt2 = _rank(O.structure_matrix(Factor("rw2", 5)))
        k3 = (5 - rt2) + (ns_ - rs_) + null([5, ns_], [rt2, rs_])
        assert k3 == 5 + 2 * ns_ + 1
    assert [5 + 2 * s + 1 for s in (200, 400, 800)] == [406, 806, 1606]


def test_workload_constraints_span_the_intrinsic_null_spaces():
    spec, _ = synth.spacetime_n8149_m8000_fd13()
    C = sp.csr_matrix((spec.C.val, spec.C.col, spec.C.rowptr), shape=(spec.k, spec.n))
    assert spec.k == 1486 and spec.n == 8149
    # C Q_p = eps C for the intrinsic blocks, i.e. C R = 0 blockwise
    start = 0
    R_blocks = []
    for blk in spec.blocks:
        if blk.kind == "kron":
            R = sp.csr_matrix(np.ones((1, 1)))
            for f in blk.factors:
                R = sp.kron(R, sp.csr_matrix(O.structure_matrix(f)))
            R_blocks.append(R)
        else:
            R_blocks.append(sp.csr_matrix((blk.size, blk.size)))
        start += blk.size
    R = sp.block_diag(R_blocks).tocsr()
    assert abs(C @ R).max() < 1e-12
    # full row rank: C C^T is positive definite
    CCt = (C @ C.T).toarray()
    assert np.all(np.diag(np.linalg.cholesky(CCt)) > 1e-8)


# ---------------------------------------------------------------------------------
# structure matrices by value (Section 5.1 structures; Appendix C prints RW1(4))
# ---------------------------------------------------------------------------------

def test_rw1_structure_equals_appendix_c_printed_precision():
    """Appendix C's prior precision Q_e of four effects is the RW1 structure of size 4."""
    g = _read_golden("appendix_c_example.txt")
    R = O.structure_matrix(Factor("rw1", 4))
    assert np.array_equal(R, g["Qe"])


def test_rw2_structure_is_the_second_difference_stencil():
    """RW2 of size 5, written out by hand: the boundary rows (1, -2, 1) and (-2, 5, -4, 1),
    the interior row (1, -4, 6, -4, 1), and their mirror images."""
    R_hand = np.array([[1, -2, 1, 0, 0],
                       [-2, 5, -4, 1, 0],
                       [1, -4, 6, -4, 1],
                       [0, 1, -4, 5, -2],
                       [0, 0, 1, -2, 1]], dtype=float)
    assert np.array_equal(O.structure_matrix(Factor("rw2", 5)), R_hand)


def test_icar_structure_is_degree_minus_adjacency_by_hand():
    """Besag/ICAR on a hand-drawn 5-node graph with edges 0-1, 0-2, 1-2, 2-3, 3-4: the
    diagonal holds the neighbour counts (2, 2, 3, 2, 1), each edge a -1."""
    edges = [(0, 1), (0, 2), (1, 2), (2, 3), (3, 4)]
    nbrs = [sorted([b for a, b in edges if a == i] + [a for a, b in edges if b == i]) for i in range(5)]
    graph = CSR.from_rows(5, 5, [np.array(v) for v in nbrs], [np.ones(len(v)) for v in nbrs])
    R_hand = np.array([[2, -1, -1, 0, 0],
                       [-1, 2, -1, 0, 0],
                       [-1, -1, 3, -1, 0],
                       [0, 0, -1, 2, -1],
                       [0, 0, 0, -1, 1]], dtype=float)
    assert np.array_equal(O.structure_matrix(Factor("icar", 5, graph)), R_hand)
    assert np.array_equal(O.structure_matrix(Factor("iid", 3)), np.eye(3))


def test_kronecker_block_entries_follow_the_latent_order():
    """A kron block of factors (F1, F2) orders the latent effects with the last factor
    fastest: entry ((i1, i2), (j1, j2)) at (i1 n2 + i2, j1 n2 + j2) is
    tau R1[i1, j1] R2[i2, j2] (+ eps on the diagonal); checked entry by entry on RW1(3) x
    RW2(4) against the hand-written stencils, tau = 2, eps = 0.5."""
    rw1 = {(0, 0): 1, (1, 1): 2, (2, 2): 1, (0, 1): -1, (1, 0): -1, (1, 2): -1, (2, 1): -1}
    rw2 = np.array([[1, -2, 1, 0], [-2, 5, -4, 1], [1, -4, 5, -2], [0, 1, -2, 1]], dtype=float)
    blk = Block("kron", 12, theta_idx=0, factors=[Factor("rw1", 3), Factor("rw2", 4)], eps=0.5)
    spec = ModelSpec("kron_pin", 12, "gaussian", CSR(0, 12, np.zeros(1, np.int64), np.zeros(0, np.int32),
                                                      np.zeros(0)), np.zeros(0), None, [blk], [("gauss", 0, 1)])
    Qp, logdet = O.prior_precision(spec, np.array([math.log(2.0)]))
    for i1 in range(3):
        for i2 in range(4):
            for j1 in range(3):
                for j2 in range(4):
                    want = 2.0 * rw1.get((i1, j1), 0) * rw2[i2, j2] + (0.5 if (i1, i2) == (j1, j2) else 0.0)
                    assert Qp[i1 * 4 + i2, j1 * 4 + j2] == pytest.approx(want, abs=1e-14)
    assert logdet == pytest.approx(np.linalg.slogdet(Qp)[1], rel=1e-12)


# ---------------------------------------------------------------------------------
# invariance
# ---------------------------------------------------------------------------------

def test_log_post_invariant_to_latent_permutation():
    spec, thetas = synth.poisson_n256_m1000_5pts()
    r = O.evaluate(spec, thetas[1], want_var=True)
    perm = np.random.default_rng(3).permutation(255)
    blk = spec.blocks[1]
    pts = blk.points[perm]
    inv = np.argsort(perm)
    col = spec.A.col.copy()
    mask = col >= 1
    col[mask] = 1 + inv[col[mask] - 1]
    A2 = CSR(spec.A.nrows, spec.A.ncols, spec.A.rowptr, col, spec.A.val)
    b2 = Block("dense_exp", 255, points=pts, theta_sigma=0, theta_range_x=1, theta_range_y=1,
               nugget=blk.nugget)
    spec2 = ModelSpec("perm", spec.n, "poisson", A2, spec.y, None, [spec.blocks[0], b2],
                      spec.theta_prior)
    r2 = O.evaluate(spec2, thetas[1])
    assert abs(r["log_post"] - r2["log_post"]) < 1e-9 * abs(r["log_post"])
    assert np.max(np.abs(r["x_hat"][1:][perm] - r2["x_hat"][1:])) < 1e-9
    assert np.max(np.abs(r["var"][1:][perm] / r2["var"][1:] - 1)) < 1e-9


# ---------------------------------------------------------------------------------
# stage 2: Hessian, exploration points, integrated latent marginals
# ---------------------------------------------------------------------------------

def test_ccd_design_counts_and_gaussian_moments():
    """45 CCD points for t = 6 (the number the paper's hyperparameter exploration cites, with
    the half fraction of the factorial part); for every t, an exactly Gaussian pi(theta|y)
    (log density -|z|^2 / 2) weighted by the design's quadrature weights has mean 0 and
    covariance I, the moments of N(0, I)."""
    assert len(O.ccd_design(6)[0]) == 45
    assert [len(O.ccd_design(t)[0]) for t in (2, 3, 4, 5)] == [9, 15, 25, 27]
    for t in (2, 3, 4, 5, 6):
        Z, d = O.ccd_design(t)
        w = d * np.exp(-0.5 * np.sum(Z * Z, axis=1))
        w /= w.sum()
        assert np.max(np.abs(w @ Z)) < 1e-12
        assert np.max(np.abs((Z * w[:, None]).T @ Z - np.eye(t))) < 1e-12


def test_hessian_fd_exact_on_quadratics_and_second_order_on_cubics():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((3, 3))
    M = M + M.T
    b = rng.standard_normal(3)
    x0 = rng.standard_normal(3)
    H = O.hessian_fd(lambda x: 0.5 * x @ M @ x + b @ x + 3.0, x0, 0.1)
    assert np.max(np.abs(H - M)) < 1e-12
    # cubic term c (x . u)^3: exact Hessian 6 c (x . u) u u^T; central differences carry
    # an O(h^2) error on the off-diagonal only in the mixed fourth-order terms (here zero)
    u = np.array([0.3, -0.2, 0.5])
    f = lambda x: (x @ u) ** 3
    H = O.hessian_fd(f, x0, 1e-3)
    assert np.max(np.abs(H - 6.0 * (x0 @ u) * np.outer(u, u))) < 1e-7


def _iid_gauss_model(seed, n=6, m=15, tau_y=4.0):
    """Gaussian likelihood on one iid block of precision exp(theta): t = 1, every posterior
    quantity in closed form."""
    rng = np.random.default_rng(seed)
    cols = [np.array(sorted(rng.choice(n, 2, replace=False))) for _ in range(m)]
    vals = [rng.uniform(0.5, 1.5, 2) for _ in range(m)]
    A = CSR.from_rows(m, n, cols, vals)
    y = rng.standard_normal(m) * 1.5
    off = 0.2 * rng.standard_normal(m)
    # a Gaussian prior on the log precision keeps the posterior's tails light (with a PC prior
    # the right tail follows the prior's exp(-theta / 2) and no finite range holds the integral)
    return ModelSpec("iid_gauss", n, "gaussian", A, y, off, [Block("iid", n, theta_idx=0)],
                     [("gauss", 1.0, 0.7)], lik_prec=tau_y)


def test_grid_integration_matches_adaptive_quadrature_of_the_closed_forms():
    """For a Gaussian likelihood pi~(theta|y) and pi(x|theta, y) are exact, so the integrated
    marginals are the exact posterior moments of x_i.  The oracle's grid integration (dz = 0.2
    in the z-coordinates of the Laplace approximation, |z| <= 9) against adaptive quadrature
    over theta of the closed forms: pi(theta|y) from N(y; o, e^-theta A A^T + I / tau_y) and the
    Gaussian conditional moments of x."""
    spec = _iid_gauss_model(1)
    A = spec.A.to_dense()
    tau_y = spec.lik_prec

    def closed(theta):
        S = math.exp(-theta) * np.eye(spec.n)
        cov_y = A @ S @ A.T + np.eye(spec.m) / tau_y
        lp = O.log_theta_prior(spec, [theta]) + multivariate_normal(spec.offset, cov_y).logpdf(spec.y)
        K = S @ A.T @ np.linalg.inv(cov_y)
        mu = K @ (spec.y - spec.offset)
        var = np.diag(S - K @ A @ S)
        return lp, mu, var

    res = so.minimize_scalar(lambda th: -closed(th)[0], bounds=(-5, 8), method="bounded",
                             options=dict(xatol=1e-10))
    th_star = res.x
    negH = -O.hessian_fd(lambda th: O.evaluate(spec, th)["log_post"], np.array([th_star]), 1e-3)
    sd = 1.0 / math.sqrt(negH[0, 0])
    lp_star = closed(th_star)[0]
    lo, hi = th_star - 14 * sd, th_star + 14 * sd
    Zc = quad(lambda th: math.exp(closed(th)[0] - lp_star), lo, hi, epsabs=0, epsrel=1e-12, limit=200)[0]
    mean = np.array([quad(lambda th: closed(th)[1][i] * math.exp(closed(th)[0] - lp_star), lo, hi,
                          epsabs=0, epsrel=1e-12, limit=200)[0] for i in range(spec.n)]) / Zc
    second = np.array([quad(lambda th: (closed(th)[2][i] + closed(th)[1][i] ** 2) * math.exp(closed(th)[0] - lp_star),
                            lo, hi, epsabs=0, epsrel=1e-12, limit=200)[0] for i in range(spec.n)]) / Zc
    var = second - mean ** 2
    Z, d = O.grid_design(1, 0.2, 9.0)
    r = O.integrate_marginals(spec, np.array([th_star]), negH, Z, d)
    assert np.max(np.abs(r["mean"] - mean)) <= 1e-7 * np.max(np.abs(mean))
    assert np.max(np.abs(r["var"] / var - 1.0)) <= 1e-7


# ---------------------------------------------------------------------------------
# variational Bayes mean correction (Algorithm 2)
# ---------------------------------------------------------------------------------

def test_vb_gauss_hermite_means_match_the_lognormal_closed_form():
    """For a Poisson likelihood l''(eta) = e^eta, whose mean under N(nu, s^2) is e^(nu + s^2/2)."""
    spec, _ = synth.poisson_n256_m1000_5pts()
    rng = np.random.default_rng(8)
    nu = rng.normal(0.5, 1.0, spec.m)
    s2 = rng.uniform(0.01, 0.8, spec.m)
    I1, I2 = O.vb_expected_derivs(spec, nu, s2)
    closed = np.exp(nu + 0.5 * s2)
    assert np.max(np.abs(I2 / closed - 1.0)) < 1e-12
    assert np.max(np.abs(I1 - (closed - spec.y))) < 1e-12 * np.max(closed)


def test_vb_correction_vanishes_for_a_gaussian_likelihood():
    """With a Gaussian likelihood the Laplace mode is the exact posterior mean: c = 0 there, so
    Algorithm 2 stops after one step of size zero (to rounding)."""
    spec = _dense_gauss_model(2, with_offset=True)
    theta = np.array([0.2, np.log(0.3), np.log(0.15), np.log(5.0)])
    r = O.vb_mean(spec, theta)
    assert r["iters"] == 1
    assert np.max(np.abs(r["mean"] - r["laplace"]["x_hat"])) < 1e-12 * max(1.0, np.max(np.abs(r["mean"])))


def test_vb_mean_minimises_the_stated_objective_by_brute_force():
    """Tiny Poisson model: the fixed point of Algorithm 2 is the minimiser of
    E[-log pi(y|x)] + 1/2 mu^T Q_p mu under x ~ N(mu, Q*^-1) (Q* fixed at the Laplace mode),
    computed here by scipy with the closed-form lognormal expectation."""
    rng = np.random.default_rng(12)
    n, m = 6, 25
    cols = [np.array(sorted({0, 1 + rng.integers(0, n - 1)})) for _ in range(m)]
    A = CSR.from_rows(m, n, cols, [np.ones(len(c)) for c in cols])
    y = rng.poisson(2.0, m).astype(float)
    pts = rng.uniform(0, 1, (n - 1, 2))
    blocks = [Block("fixed", 1, prec=1e-3),
              Block("dense_exp", n - 1, points=pts, theta_sigma=0, theta_range_x=1, theta_range_y=1, nugget=1e-6)]
    spec = ModelSpec("vb_tiny", n, "poisson", A, y, None, blocks, [("gauss", 0.0, 1.0), ("gauss", 0.0, 1.0)])
    theta = np.array([-0.2, np.log(0.3)])
    r = O.vb_mean(spec, theta)
    Qp, _ = O.prior_precision(spec, theta)
    Ad = A.to_dense()
    s2 = r["sigma_eta2"]

    def F(mu):
        nu = Ad @ mu
        return float(np.sum(np.exp(nu + 0.5 * s2) - y * nu) + 0.5 * mu @ Qp @ mu)

    def G(mu):
        nu = Ad @ mu
        return Ad.T @ (np.exp(nu + 0.5 * s2) - y) + Qp @ mu

    res = so.minimize(F, r["laplace"]["x_hat"], jac=G, method="BFGS", options=dict(gtol=1e-12, maxiter=10000))
    assert np.max(np.abs(r["mean"] - res.x)) < 1e-7 * max(1.0, np.max(np.abs(res.x)))
    # the correction is not zero for a Poisson likelihood
    assert np.max(np.abs(r["mean"] - r["laplace"]["x_hat"])) > 1e-4


# ---------------------------------------------------------------------------------
# Moore-Penrose / Woodbury route (Section 3.1, Eq. (woodeqn))
# ---------------------------------------------------------------------------------

def test_woodbury_route_reproduces_appendix_c_and_the_kriging_limit():
    """The oracle's Eq. (woodeqn) on Appendix C's printed inputs gives the printed Sigma*; its
    pseudo-inverse of RW1(4) is the printed Q_e+; and on a constrained model its variances equal
    the kriging route's as eps -> 0 (eps = 1e-9 here: relative differences ~1e-6)."""
    g = _read_golden("appendix_c_example.txt")
    A, Ql, Qe = g["A"], np.diag(g["Ql"]), g["Qe"]
    P = np.linalg.pinv(Qe, hermitian=True)
    assert np.max(np.abs(P - g["Qe_pinv"])) <= 5e-4
    S = O.woodbury_covariance(P, A.T @ Ql @ A)
    assert np.max(np.abs(S - g["Sigma_star"])) <= 5e-4
    spec = _structured_model(3, "poisson")
    for blk in spec.blocks:
        if blk.kind == "kron":
            blk.eps = 1e-9
    theta = np.array([0.5, 1.0, -0.3, 0.8])
    wb = O.woodbury_marginals(spec, theta)
    kr = O.evaluate(spec, theta)
    assert np.max(np.abs(wb["var"] / kr["var"] - 1.0)) < 1e-5

// Model creation: validation, internal latent ordering, theta-independent precomputation
// and the copy of the model to the device.
//
// Internal latent order: the dense covariance block (if any) first, at offset 0, then the
// remaining blocks in the caller's order, then identity padding up to a multiple of PAD.
// Theta-independent structures built here:
//   * A (m x n_pad) in CSR and its transpose, for eta = A x and A^T r;
//   * the list of (row >= col) pairs of A^T diag(w) A with their contributions
//     (observation, A_ij A_ik), so that Q* = Q_p + A^T D A is a segmented sum;
//   * the structured prior entries a + b exp(theta_t) of Q_p (Section 5.1: tau R + eps I
//     with R = R_1 kron R_2 kron ..., ICAR R = D - W, RW1/RW2 R = D^T D);
//   * eigenvalues of each Kronecker structure (products of the factors' eigenvalues) for
//     log|tau R + eps I|; for a block whose constraint rows span the null space of R,
//     1/2 log|Q_b| + 1/2 log|C_b Q_b^-1 C_b^T| = 1/2 sum_{lambda>0} log(tau lambda + eps)
//     + 1/2 log|C_b C_b^T| exactly (the eps terms of the null directions cancel).
#include "kernels.h"
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>

namespace inla {

// cyclic Jacobi eigenvalues of a small symmetric matrix (row-major, n x n); with vecs, also the
// eigenvectors (columns of the accumulated rotations: a = V diag(ev) V^T)
static std::vector<double> jacobi_eigenvalues(std::vector<double> a, int n, std::vector<double>* vecs = nullptr) {
  if (vecs) {
    vecs->assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) (*vecs)[(size_t)i * n + i] = 1.0;
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += a[i * n + j] * a[i * n + j];
        if (i != j) off += a[i * n + j] * a[i * n + j];
      }
    if (off <= 1e-30 * (tot + 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[p * n + p], aqq = a[q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // rotate rows/cols p, q
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        if (vecs)
          for (int k = 0; k < n; ++k) {
            double* V = vecs->data();
            const double vkp = V[k * n + p], vkq = V[k * n + q];
            V[k * n + p] = c * vkp - s * vkq;
            V[k * n + q] = s * vkp + c * vkq;
          }
      }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
  return ev;
}

// dense structure matrix of one Kronecker factor
static int factor_matrix(const inla_factor& f, std::vector<double>& R) {
  const int n = f.size;
  if (n <= 0 || n > 4096) return INLA_E_BADARG;
  R.assign((size_t)n * n, 0.0);
  switch (f.kind) {
    case INLA_FACTOR_ICAR:
      if (!f.graph_rowptr || !f.graph_col) return INLA_E_BADARG;
      for (int i = 0; i < n; ++i)
        for (int64_t e = f.graph_rowptr[i]; e < f.graph_rowptr[i + 1]; ++e) {
          const int j = f.graph_col[e];
          if (j < 0 || j >= n || j == i) return INLA_E_BADARG;
          R[(size_t)i * n + j] -= 1.0;
          R[(size_t)i * n + i] += 1.0;
        }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j)
          if (R[(size_t)i * n + j] != R[(size_t)j * n + i]) return INLA_E_BADARG;  // graph must be symmetric
      return INLA_OK;
    case INLA_FACTOR_RW1:
    case INLA_FACTOR_RW2: {
      const int o = f.kind == INLA_FACTOR_RW1 ? 1 : 2;
      if (n <= o) return INLA_E_BADARG;
      // R = D^T D with D the (n-o) x n difference matrix of order o
      const double c1[2] = {-1.0, 1.0}, c2[3] = {1.0, -2.0, 1.0};
      const double* c = o == 1 ? c1 : c2;
      for (int r = 0; r + o < n; ++r)
        for (int a = 0; a <= o; ++a)
          for (int b = 0; b <= o; ++b) R[(size_t)(r + a) * n + (r + b)] += c[a] * c[b];
      return INLA_OK;
    }
    case INLA_FACTOR_IID:
      for (int i = 0; i < n; ++i) R[(size_t)i * n + i] = 1.0;
      return INLA_OK;
    default:
      return INLA_E_BADARG;
  }
}

template <typename T>
static int dev_copy(inla_model* M, T** dst, const T* src, size_t count) {
  *dst = nullptr;
  if (count == 0) return INLA_OK;
  void* p = nullptr;
  INLA_CUDA_TRY(cudaMalloc(&p, count * sizeof(T)));
  M->allocations.push_back(p);
  INLA_CUDA_TRY(cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice));
  *dst = static_cast<T*>(p);
  return INLA_OK;
}

int logdet_spd_device(const std::vector<double>& Mhost, int k, double* out);  // eval.cu

static int validate_csr(const int64_t* rowptr, const int32_t* col, const double* val, int64_t nrows, int64_t ncols) {
  if (!rowptr || !col || !val) return INLA_E_BADARG;
  if (rowptr[0] != 0) return INLA_E_BADARG;
  for (int64_t i = 0; i < nrows; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return INLA_E_BADARG;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (col[e] < 0 || col[e] >= ncols || !std::isfinite(val[e])) return INLA_E_BADARG;
      for (int64_t f = rowptr[i]; f < e; ++f)
        if (col[f] == col[e]) return INLA_E_BADARG;  // no duplicate columns in a row
    }
  }
  return INLA_OK;
}

static int create_impl(const inla_model_desc* D, inla_model* M) {
  ModelDev& d = M->d;
  std::memset(&d, 0, sizeof(d));
  if (D->n <= 0 || D->m < 0 || D->k < 0 || D->nblocks <= 0 || !D->blocks) return INLA_E_BADARG;
  if (D->theta_dim < 0 || D->theta_dim > MAX_THETA) return INLA_E_UNSUPPORTED;
  if (D->likelihood != INLA_LIK_POISSON && D->likelihood != INLA_LIK_GAUSSIAN) return INLA_E_BADARG;
  if (D->likelihood == INLA_LIK_GAUSSIAN && !(D->lik_prec > 0)) return INLA_E_BADARG;
  if (D->m > 0 && !D->y) return INLA_E_BADARG;
  if (D->m > 0) INLA_TRY(validate_csr(D->A_rowptr, D->A_col, D->A_val, D->m, D->n));
  if (D->k > 0) INLA_TRY(validate_csr(D->C_rowptr, D->C_col, D->C_val, D->k, D->n));
  for (int t = 0; t < D->theta_dim; ++t) {
    const int kd = D->theta_prior_kind[t];
    const double a = D->theta_prior_a[t], b = D->theta_prior_b[t];
    if (kd == INLA_PRIOR_GAUSS && !(b > 0)) return INLA_E_BADARG;
    if (kd == INLA_PRIOR_PC_PREC && !(a > 0 && b > 0 && b < 1)) return INLA_E_BADARG;
    if (kd != INLA_PRIOR_GAUSS && kd != INLA_PRIOR_PC_PREC) return INLA_E_BADARG;
    d.prior_kind[t] = kd;
    d.prior_a[t] = a;
    d.prior_b[t] = b;
  }
  for (int i = 0; i < D->m; ++i) {
    if (!std::isfinite(D->y[i])) return INLA_E_BADARG;
    if (D->likelihood == INLA_LIK_POISSON && (D->y[i] < 0 || D->y[i] != std::floor(D->y[i]))) return INLA_E_BADARG;
    if (D->offset && !std::isfinite(D->offset[i])) return INLA_E_BADARG;
  }
  const int n = D->n, m = D->m, k = D->k;
  auto theta_ok = [&](int t) { return t >= 0 && t < D->theta_dim; };

  // ---- blocks and internal order ----
  int dense_b = -1, total = 0;
  for (int b = 0; b < D->nblocks; ++b) {
    const inla_block& B = D->blocks[b];
    if (B.size <= 0) return INLA_E_BADARG;
    total += B.size;
    switch (B.kind) {
      case INLA_BLOCK_FIXED:
        if (!(B.prec > 0)) return INLA_E_BADARG;
        break;
      case INLA_BLOCK_IID:
        if (!theta_ok(B.theta_idx)) return INLA_E_BADARG;
        break;
      case INLA_BLOCK_DENSE_EXP:
        if (dense_b >= 0) return INLA_E_UNSUPPORTED;
        if (!B.points || !theta_ok(B.theta_sigma) || !theta_ok(B.theta_range_x) || !theta_ok(B.theta_range_y))
          return INLA_E_BADARG;
        if (B.theta_iid >= D->theta_dim || !(B.nugget >= 0)) return INLA_E_BADARG;
        dense_b = b;
        break;
      case INLA_BLOCK_KRON: {
        if (!theta_ok(B.theta_idx) || B.nfactors < 1 || B.nfactors > 3 || !B.factors || !(B.eps >= 0))
          return INLA_E_BADARG;
        int64_t prod = 1;
        for (int f = 0; f < B.nfactors; ++f) prod *= B.factors[f].size;
        if (prod != B.size) return INLA_E_BADARG;
        break;
      }
      default:
        return INLA_E_BADARG;
    }
  }
  if (total != n) return INLA_E_BADARG;
  std::vector<int> bstart(D->nblocks), bstart_int(D->nblocks);
  {
    int s = 0;
    for (int b = 0; b < D->nblocks; ++b) {
      bstart[b] = s;
      s += D->blocks[b].size;
    }
    // structured / fixed blocks first, the dense block last: an intercept (or any effect
    // observed by many rows) is then eliminated first with an exact large pivot, and the
    // near-null direction it shares with the dense field ends up in pivots of the dense
    // field's own scale instead of cancelling against the intercept's.
    int p = 0;
    for (int b = 0; b < D->nblocks; ++b)
      if (b != dense_b) {
        bstart_int[b] = p;
        p += D->blocks[b].size;
      }
    if (dense_b >= 0) bstart_int[dense_b] = p;
  }
  M->perm.assign(n, 0);
  std::vector<int> block_of_int(n);
  for (int b = 0; b < D->nblocks; ++b)
    for (int i = 0; i < D->blocks[b].size; ++i) {
      M->perm[bstart[b] + i] = bstart_int[b] + i;
      block_of_int[bstart_int[b] + i] = b;
    }
  d.n = n;
  d.m = m;
  d.k = k;
  d.n_pad = (int)round_up(n, PAD);
  d.k_pad = k > 0 ? (int)round_up(k, PAD) : 0;
  d.nd = dense_b >= 0 ? D->blocks[dense_b].size : 0;
  d.nd_pad = d.nd > 0 ? (int)round_up(d.nd, PAD) : 0;
  d.nd_off = dense_b >= 0 ? bstart_int[dense_b] : 0;
  d.likelihood = D->likelihood;
  d.lik_prec = D->lik_prec;
  d.theta_dim = D->theta_dim;
  const int n_pad = d.n_pad;
  const auto& perm = M->perm;

  // ---- likelihood structures ----
  std::vector<int64_t> Arp(m + 1, 0);
  std::vector<int32_t> Acol;
  std::vector<double> Aval;
  Acol.reserve(m > 0 ? D->A_rowptr[m] : 0);
  for (int i = 0; i < m; ++i) {
    for (int64_t e = D->A_rowptr[i]; e < D->A_rowptr[i + 1]; ++e) {
      Acol.push_back(perm[D->A_col[e]]);
      Aval.push_back(D->A_val[e]);
    }
    Arp[i + 1] = (int64_t)Acol.size();
  }
  std::vector<int64_t> Atp(n_pad + 1, 0);
  for (int32_t c : Acol) Atp[c + 1]++;
  for (int j = 0; j < n_pad; ++j) Atp[j + 1] += Atp[j];
  std::vector<int32_t> Atr(Acol.size());
  std::vector<double> Atv(Acol.size());
  {
    std::vector<int64_t> pos(Atp.begin(), Atp.end() - 1);
    for (int i = 0; i < m; ++i)
      for (int64_t e = Arp[i]; e < Arp[i + 1]; ++e) {
        const int64_t q = pos[Acol[e]]++;
        Atr[q] = i;
        Atv[q] = Aval[e];
      }
  }
  struct Contrib {
    int64_t key;
    int32_t obs;
    double coef;
  };
  // the contributions ordered by (row, column) of the pair, observations ascending within a pair:
  // a counting sort by the row (observations are visited in order, so each row's bucket is
  // already ordered by observation), then a stable sort by column inside the buckets that need it
  std::vector<Contrib> con;
  {
    auto for_each_pair = [&](auto&& f) {
      for (int i = 0; i < m; ++i)
        for (int64_t a = Arp[i]; a < Arp[i + 1]; ++a)
          for (int64_t b = Arp[i]; b < Arp[i + 1]; ++b) {
            const int ca = Acol[a], cb = Acol[b];
            if (ca < cb || (ca == cb && a != b)) continue;
            f(i, ca, cb, Aval[a] * Aval[b]);
          }
    };
    std::vector<int64_t> start((size_t)n_pad + 1, 0);
    for_each_pair([&](int, int ca, int, double) { ++start[(size_t)ca + 1]; });
    for (int j = 0; j < n_pad; ++j) start[j + 1] += start[j];
    con.resize((size_t)start[n_pad]);
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for_each_pair([&](int i, int ca, int cb, double v) {
      con[(size_t)fill[ca]++] = Contrib{(int64_t)ca * n_pad + cb, i, v};
    });
    for (int j = 0; j < n_pad; ++j) {
      auto lo = con.begin() + start[j], hi = con.begin() + start[j + 1];
      if (!std::is_sorted(lo, hi, [](const Contrib& x, const Contrib& y) { return x.key < y.key; }))
        std::stable_sort(lo, hi, [](const Contrib& x, const Contrib& y) { return x.key < y.key; });
    }
  }
  std::vector<int32_t> prow, pcol, pobs;
  std::vector<int64_t> pptr;
  std::vector<double> pcoef;
  for (size_t c = 0; c < con.size(); ++c) {
    if (c == 0 || con[c].key != con[c - 1].key) {
      prow.push_back((int32_t)(con[c].key / n_pad));
      pcol.push_back((int32_t)(con[c].key % n_pad));
      pptr.push_back((int64_t)c);
    }
    pobs.push_back(con[c].obs);
    pcoef.push_back(con[c].coef);
  }
  pptr.push_back((int64_t)con.size());
  d.npairs = (int64_t)prow.size();
  std::vector<int32_t> heavy_cols;
  for (int j = 0; j < n_pad; ++j)
    if (Atp[j + 1] - Atp[j] > HEAVY_LEN) heavy_cols.push_back(j);
  std::vector<int64_t> heavy_pairs;
  for (int64_t q = 0; q < d.npairs; ++q)
    if (pptr[q + 1] - pptr[q] > HEAVY_LEN) heavy_pairs.push_back(q);
  d.n_heavy_cols = (int32_t)heavy_cols.size();
  d.n_heavy_pairs = (int32_t)heavy_pairs.size();
  std::vector<int64_t> optr((size_t)m + 1, 0);
  for (size_t c = 0; c < con.size(); ++c) optr[(size_t)con[c].obs + 1]++;
  for (int i = 0; i < m; ++i) optr[i + 1] += optr[i];
  std::vector<int32_t> opair(con.size());
  std::vector<double> ocoef(con.size());
  {
    std::vector<int64_t> fill(optr.begin(), optr.end() - 1);
    for (int64_t q = 0; q < d.npairs; ++q)
      for (int64_t c = pptr[q]; c < pptr[q + 1]; ++c) {
        const int64_t at = fill[pobs[c]]++;
        opair[at] = (int32_t)q;
        ocoef[at] = pcoef[c] * (prow[q] != pcol[q] ? 2.0 : 1.0);
      }
  }
  if (D->likelihood == INLA_LIK_POISSON) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += std::lgamma(D->y[i] + 1.0);
    d.lgamma_sum = s;
  }

  // ---- structured prior entries, Kronecker eigenvalues ----
  std::vector<PriorEntry> ent;
  std::vector<double> eig;
  double const_logdet = 0.0;
  std::vector<int> constrained_block(D->nblocks, 0);
  // which block each constraint row lies in
  std::vector<int> crow_block(k, -1);
  for (int r = 0; r < k; ++r) {
    for (int64_t e = D->C_rowptr[r]; e < D->C_rowptr[r + 1]; ++e) {
      const int b = block_of_int[perm[D->C_col[e]]];
      if (crow_block[r] < 0) crow_block[r] = b;
      if (crow_block[r] != b) return INLA_E_UNSUPPORTED;
    }
    if (crow_block[r] < 0) return INLA_E_BADARG;  // empty constraint row
    if (D->blocks[crow_block[r]].kind != INLA_BLOCK_KRON) return INLA_E_UNSUPPORTED;
    constrained_block[crow_block[r]]++;
  }
  // per block in internal order, for the Moore-Penrose route: kind, offset, size, and the
  // factors' pseudo-inverses of the Kronecker blocks
  if (D->nblocks > MAX_BLOCKS) return INLA_E_UNSUPPORTED;
  std::vector<BlockInfo> binfo(D->nblocks);
  std::vector<double> pinv;
  for (int b = 0; b < D->nblocks; ++b) {
    const inla_block& B = D->blocks[b];
    BlockInfo& bi = binfo[b];
    std::memset(&bi, 0, sizeof(bi));
    bi.kind = B.kind;
    bi.off = bstart_int[b];
    bi.size = B.size;
    bi.theta_idx = B.kind == INLA_BLOCK_FIXED ? -1 : B.theta_idx;
    bi.prec = B.prec;
  }
  for (int b = 0; b < D->nblocks; ++b) {
    const inla_block& B = D->blocks[b];
    const int s0 = bstart_int[b];
    if (B.kind == INLA_BLOCK_FIXED) {
      for (int i = 0; i < B.size; ++i) ent.push_back(PriorEntry{s0 + i, s0 + i, -1, 0, B.prec, 0.0});
      const_logdet += B.size * std::log(B.prec);
    } else if (B.kind == INLA_BLOCK_IID) {
      for (int i = 0; i < B.size; ++i) ent.push_back(PriorEntry{s0 + i, s0 + i, B.theta_idx, 0, 0.0, 1.0});
      if (d.n_iid >= MAX_KRON) return INLA_E_UNSUPPORTED;
      d.iid_theta[d.n_iid] = B.theta_idx;
      d.iid_size[d.n_iid] = B.size;
      d.n_iid++;
    } else if (B.kind == INLA_BLOCK_KRON) {
      if (d.nkron >= MAX_KRON) return INLA_E_UNSUPPORTED;
      const int nf = B.nfactors;
      std::vector<std::vector<double>> R(nf);
      std::vector<std::vector<double>> ev(nf);
      for (int f = 0; f < nf; ++f) {
        INLA_TRY(factor_matrix(B.factors[f], R[f]));
        std::vector<double> V;
        const int fs = B.factors[f].size;
        ev[f] = jacobi_eigenvalues(R[f], fs, &V);
        double mx = 0.0;
        for (double v : ev[f]) mx = std::max(mx, std::fabs(v));
        for (double& v : ev[f])
          if (std::fabs(v) <= 1e-9 * mx) v = 0.0;
          else if (v < 0) return INLA_E_BADARG;  // structure must be positive semi-definite
        // Moore-Penrose pseudo-inverse of the factor: sum over the nonzero eigenvalues of
        // v v^T / lambda (the pseudo-inverse of a Kronecker product is that of the factors)
        BlockInfo& bi = binfo[b];
        bi.pinv_off[f] = (int64_t)pinv.size();
        bi.fsize[f] = fs;
        for (int i = 0; i < fs; ++i)
          for (int j = 0; j < fs; ++j) {
            double a = 0.0;
            for (int e = 0; e < fs; ++e)
              if (ev[f][e] != 0.0) a += V[(size_t)i * fs + e] * V[(size_t)j * fs + e] / ev[f][e];
            pinv.push_back(a);
          }
      }
      binfo[b].nf = nf;
      // sparse Kronecker product, lower triangle, every diagonal present
      int sz[3] = {1, 1, 1};
      for (int f = 0; f < nf; ++f) sz[f + (3 - nf)] = B.factors[f].size;
      auto Rf = [&](int f, int i, int j) -> double {
        const int ff = f - (3 - nf);
        if (ff < 0) return 1.0;
        return R[ff][(size_t)i * sz[f] + j];
      };
      // enumerate nonzeros factor by factor
      std::vector<std::vector<std::pair<int, int>>> nz(3);
      for (int f = 0; f < 3; ++f)
        for (int i = 0; i < sz[f]; ++i)
          for (int j = 0; j < sz[f]; ++j)
            if (Rf(f, i, j) != 0.0 || i == j) nz[f].push_back({i, j});
      for (auto& a : nz[0])
        for (auto& bq : nz[1])
          for (auto& c : nz[2]) {
            const int i = (a.first * sz[1] + bq.first) * sz[2] + c.first;
            const int j = (a.second * sz[1] + bq.second) * sz[2] + c.second;
            if (j > i) continue;
            const double v = Rf(0, a.first, a.second) * Rf(1, bq.first, bq.second) * Rf(2, c.first, c.second);
            if (v == 0.0 && i != j) continue;
            ent.push_back(PriorEntry{s0 + i, s0 + j, B.theta_idx, 0, i == j ? B.eps : 0.0, v});
          }
      KronLogdet kl;
      kl.offset = (int32_t)eig.size();
      kl.size = B.size;
      kl.theta_idx = B.theta_idx;
      kl.eps = B.eps;
      int64_t nzero = 0;
      auto lam = [&](int p, int i) { const int ff = p - (3 - nf); return ff < 0 ? 1.0 : ev[ff][i]; };
      for (int i1 = 0; i1 < sz[0]; ++i1)
        for (int i2 = 0; i2 < sz[1]; ++i2)
          for (int i3 = 0; i3 < sz[2]; ++i3) {
            const double v = lam(0, i1) * lam(1, i2) * lam(2, i3);
            eig.push_back(v);
            nzero += (v == 0.0);
          }
      kl.constrained = constrained_block[b] > 0;
      if (kl.constrained) {
        if (constrained_block[b] != nzero) return INLA_E_UNSUPPORTED;
        // every constraint row of this block must be annihilated by R (C_b R_b = 0)
        std::map<int, std::vector<std::pair<int, double>>> rows_by_col;  // R rows (local)
        for (const auto& pe : ent)
          if (pe.row >= s0 && pe.row < s0 + B.size && pe.b != 0.0) {
            rows_by_col[pe.row - s0].push_back({pe.col - s0, pe.b});
            if (pe.row != pe.col) rows_by_col[pe.col - s0].push_back({pe.row - s0, pe.b});
          }
        for (int r = 0; r < k; ++r) {
          if (crow_block[r] != b) continue;
          std::map<int, double> acc;
          double scale = 0.0;
          for (int64_t e = D->C_rowptr[r]; e < D->C_rowptr[r + 1]; ++e) {
            const int l = perm[D->C_col[e]] - s0;
            scale = std::max(scale, std::fabs(D->C_val[e]));
            for (auto& pr : rows_by_col[l]) acc[pr.first] += D->C_val[e] * pr.second;
          }
          for (auto& kv : acc)
            if (std::fabs(kv.second) > 1e-8 * scale * 16.0) return INLA_E_UNSUPPORTED;
        }
      }
      d.kron[d.nkron++] = kl;
    }
  }
  for (int i = n; i < n_pad; ++i) ent.push_back(PriorEntry{i, i, -1, 0, 1.0, 0.0});
  d.nentries = (int64_t)ent.size();
  // gamma C^T C (lower triangle, internal indices): added to Q* for the constrained solves.
  // For x with C x = 0 it changes neither the kriged mode, nor the constrained covariance
  // N (N^T Q* N)^-1 N^T, nor log|Q*| + log|C Q*^-1 C^T| = log|N^T Q* N| + log|C C^T|
  // (N an orthonormal basis of null(C)); it lifts the eps-sized eigenvalues of Q* along the
  // intrinsic null directions to O(gamma), which the reduced-precision factor needs.
  std::vector<PriorEntry> cct;
  if (k > 0) {
    std::map<int64_t, double> acc;
    for (int r = 0; r < k; ++r)
      for (int64_t a = D->C_rowptr[r]; a < D->C_rowptr[r + 1]; ++a)
        for (int64_t b = D->C_rowptr[r]; b < D->C_rowptr[r + 1]; ++b) {
          const int ia = perm[D->C_col[a]], ib = perm[D->C_col[b]];
          if (ia < ib) continue;
          acc[(int64_t)ia * n_pad + ib] += D->C_val[a] * D->C_val[b];
        }
    for (auto& kv : acc) cct.push_back(PriorEntry{(int32_t)(kv.first / n_pad), (int32_t)(kv.first % n_pad), -1, 0, kv.second, 0.0});
  }
  d.ncct = (int64_t)cct.size();
  d.gamma_c = 1.0;
  d.prior_const_logdet = const_logdet;
  d.logdet_CCt = 0.0;
  if (k > 0) {
    // log|C C^T| on the device (FP64 Cholesky); C C^T is dense k x k here
    std::vector<std::map<int, double>> crow(k);
    std::vector<std::vector<std::pair<int, double>>> by_col(n);
    for (int r = 0; r < k; ++r)
      for (int64_t e = D->C_rowptr[r]; e < D->C_rowptr[r + 1]; ++e) by_col[D->C_col[e]].push_back({r, D->C_val[e]});
    std::vector<double> CCt((size_t)d.k_pad * d.k_pad, 0.0);
    for (int j = 0; j < n; ++j)
      for (auto& a : by_col[j])
        for (auto& bq : by_col[j]) CCt[(size_t)a.first * d.k_pad + bq.first] += a.second * bq.second;
    for (int r = k; r < d.k_pad; ++r) CCt[(size_t)r * d.k_pad + r] = 1.0;
    INLA_TRY(logdet_spd_device(CCt, d.k_pad, &d.logdet_CCt));
  }

  // ---- device copies ----
  INLA_TRY(dev_copy(M, &d.A_rowptr, Arp.data(), Arp.size()));
  INLA_TRY(dev_copy(M, &d.A_col, Acol.data(), Acol.size()));
  INLA_TRY(dev_copy(M, &d.A_val, Aval.data(), Aval.size()));
  INLA_TRY(dev_copy(M, &d.At_rowptr, Atp.data(), Atp.size()));
  INLA_TRY(dev_copy(M, &d.At_row, Atr.data(), Atr.size()));
  INLA_TRY(dev_copy(M, &d.At_val, Atv.data(), Atv.size()));
  INLA_TRY(dev_copy(M, &d.pair_row, prow.data(), prow.size()));
  INLA_TRY(dev_copy(M, &d.pair_col, pcol.data(), pcol.size()));
  INLA_TRY(dev_copy(M, &d.pair_ptr, pptr.data(), pptr.size()));
  INLA_TRY(dev_copy(M, &d.pc_obs, pobs.data(), pobs.size()));
  INLA_TRY(dev_copy(M, &d.pc_coef, pcoef.data(), pcoef.size()));
  INLA_TRY(dev_copy(M, &d.heavy_cols, heavy_cols.data(), heavy_cols.size()));
  d.nblk = D->nblocks;
  for (int b = 0; b < D->nblocks; ++b) d.blk[b] = binfo[b];
  INLA_TRY(dev_copy(M, &d.factor_pinv, pinv.data(), pinv.size()));
  INLA_TRY(dev_copy(M, &d.obs_ptr, optr.data(), optr.size()));
  INLA_TRY(dev_copy(M, &d.obs_pair, opair.data(), opair.size()));
  INLA_TRY(dev_copy(M, &d.obs_coef, ocoef.data(), ocoef.size()));
  INLA_TRY(dev_copy(M, &d.heavy_pairs, heavy_pairs.data(), heavy_pairs.size()));
  INLA_TRY(dev_copy(M, &d.y, D->y, (size_t)m));
  if (D->offset) INLA_TRY(dev_copy(M, &d.offset, D->offset, (size_t)m));
  INLA_TRY(dev_copy(M, &d.entries, ent.data(), ent.size()));
  INLA_TRY(dev_copy(M, &d.cct, cct.data(), cct.size()));
  INLA_TRY(dev_copy(M, &d.kron_eig, eig.data(), eig.size()));
  if (dense_b >= 0) {
    const inla_block& B = D->blocks[dense_b];
    INLA_TRY(dev_copy(M, &d.points, B.points, (size_t)2 * B.size));
    d.theta_sigma = B.theta_sigma;
    d.theta_rx = B.theta_range_x;
    d.theta_ry = B.theta_range_y;
    d.theta_iid = B.theta_iid;
    d.nugget = B.nugget;
  }
  if (k > 0) {
    std::vector<int64_t> Crp(k + 1, 0);
    std::vector<int32_t> Ccol;
    std::vector<double> Cval;
    for (int r = 0; r < k; ++r) {
      for (int64_t e = D->C_rowptr[r]; e < D->C_rowptr[r + 1]; ++e) {
        Ccol.push_back(perm[D->C_col[e]]);
        Cval.push_back(D->C_val[e]);
      }
      Crp[r + 1] = (int64_t)Ccol.size();
    }
    INLA_TRY(dev_copy(M, &d.C_rowptr, Crp.data(), Crp.size()));
    INLA_TRY(dev_copy(M, &d.C_col, Ccol.data(), Ccol.size()));
    INLA_TRY(dev_copy(M, &d.C_val, Cval.data(), Cval.size()));
  }
  return INLA_OK;
}

}  // namespace inla

using namespace inla;

extern "C" int inla_model_create(const inla_model_desc* desc, inla_model** out) {
  if (!desc || !out) return INLA_E_BADARG;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return INLA_E_CUDA;
  inla_model* M = new (std::nothrow) inla_model();
  if (!M) return INLA_E_NOMEM;
  M->device = dev;
  int st = create_impl(desc, M);
  if (st != INLA_OK) {
    inla_model_destroy(M);
    return st;
  }
  *out = M;
  return INLA_OK;
}

extern "C" int inla_model_destroy(inla_model* model) {
  if (!model) return INLA_OK;
  for (void* p : model->allocations) cudaFree(p);
  delete model;
  return INLA_OK;
}

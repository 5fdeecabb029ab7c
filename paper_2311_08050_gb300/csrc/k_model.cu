// Prior, likelihood and vector kernels of one theta evaluation, batched over slots.
//
// Prior precision (Section 1 LGM statement; Section 5.1 structures): the dense block is the
// inverse of sigma^2 exp(-d) + (1/tau_iid + nugget) I, the structured blocks are
// a + b exp(theta_t) entries.  Likelihood quantities of one Newton step of Algorithm 1
// (Appendix A.2.1): eta = A x + o, w = exp(eta) (Poisson) or tau (Gaussian), the gradient
// A^T (y - w) - Q_p x, and Q* = Q_p + A^T diag(w) A assembled from a theta-independent list
// of (row, col) pairs with a fixed-order segmented sum (no atomics, deterministic).
#include "kernels.h"
#include "device_util.cuh"
#include <cmath>
#include <algorithm>

namespace inla {


// ---------------- dense covariance block ----------------
__global__ void __launch_bounds__(256) k_cov_build(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.nd == 0) return;
  const ModelDev& md = *s.md;
  const int Td = s.nd_pad / TB;
  int ti, tj;
  {
    int x = blockIdx.x;
    int t = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while (t * (t + 1) / 2 > x) --t;
    while ((t + 1) * (t + 2) / 2 <= x) ++t;
    ti = t;
    tj = x - t * (t + 1) / 2;
  }
  if (ti >= Td) return;
  const double sigma2 = exp(2.0 * s.theta[md.theta_sigma]);
  const double rx = exp(s.theta[md.theta_rx]);
  const double ry = exp(s.theta[md.theta_ry]);
  double diag_add = md.nugget;
  if (md.theta_iid >= 0) diag_add += exp(-s.theta[md.theta_iid]);
  const double* P = md.points;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int i = ti * TB + e / TB, j = tj * TB + e % TB;
    double v;
    if (i < s.nd && j < s.nd) {
      const double dx = (P[2 * i] - P[2 * j]) / rx;
      const double dy = (P[2 * i + 1] - P[2 * j + 1]) / ry;
      v = sigma2 * exp(-sqrt(dx * dx + dy * dy));
      if (i == j) v += diag_add;
    } else {
      v = (i == j) ? 1.0 : 0.0;
    }
    s.Wk[(size_t)i * s.n_pad + j] = v;
  }
}

// ---------------- structured prior entries (value = a + b exp(theta_t)) ----------------
__global__ void k_prior_entries(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < md.nentries;
       e += (int64_t)gridDim.x * blockDim.x) {
    const PriorEntry pe = md.entries[e];
    const double v = pe.t >= 0 ? pe.a + pe.b * exp(s.theta[pe.t]) : pe.a;
    s.Qp[(size_t)pe.row * s.n_pad + pe.col] = v;
  }
}

// copy the lower triangle of Q_p to its upper triangle (tile transpose via shared memory)
__global__ void __launch_bounds__(256) k_mirror_qp(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int T = s.n_pad / TB;
  int ti, tj;
  {
    int x = blockIdx.x;
    int t = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while (t * (t + 1) / 2 > x) --t;
    while ((t + 1) * (t + 2) / 2 <= x) ++t;
    ti = t;
    tj = x - t * (t + 1) / 2;
  }
  if (ti >= T) return;
  __shared__ double tile[TB][TB + 1];
  const double* src = s.Qp + (size_t)ti * TB * s.n_pad + (size_t)tj * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) tile[e / TB][e % TB] = src[(size_t)(e / TB) * s.n_pad + e % TB];
  __syncthreads();
  double* dst = s.Qp + (size_t)tj * TB * s.n_pad + (size_t)ti * TB;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = e / TB, c = e % TB;  // dst(r, c) = src(c, r)
    if (ti != tj || c > r) dst[(size_t)r * s.n_pad + c] = tile[c][r];
  }
}

// L = Q_p on the lower tiles
__global__ void __launch_bounds__(256) k_copy_qp_to_l(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int T = s.n_pad / TB;
  int ti, tj;
  {
    int x = blockIdx.x;
    int t = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while (t * (t + 1) / 2 > x) --t;
    while ((t + 1) * (t + 2) / 2 <= x) ++t;
    ti = t;
    tj = x - t * (t + 1) / 2;
  }
  if (ti >= T) return;
  for (int e = threadIdx.x; e < TB * TB / 2; e += blockDim.x) {
    const int r = e / (TB / 2), c = 2 * (e % (TB / 2));
    const size_t off = (size_t)(ti * TB + r) * s.n_pad + tj * TB + c;
    *reinterpret_cast<double2*>(s.L + off) = *reinterpret_cast<const double2*>(s.Qp + off);
  }
}

// L[row][col] += sum_{c in segment} w[obs_c] * coef_c   (one warp per pair, fixed order)
__global__ void __launch_bounds__(256) k_add_pairs(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  if (blockIdx.x < HEAVY_BLOCKS) {  // heavy pairs: a whole block each
    for (int h = blockIdx.x; h < md.n_heavy_pairs; h += HEAVY_BLOCKS) {
      const int64_t p = md.heavy_pairs[h];
      double v = 0.0;
      for (int64_t c = md.pair_ptr[p] + threadIdx.x; c < md.pair_ptr[p + 1]; c += 256)
        v = fma(s.w[md.pc_obs[c]], md.pc_coef[c], v);
      v = block_sum_256(v);
      if (threadIdx.x == 0) s.L[(size_t)md.pair_row[p] * s.n_pad + md.pair_col[p]] += v;
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((blockIdx.x - HEAVY_BLOCKS) * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)(gridDim.x - HEAVY_BLOCKS) * blockDim.x) >> 5;
  for (int64_t p = warp0; p < md.npairs; p += nwarps) {
    const int64_t lo = md.pair_ptr[p], hi = md.pair_ptr[p + 1];
    if (hi - lo > HEAVY_LEN) continue;
    double v = 0.0;
    for (int64_t c = lo + lane; c < hi; c += 32) v = fma(s.w[md.pc_obs[c]], md.pc_coef[c], v);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s.L[(size_t)md.pair_row[p] * s.n_pad + md.pair_col[p]] += v;
  }
}

// structured part of 1/2 log|Q_p| + 1/2 log|C Q_p^-1 C^T| (times 2): fixed blocks, iid blocks,
// Kronecker blocks via their structure eigenvalues (constrained blocks: positive ones only,
// plus log|C C^T|, which equals the eps-jittered form exactly when the constraints span
// the null space).
__global__ void __launch_bounds__(256) k_prior_logdet(Slot* slots) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  double v = 0.0;
  for (int b = 0; b < md.nkron; ++b) {
    const KronLogdet kb = md.kron[b];
    const double tau = exp(s.theta[kb.theta_idx]);
    for (int i = threadIdx.x; i < kb.size; i += 256) {
      const double lam = md.kron_eig[kb.offset + i];
      if (kb.constrained && lam == 0.0) continue;
      v += log(tau * lam + kb.eps);
    }
  }
  v = block_sum_256(v);
  if (threadIdx.x == 0) {
    double c = md.prior_const_logdet + md.logdet_CCt;
    for (int b = 0; b < md.n_iid; ++b) c += md.iid_size[b] * s.theta[md.iid_theta[b]];
    s.out[OUT_PRIOR_STRUCT] = v + c;
  }
}

__global__ void k_theta_prior(Slot* slots) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active || threadIdx.x != 0) return;
  const ModelDev& md = *s.md;
  double lp = 0.0;
  for (int t = 0; t < md.theta_dim; ++t) {
    const double th = s.theta[t], a = md.prior_a[t], b = md.prior_b[t];
    if (md.prior_kind[t] == INLA_PRIOR_GAUSS) {
      const double z = (th - a) / b;
      lp += -0.91893853320467274178 - log(b) - 0.5 * z * z;  // -1/2 log(2 pi)
    } else {
      const double lam = -log(b) / a;
      lp += log(lam / 2.0) - th / 2.0 - lam * exp(-th / 2.0);
    }
  }
  s.out[OUT_LOG_THETA_PRIOR] = lp;
}

// ---------------- likelihood ----------------
// eta = A v + o ; w ; r (stored in eta) ; partial sums of the log-likelihood kernel into red
__global__ void __launch_bounds__(256) k_eval_lik(Slot* slots, int which) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  const double* v = which ? s.xn : s.x;
  const int m = s.m, nb = gridDim.x;
  const int chunk = (m + nb - 1) / nb;
  const int lo = blockIdx.x * chunk, hi = min(m, lo + chunk);
  double acc = 0.0;
  for (int i = lo + threadIdx.x; i < hi; i += 256) {
    double eta = md.offset ? md.offset[i] : 0.0;
    for (int64_t e = md.A_rowptr[i]; e < md.A_rowptr[i + 1]; ++e) eta = fma(md.A_val[e], v[md.A_col[e]], eta);
    const double y = md.y[i];
    if (md.likelihood == INLA_LIK_POISSON) {
      const double w = exp(eta);
      s.w[i] = w;
      s.eta[i] = y - w;
      acc += y * eta - w;
    } else {
      const double tau = md.lik_prec, d = y - eta;
      s.w[i] = tau;
      s.eta[i] = tau * d;
      acc += -0.5 * tau * d * d;
    }
  }
  acc = block_sum_256(acc);
  if (threadIdx.x == 0) s.red[blockIdx.x] = acc;
}

// out[idx] = sum of red[0..nb) in fixed order
__global__ void k_finish_sum(Slot* slots, int nb, int out_idx) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active || threadIdx.x != 0) return;
  double v = 0.0;
  for (int b = 0; b < nb; ++b) v += s.red[b];
  s.out[out_idx] = v;
}

// t1 = Q_p v (full symmetric storage), one warp per row; quad partials into red
__global__ void __launch_bounds__(256) k_qp_gemv(Slot* slots, int which) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const double* v = which ? s.xn : s.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = s.n_pad;
  for (int row = blockIdx.x * 8 + warp; row < n; row += gridDim.x * 8) {
    const double* q = s.Qp + (size_t)row * n;
    double a0 = 0.0, a1 = 0.0;
    for (int c = lane * 2; c < n; c += 64) {
      const double2 qq = *reinterpret_cast<const double2*>(q + c);
      a0 = fma(qq.x, v[c], a0);
      a1 = fma(qq.y, v[c + 1], a1);
    }
    double r = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) s.t1[row] = r;
  }
}

// red[0] = sum_i v_i t1_i in fixed order (single block)
__global__ void __launch_bounds__(256) k_quad(Slot* slots, int which) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  const double* v = which ? s.xn : s.x;
  double a = 0.0;
  for (int i = threadIdx.x; i < s.n_pad; i += 256) a = fma(v[i], s.t1[i], a);
  a = block_sum_256(a);
  if (threadIdx.x == 0) s.out[OUT_QUAD] = a;
}

// g = A^T r - t1, one warp per latent entry (a column of A such as an intercept can carry
// every observation); lanes stride the column, fixed-order shuffle reduction
// The first HEAVY_BLOCKS blocks reduce the heavy rows of A^T (a whole block each, fixed-order
// tree); the others take one warp per remaining row.
__global__ void __launch_bounds__(256) k_gradient(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  if (blockIdx.x < HEAVY_BLOCKS) {
    for (int h = blockIdx.x; h < md.n_heavy_cols; h += HEAVY_BLOCKS) {
      const int j = md.heavy_cols[h];
      double a = 0.0;
      for (int64_t e = md.At_rowptr[j] + threadIdx.x; e < md.At_rowptr[j + 1]; e += 256)
        a = fma(md.At_val[e], s.eta[md.At_row[e]], a);
      a = block_sum_256(a);
      if (threadIdx.x == 0) s.g[j] = a - s.t1[j];
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int nb = gridDim.x - HEAVY_BLOCKS;
  for (int j = ((blockIdx.x - HEAVY_BLOCKS) * 256 + threadIdx.x) >> 5; j < s.n_pad; j += (nb * 256) >> 5) {
    if (md.At_rowptr[j + 1] - md.At_rowptr[j] > HEAVY_LEN) continue;
    double a = 0.0;
    for (int64_t e = md.At_rowptr[j] + lane; e < md.At_rowptr[j + 1]; e += 32) a = fma(md.At_val[e], s.eta[md.At_row[e]], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) s.g[j] = a - s.t1[j];
  }
}

// Start system of the mixed path's Newton iteration: likelihood weights and residual of a
// weighted least-squares fit of the linear predictor to pseudo-data (Poisson: weights y + 1/2,
// targets log(y + 1/2) - offset, the log link's working response with counts shifted off zero;
// Gaussian: its own weights tau and data, so the start is its exact mode): w = weights,
// r (held in eta) = weights * targets, and t1 = 0, so that the gradient kernel forms A^T r.
__global__ void __launch_bounds__(256) k_wls_start(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < s.m; i += gridDim.x * 256) {
    const double o = md.offset ? md.offset[i] : 0.0;
    const double y = md.y[i];
    double w, z;
    if (md.likelihood == INLA_LIK_POISSON) {
      w = y + 0.5;
      z = log(w) - o;
    } else {
      w = md.lik_prec;
      z = y - o;
    }
    s.w[i] = w;
    s.eta[i] = w * z;
  }
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) s.t1[j] = 0.0;
}

__global__ void __launch_bounds__(256) k_newton_xu(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) s.xn[j] = s.x[j] + s.g[j];
}

__global__ void __launch_bounds__(256) k_cx(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const ModelDev& md = *s.md;
  for (int r = blockIdx.x * 256 + threadIdx.x; r < s.k_pad; r += gridDim.x * 256) {
    double a = 0.0;
    if (r < s.k)
      for (int64_t e = md.C_rowptr[r]; e < md.C_rowptr[r + 1]; ++e) a = fma(md.C_val[e], s.xn[md.C_col[e]], a);
    s.kv1[r] = a;
  }
}

// t2 = Z kv1 (n_pad x k_pad), one warp per row
__global__ void __launch_bounds__(256) k_z_gemv(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row = blockIdx.x * 8 + warp; row < s.n_pad; row += gridDim.x * 8) {
    const double* z = s.Z + (size_t)row * s.k_pad;
    double a = 0.0;
    for (int c = lane; c < s.k_pad; c += 32) a = fma(z[c], s.kv1[c], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) s.t2[row] = a;
  }
}

__global__ void __launch_bounds__(256) k_krige_apply(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) s.xn[j] -= s.g[j];
}

__global__ void __launch_bounds__(256) k_step_norm(Slot* slots) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  __shared__ double sh[256];
  double a = 0.0;
  for (int j = threadIdx.x; j < s.n_pad; j += 256) a = fmax(a, fabs(s.xn[j] - s.x[j]));
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) s.out[OUT_STEP] = sh[0];
}

__global__ void __launch_bounds__(256) k_halve(Slot* slots, const int* flags) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || !flags[blockIdx.y]) return;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256)
    s.xn[j] = s.x[j] + 0.5 * (s.xn[j] - s.x[j]);
}

__global__ void __launch_bounds__(256) k_accept(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) s.x[j] = s.xn[j];
}

__global__ void __launch_bounds__(256) k_zero_vec(Slot* slots, int which) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  double* v = which == 0 ? s.x : s.xn;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) v[j] = 0.0;
}

// Z = dense C^T (the caller zeroed Z)
__global__ void __launch_bounds__(256) k_ct_fill(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const ModelDev& md = *s.md;
  for (int r = blockIdx.x * 256 + threadIdx.x; r < s.k; r += gridDim.x * 256)
    for (int64_t e = md.C_rowptr[r]; e < md.C_rowptr[r + 1]; ++e) s.Z[(size_t)md.C_col[e] * s.k_pad + r] = md.C_val[e];
}

__global__ void __launch_bounds__(256) k_var_finish(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) s.t1[j] -= s.t2[j];
}

// log pi~(theta|y) = log pi(theta) + sum log p(y|eta) - 1/2 x^T Q_p x + 1/2 log|Q_p|
//                    + 1/2 log|S_p| - 1/2 log|Q*| - 1/2 log|S|       (Eq. (41) at the mode)
__global__ void k_assemble(Slot* slots) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active || threadIdx.x != 0) return;
  const ModelDev& md = *s.md;
  double loglik = s.out[OUT_LOGLIK];
  if (md.likelihood == INLA_LIK_POISSON)
    loglik -= md.lgamma_sum;
  else
    loglik += s.m * (0.5 * log(md.lik_prec) - 0.91893853320467274178);
  const double half_logdet_prior = 0.5 * (s.out[OUT_PRIOR_STRUCT] - s.out[OUT_LOGDET_COV]);
  s.out[OUT_LOGPOST] = s.out[OUT_LOG_THETA_PRIOR] + loglik - 0.5 * s.out[OUT_QUAD] + half_logdet_prior -
                       0.5 * s.out[OUT_LOGDET_Q] - 0.5 * s.out[OUT_LOGDET_S];
}

// ---------------- launchers ----------------
static int tri(int t) { return t * (t + 1) / 2; }
static int vgrid(int n) { return min(1024, max(1, (n + 255) / 256)); }

void launch_cov_build(Slot* slots, int nslots, int max_td, cudaStream_t st) {
  if (max_td > 0) count_launch("k_cov_build"), k_cov_build<<<dim3(tri(max_td), nslots), 256, 0, st>>>(slots);
}
void launch_prior_entries(Slot* slots, int nslots, int64_t max_entries, cudaStream_t st) {
  if (max_entries > 0) count_launch("k_prior_entries"), k_prior_entries<<<dim3((unsigned)std::min<int64_t>(2048, (max_entries + 255) / 256), nslots), 256, 0, st>>>(slots);
}
void launch_mirror_qp(Slot* slots, int nslots, int max_t, cudaStream_t st) {
  count_launch("k_mirror_qp"), k_mirror_qp<<<dim3(tri(max_t), nslots), 256, 0, st>>>(slots);
}
void launch_copy_qp_to_l(Slot* slots, int nslots, int max_t, cudaStream_t st) {
  count_launch("k_copy_qp_to_l"), k_copy_qp_to_l<<<dim3(tri(max_t), nslots), 256, 0, st>>>(slots);
}
void launch_add_pairs(Slot* slots, int nslots, int64_t max_pairs, cudaStream_t st) {
  if (max_pairs > 0)
    count_launch("k_add_pairs"), k_add_pairs<<<dim3(HEAVY_BLOCKS + (unsigned)std::min<int64_t>(4096, (max_pairs + 7) / 8), nslots), 256, 0, st>>>(slots);
}
void launch_prior_logdet(Slot* slots, int nslots, cudaStream_t st) { count_launch("k_prior_logdet"), k_prior_logdet<<<nslots, 256, 0, st>>>(slots); }
void launch_theta_prior(Slot* slots, int nslots, cudaStream_t st) { count_launch("k_theta_prior"), k_theta_prior<<<nslots, 32, 0, st>>>(slots); }
void launch_eval_lik(Slot* slots, int nslots, int which, int max_m, cudaStream_t st) {
  (void)max_m;
  count_launch("k_eval_lik"), k_eval_lik<<<dim3(128, nslots), 256, 0, st>>>(slots, which);
  count_launch("k_finish_sum"), k_finish_sum<<<nslots, 32, 0, st>>>(slots, 128, OUT_LOGLIK);
}
void launch_qp_gemv(Slot* slots, int nslots, int which, int max_n, cudaStream_t st) {
  count_launch("k_qp_gemv"), k_qp_gemv<<<dim3(min(4096, (max_n + 7) / 8), nslots), 256, 0, st>>>(slots, which);
  count_launch("k_quad"), k_quad<<<nslots, 256, 0, st>>>(slots, which);
}
void launch_quad(Slot* slots, int nslots, int which, cudaStream_t st) { count_launch("k_quad"), k_quad<<<nslots, 256, 0, st>>>(slots, which); }
void launch_gradient(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_gradient"), k_gradient<<<dim3(HEAVY_BLOCKS + std::min(4096, (max_n + 7) / 8), nslots), 256, 0, st>>>(slots);
}
void launch_wls_start(Slot* slots, int nslots, int max_m, int max_n, cudaStream_t st) {
  count_launch("k_wls_start"), k_wls_start<<<dim3(vgrid(std::max(max_m, max_n)), nslots), 256, 0, st>>>(slots);
}
void launch_newton_xu(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_newton_xu"), k_newton_xu<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots);
}
void launch_cx(Slot* slots, int nslots, int max_k, cudaStream_t st) {
  count_launch("k_cx"), k_cx<<<dim3(vgrid(max_k), nslots), 256, 0, st>>>(slots);
}
void launch_z_gemv(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_z_gemv"), k_z_gemv<<<dim3(min(4096, (max_n + 7) / 8), nslots), 256, 0, st>>>(slots);
}
void launch_krige_apply(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_krige_apply"), k_krige_apply<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots);
}
void launch_step_norm(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  (void)max_n;
  count_launch("k_step_norm"), k_step_norm<<<nslots, 256, 0, st>>>(slots);
}
void launch_halve(Slot* slots, int nslots, const int* flags, int max_n, cudaStream_t st) {
  count_launch("k_halve"), k_halve<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots, flags);
}
void launch_accept(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_accept"), k_accept<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots);
}
void launch_zero_vec(Slot* slots, int nslots, int which, int max_n, cudaStream_t st) {
  count_launch("k_zero_vec"), k_zero_vec<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots, which);
}
void launch_ct_fill(Slot* slots, int nslots, int max_k, cudaStream_t st) {
  count_launch("k_ct_fill"), k_ct_fill<<<dim3(vgrid(max_k), nslots), 256, 0, st>>>(slots);
}
void launch_var_finish(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_var_finish"), k_var_finish<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots);
}
void launch_assemble(Slot* slots, int nslots, cudaStream_t st) { count_launch("k_assemble"), k_assemble<<<nslots, 32, 0, st>>>(slots); }

}  // namespace inla

namespace inla {
// L[row][col] += gamma_c * (C^T C)[row][col] on the lower triangle (constrained models)
__global__ void k_add_cct(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const ModelDev& md = *s.md;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < md.ncct; e += (int64_t)gridDim.x * blockDim.x) {
    const PriorEntry pe = md.cct[e];
    s.L[(size_t)pe.row * s.n_pad + pe.col] += md.gamma_c * pe.a;
  }
}
void launch_add_cct(Slot* slots, int nslots, cudaStream_t st) {
  count_launch("k_add_cct"), k_add_cct<<<dim3(1024, nslots), 256, 0, st>>>(slots);
}
}  // namespace inla

// Variational Bayes correction of the posterior mean (Appendix A.2.2, Algorithm 2), on the
// device, after the factor at the mode and its inverse are known.
//
// The Gaussian posterior keeps the Laplace precision Q* and moves its mean: each step solves
// Q^c lambda = -c with c = A^T I'(0) + Q_p mu, Q^c = Q_p + A^T diag(I''(0)) A, where I'(0)_i and
// I''(0)_i are the means of l', l'' (l = -log pi(y_i|eta)) under eta ~ N(nu_i, sigma_i^2),
// nu = A mu + offset, sigma_i^2 = (A Q*^-1 A^T)_ii fixed at the Laplace approximation, taken by
// Gauss-Hermite quadrature.  Algorithm 2 refactors Q^c at every step; here every step uses the
// factor of Q* instead (the two differ by A^T diag(I'' - w) A, w the Newton weights at the mode),
// which changes the path but not the fixed point c(mu) = 0; the steps are repeated until
// max |lambda| <= 1e-8.
#include <algorithm>
#include <cmath>
#include <vector>
#include "df64.cuh"
#include "mixed.h"

namespace inla {

constexpr int VB_GH_MAX = 32;
struct GhRule {
  int n;
  double x[VB_GH_MAX], w[VB_GH_MAX];  // nodes and weights / sqrt(pi) of the weight e^-x^2
};

// Gauss-Hermite rule for the weight e^{-x^2}: the nodes are the roots of the orthonormal
// Hermite polynomial p_n (p_0 = pi^-1/4, p_{k+1} = x sqrt(2 / (k + 1)) p_k - sqrt(k / (k + 1))
// p_{k-1}), located by sign changes on a fine grid over (-sqrt(2n + 1), sqrt(2n + 1)) and refined
// by bisection; the weights are the Christoffel numbers 1 / sum_{k < n} p_k(x_j)^2.
static void hermite_values(int n, double x, double* p) {  // p[0..n]
  p[0] = std::pow(M_PI, -0.25);
  if (n == 0) return;
  p[1] = x * std::sqrt(2.0) * p[0];
  for (int k = 1; k < n; ++k) p[k + 1] = x * std::sqrt(2.0 / (k + 1)) * p[k] - std::sqrt((double)k / (k + 1)) * p[k - 1];
}
static int gauss_hermite(int n, double* nodes, double* weights) {
  if (n < 1 || n > VB_GH_MAX) return INLA_E_BADARG;
  std::vector<double> p(n + 1);
  auto pn = [&](double x) {
    hermite_values(n, x, p.data());
    return p[n];
  };
  // grid points offset by an irrational fraction of a cell, so that none falls on a root
  const double lim = std::sqrt(2.0 * n + 1.0) + 1.0;
  const int grid = 20000;
  int found = 0;
  double xa = -lim, fa = pn(xa);
  for (int g = 1; g <= grid && found < n; ++g) {
    const double xb = -lim + 2.0 * lim * (g + 0.3819660112501051) / grid, fb = pn(xb);
    if ((fa < 0.0) != (fb < 0.0)) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo)); ++it) {
        const double mid = 0.5 * (lo + hi), fm = pn(mid);
        if ((fm < 0.0) == (flo < 0.0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      const double r = 0.5 * (lo + hi);
      nodes[found] = r;
      hermite_values(n, r, p.data());
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += p[k] * p[k];
      weights[found] = 1.0 / s;
      ++found;
    }
    xa = xb;
    fa = fb;
  }
  return found == n ? INLA_OK : INLA_E_CUDA;
}

// (Q*^-1)_kl for every unique pair (k >= l) of the model's A^T A pattern, one warp per pair.
// Mixed path: Wk holds Y = L^-T (upper), (Q*^-1)_kl = sum_{j >= k} Y_kj Y_lj; FP64 path: Wk holds
// W = L^-1 (lower), (Q*^-1)_kl = sum_{j >= k} W_jk W_jl.
__global__ void __launch_bounds__(256) k_pair_cov(Slot* slots, int mixed) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int n = s.n_pad;
  for (int64_t q = warp0; q < md.npairs; q += nwarps) {
    const int k = md.pair_row[q], l = md.pair_col[q];
    double a = 0.0;
    if (mixed) {
      const float2* Y = reinterpret_cast<const float2*>(s.Wk);
      df acc = df_make(0.f, 0.f);
      for (int j = k + lane; j < n; j += 32)
        acc = df_fma(acc, df_load(Y + (size_t)k * n + j), df_load(Y + (size_t)l * n + j));
      a = df_to_double(acc);
    } else {
      for (int j = k + lane; j < n; j += 32) a = fma(s.Wk[(size_t)j * n + k], s.Wk[(size_t)j * n + l], a);
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) s.pcov[q] = a;
  }
}

// sigma_i^2 = sum over observation i's pairs of coef * (Q*^-1)_kl
__global__ void __launch_bounds__(256) k_eta_var(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < s.m; i += gridDim.x * 256) {
    double v = 0.0;
    for (int64_t e = md.obs_ptr[i]; e < md.obs_ptr[i + 1]; ++e) v = fma(md.obs_coef[e], s.pcov[md.obs_pair[e]], v);
    s.etav[i] = v;
  }
}

// nu = A x + offset; I'(0), I''(0) by the Gauss-Hermite rule; the gradient kernel's residual
// (held in eta) is -I'(0), so that it forms A^T (-I') - Q_p x = -c
__global__ void __launch_bounds__(256) k_vb_terms(Slot* slots, GhRule gh) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < s.m; i += gridDim.x * 256) {
    double nu = md.offset ? md.offset[i] : 0.0;
    for (int64_t e = md.A_rowptr[i]; e < md.A_rowptr[i + 1]; ++e) nu = fma(md.A_val[e], s.x[md.A_col[e]], nu);
    const double sd = sqrt(2.0 * fmax(s.etav[i], 0.0)), y = md.y[i];
    double d1 = 0.0, d2 = 0.0;
    for (int j = 0; j < gh.n; ++j) {
      const double eta = fma(sd, gh.x[j], nu);
      if (md.likelihood == INLA_LIK_POISSON) {
        const double e = exp(eta);
        d1 = fma(gh.w[j], e - y, d1);
        d2 = fma(gh.w[j], e, d2);
      } else {
        d1 = fma(gh.w[j], md.lik_prec * (eta - y), d1);
        d2 = fma(gh.w[j], md.lik_prec, d2);
      }
    }
    s.eta[i] = -d1;
    s.w[i] = d2;
  }
}

void launch_vb_prepare(Slot* slots, int nslots, int mixed, int64_t max_pairs, int max_m, cudaStream_t st) {
  if (max_pairs > 0)
    count_launch("k_pair_cov"), k_pair_cov<<<dim3((unsigned)std::min<int64_t>(4096, (max_pairs + 7) / 8), nslots), 256, 0, st>>>(slots, mixed);
  if (max_m > 0) count_launch("k_eta_var"), k_eta_var<<<dim3(std::min(1024, (max_m + 255) / 256), nslots), 256, 0, st>>>(slots);
}

int launch_vb_terms(Slot* slots, int nslots, int max_m, cudaStream_t st) {
  static GhRule rule = [] {
    GhRule r;
    r.n = 15;
    if (gauss_hermite(r.n, r.x, r.w) != INLA_OK) r.n = 0;
    for (int j = 0; j < r.n; ++j) r.w[j] /= std::sqrt(M_PI);
    return r;
  }();
  if (rule.n == 0) return INLA_E_CUDA;
  if (max_m > 0) count_launch("k_vb_terms"), k_vb_terms<<<dim3(std::min(1024, (max_m + 255) / 256), nslots), 256, 0, st>>>(slots, rule);
  return INLA_OK;
}

}  // namespace inla

// test hook: the Gauss-Hermite rule the variational Bayes correction uses
extern "C" int inla_test_gauss_hermite(int32_t n, double* nodes, double* weights) {
  if (!nodes || !weights) return INLA_E_BADARG;
  return inla::gauss_hermite(n, nodes, weights);
}

// Stage 2 of the method (Section 2, Stage 2; Appendix A.2): the latent marginals integrated over
// the exploration points theta_k of the hyperparameter space.  The batched evaluation gives, per
// point, log pi~(theta_k|y) and the Gaussian marginals N(x_hat_i(theta_k), var_i(theta_k)); the
// integrated marginal of x_i is their mixture with weights w_k proportional to
// delta_k pi~(theta_k|y) (delta_k: the design's quadrature weight), whose moments this computes:
//   mean_i = sum_k w_k x_hat_ki,   var_i = sum_k w_k (var_ki + x_hat_ki^2) - mean_i^2.
#include <cmath>
#include "internal.h"

namespace inla {

constexpr int INTEG_MAX_K = 4096;

// One block per 256 columns; every block forms the K normalised weights in shared memory
// (fixed-order reductions, so every block holds identical weights), then each thread sums its
// column over the K points (coalesced rows of X and V).
__global__ void __launch_bounds__(256) k_integrate_marginals(const double* lp, const double* delta, int K,
                                                             const double* X, const double* V, int64_t ld, int n,
                                                             double* mean, double* var) {
  __shared__ double w[INTEG_MAX_K];
  __shared__ double red[256];
  const int tid = threadIdx.x;
  double mx = -INFINITY;
  for (int k = tid; k < K; k += 256) mx = fmax(mx, lp[k]);
  red[tid] = mx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
    __syncthreads();
  }
  mx = red[0];
  __syncthreads();
  double s = 0.0;
  for (int k = tid; k < K; k += 256) {
    const double v = isfinite(lp[k]) ? delta[k] * exp(lp[k] - mx) : 0.0;
    w[k] = v;
    s += v;
  }
  red[tid] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const double inv = 1.0 / red[0];
  const int i = blockIdx.x * 256 + tid;
  if (i >= n) return;
  double m = 0.0, q = 0.0;
  for (int k = 0; k < K; ++k) {
    const double wk = w[k] * inv;
    const double x = X[(int64_t)k * ld + i];
    m = fma(wk, x, m);
    q = fma(wk, fma(x, x, V[(int64_t)k * ld + i]), q);
  }
  mean[i] = m;
  var[i] = q - m * m;
}

}  // namespace inla

using namespace inla;

extern "C" int inla_integrate_marginals(int32_t K, int32_t n, const double* log_post, const double* delta,
                                        const double* x_hat, const double* var, int64_t ld, double* mean_out,
                                        double* var_out, int32_t flags, void* stream) {
  if (K <= 0 || K > INTEG_MAX_K || n <= 0 || ld < n || !log_post || !delta || !x_hat || !var || !mean_out || !var_out)
    return INLA_E_BADARG;
  double w_any = 0.0;
  for (int k = 0; k < K; ++k) {
    if (!(delta[k] >= 0.0) || !std::isfinite(delta[k])) return INLA_E_BADARG;
    if (std::isfinite(log_post[k])) w_any += delta[k];
  }
  if (!(w_any > 0.0)) return INLA_E_BADARG;  // no point carries weight
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool dev = (flags & INLA_OPT_DEVICE_OUT) != 0;
  const size_t mat = (size_t)K * ld * sizeof(double);
  char* buf = nullptr;
  const size_t small = 2 * (size_t)K * sizeof(double);
  const size_t bytes = small + (dev ? 0 : 2 * mat + 2 * (size_t)n * sizeof(double));
  if (cudaMallocAsync((void**)&buf, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return INLA_E_NOMEM;
  }
  double* d_lp = reinterpret_cast<double*>(buf);
  double* d_delta = d_lp + K;
  const double *X = x_hat, *V = var;
  double *M = mean_out, *W = var_out;
  int rc = INLA_OK;
  if (cudaMemcpyAsync(d_lp, log_post, K * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_delta, delta, K * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = INLA_E_CUDA;
  if (rc == INLA_OK && !dev) {
    double* dX = d_delta + K;
    double* dV = dX + (size_t)K * ld;
    M = dV + (size_t)K * ld;
    W = M + n;
    if (cudaMemcpyAsync(dX, x_hat, mat, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(dV, var, mat, cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = INLA_E_CUDA;
    X = dX;
    V = dV;
  }
  if (rc == INLA_OK) {
    count_launch("k_integrate_marginals");
    k_integrate_marginals<<<(n + 255) / 256, 256, 0, st>>>(d_lp, d_delta, K, X, V, ld, n, M, W);
    if (cudaPeekAtLastError() != cudaSuccess) rc = note_launch_error("k_integrate_marginals");
  }
  if (rc == INLA_OK && !dev) {
    if (cudaMemcpyAsync(mean_out, M, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(var_out, W, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = INLA_E_CUDA;
  }
  cudaFreeAsync(buf, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == INLA_OK) rc = INLA_E_CUDA;
  if (rc != INLA_OK) cudaGetLastError();
  return rc;
}

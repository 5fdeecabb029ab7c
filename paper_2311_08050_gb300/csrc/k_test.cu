// Test hooks (include/inla_testing.h): isolated runs of the mixed-precision building blocks.
#include <algorithm>
#include <cstring>
#include <vector>
#include "../../include/inla_testing.h"
#include "df64.cuh"
#include "ozaki.h"
#include "mixed.h"

namespace inla {

__global__ void k_f64_to_df(const double* src, float2* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const df v = df_from_double(src[i]);
    dst[i] = make_float2(v.hi, v.lo);
  }
}
__global__ void k_df_to_f64(const float2* src, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i].x + (double)src[i].y;
}

}  // namespace inla

using namespace inla;

extern "C" int inla_test_ozaki_gemm(const double* A, const double* B, double* C, int32_t M, int32_t N, int32_t K,
                                    int32_t S, int32_t trans_a, int32_t trans_b, int32_t lower, int32_t k_mode,
                                    double alpha, double beta) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || (K % OZ_BK) || S < 2 || S > OZ_MAX_S) return INLA_E_BADARG;
  if (lower && M != N) return INLA_E_BADARG;
  const int64_t nA = (int64_t)M * K, nB = (int64_t)N * K, nC = (int64_t)M * N;
  const int ldk = (int)round_up(K, OZ_BK);
  const int nch = (K + OZ_CHUNK - 1) / OZ_CHUNK;
  const int rowsA = (int)round_up(M, OZ_BM), rowsB = (int)round_up(N, OZ_BN);
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  float2 *fA = nullptr, *fB = nullptr, *fC = nullptr;
  uint16_t *pA = nullptr, *pB = nullptr;
  int32_t *eA = nullptr, *eB = nullptr, *err = nullptr;
  int rc = INLA_OK;
  auto fail = [&](int code) { rc = code; };
  do {
    if (cudaMalloc(&dA, nA * 8) || cudaMalloc(&dB, nB * 8) || cudaMalloc(&dC, nC * 8) || cudaMalloc(&fA, nA * 8) ||
        cudaMalloc(&fB, nB * 8) || cudaMalloc(&fC, nC * 8) || cudaMalloc(&pA, (size_t)S * rowsA * ldk * 2) ||
        cudaMalloc(&pB, (size_t)S * rowsB * ldk * 2) || cudaMalloc(&eA, (size_t)nch * rowsA * 4) ||
        cudaMalloc(&eB, (size_t)nch * rowsB * 4) || cudaMalloc(&err, 4)) {
      fail(INLA_E_NOMEM);
      break;
    }
    cudaMemcpy(dA, A, nA * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, nB * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dC, C, nC * 8, cudaMemcpyHostToDevice);
    cudaMemset(err, 0, 4);
    cudaMemset(pA, 0, (size_t)S * rowsA * ldk * 2);
    cudaMemset(pB, 0, (size_t)S * rowsB * ldk * 2);
    k_f64_to_df<<<256, 256>>>(dA, fA, nA);
    k_f64_to_df<<<256, 256>>>(dB, fB, nB);
    k_f64_to_df<<<256, 256>>>(dC, fC, nC);
    OzOperand oa{pA, eA, M, K, ldk, (int64_t)rowsA * ldk, rowsA, 0};
    OzOperand ob{pB, eB, N, K, ldk, (int64_t)rowsB * ldk, rowsB, 0};
    // A: M x K (rows) or K x M (transposed source, ld = M)
    oz_slice_df(fA, 0, trans_a ? M : K, 0, 0, M, K, trans_a != 0, oa, S, 1, 0);
    oz_slice_df(fB, 0, trans_b ? N : K, 0, 0, N, K, trans_b != 0, ob, S, 1, 0);
    OzArgs args;
    std::memset(&args, 0, sizeof(args));
    args.C = fC;
    args.ldc = N;
    args.M = M;
    args.N = N;
    args.K = K;
    args.k_mode = k_mode;
    args.lower = lower;
    args.lower_elems = lower;
    args.alpha = (float)alpha;
    args.beta = (float)beta;
    args.S = S;
    args.spin_limit = (int64_t)1 << 26;
    args.err = err;
    rc = oz_gemm(oa, ob, args, 1, 0);
    if (rc != INLA_OK) break;
    k_df_to_f64<<<256, 256>>>(fC, dC, nC);
    if (cudaDeviceSynchronize() != cudaSuccess) {
      fail(INLA_E_CUDA);
      break;
    }
    int herr = 0;
    cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    if (herr) {
      fail(INLA_E_TIMEOUT);
      break;
    }
    cudaMemcpy(C, dC, nC * 8, cudaMemcpyDeviceToHost);
  } while (0);
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  cudaFree(fA);
  cudaFree(fB);
  cudaFree(fC);
  cudaFree(pA);
  cudaFree(pB);
  cudaFree(eA);
  cudaFree(eB);
  cudaFree(err);
  if (rc == INLA_E_CUDA) cudaGetLastError();
  return rc;
}

// Dense covariance entries sigma^2 exp(-sqrt((dx rx^-1)^2 + (dy ry^-1)^2)) of n host points
// (row-major n x 2) computed by the double-float device code of the mixed path, returned as FP64.
extern "C" int inla_test_cov_df(const double* points, int32_t n, double sigma2, double inv_rx, double inv_ry,
                                double* out) {
  if (!points || !out || n <= 0 || n > 8192) return INLA_E_BADARG;
  double *dP = nullptr, *dO = nullptr;
  int rc = INLA_OK;
  if (cudaMalloc(&dP, sizeof(double) * 2 * (size_t)n) != cudaSuccess ||
      cudaMalloc(&dO, sizeof(double) * (size_t)n * n) != cudaSuccess)
    rc = INLA_E_NOMEM;
  if (rc == INLA_OK && cudaMemcpy(dP, points, sizeof(double) * 2 * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = INLA_E_CUDA;
  if (rc == INLA_OK) {
    launch_cov_points_df(dP, n, sigma2, inv_rx, inv_ry, dO, 0);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(out, dO, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = INLA_E_CUDA;
  }
  cudaFree(dP);
  cudaFree(dO);
  if (rc != INLA_OK) cudaGetLastError();
  return rc;
}


// One cooperative double-float triangular solve (the Newton-step solve of the mixed path) on a
// caller-given factor: x = L^-1 b (backward = 0) or L^-T b (backward = 1), every dependency wait
// bounded by spin_limit iterations.  The 64 x 64 diagonal-tile inverses the kernel needs are
// formed here on the host by forward substitution (test set-up, not the product path).
extern "C" int inla_test_trsv_df(const double* L, const double* b, int32_t n, int32_t backward, int64_t spin_limit,
                                 double* x) {
  if (!L || !b || !x || n <= 0 || (n % TB) || spin_limit < 0) return INLA_E_BADARG;
  const int T = n / TB;
  std::vector<double> linv((size_t)n * TB, 0.0);
  for (int t = 0; t < T; ++t) {
    double* Y = &linv[(size_t)t * TB * TB];  // inverse of the diagonal tile t (lower)
    for (int c = 0; c < TB; ++c) {
      for (int i = c; i < TB; ++i) {
        double s = i == c ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) s -= L[(size_t)(t * TB + i) * n + t * TB + k] * Y[k * TB + c];
        const double d = L[(size_t)(t * TB + i) * n + t * TB + i];
        if (!(d != 0.0)) return INLA_E_BADARG;
        Y[i * TB + c] = s / d;
      }
    }
  }
  double *dL = nullptr, *dLinv = nullptr, *dv = nullptr, *dout = nullptr;
  Slot* dslot = nullptr;
  int32_t *flags = nullptr, *err = nullptr, *info = nullptr;
  int rc = INLA_OK;
  do {
    if (cudaMalloc(&dL, (size_t)n * n * 8) || cudaMalloc(&dLinv, (size_t)n * TB * 8) || cudaMalloc(&dv, (size_t)n * 16) ||
        cudaMalloc(&dout, 64) || cudaMalloc(&dslot, sizeof(Slot)) || cudaMalloc(&flags, sizeof(int32_t) * T) ||
        cudaMalloc(&err, 4) || cudaMalloc(&info, 8)) {
      rc = INLA_E_NOMEM;
      break;
    }
    // L and the tile inverses as double-float cells (8 bytes each)
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, (size_t)n * n * 8)) {
      rc = INLA_E_NOMEM;
      break;
    }
    cudaMemcpy(tmp, L, (size_t)n * n * 8, cudaMemcpyHostToDevice);
    k_f64_to_df<<<256, 256>>>(tmp, reinterpret_cast<float2*>(dL), (int64_t)n * n);
    cudaMemcpy(tmp, linv.data(), (size_t)n * TB * 8, cudaMemcpyHostToDevice);
    k_f64_to_df<<<256, 256>>>(tmp, reinterpret_cast<float2*>(dLinv), (int64_t)n * TB);
    cudaDeviceSynchronize();
    cudaFree(tmp);
    cudaMemcpy(dv, b, (size_t)n * 8, cudaMemcpyHostToDevice);
    cudaMemset(err, 0, 4);
    Slot s;
    std::memset(&s, 0, sizeof(s));
    s.L = dL;
    s.Linv = dLinv;
    s.g = dv;
    s.t1 = dv + n;
    s.out = reinterpret_cast<double*>(dout);
    s.info = info;
    s.n_pad = s.n = n;
    s.active = 1;
    cudaMemcpy(dslot, &s, sizeof(Slot), cudaMemcpyHostToDevice);
    TrsvArgs a;
    a.slots = dslot;
    a.sel = SEL_L;
    a.src = 0;  // g
    a.dst = 1;  // t1
    a.nslots = 1;
    a.T = T;
    a.backward = backward ? 1 : 0;
    a.flags = flags;
    a.err = err;
    a.spin_limit = spin_limit;
    if ((rc = launch_trsv_df(a, 0)) != INLA_OK) break;
    if (cudaDeviceSynchronize() != cudaSuccess) {
      rc = INLA_E_CUDA;
      break;
    }
    int herr = 0;
    cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    if (herr) {
      rc = INLA_E_TIMEOUT;
      break;
    }
    cudaMemcpy(x, dv + n, (size_t)n * 8, cudaMemcpyDeviceToHost);
  } while (0);
  cudaFree(dL);
  cudaFree(dLinv);
  cudaFree(dv);
  cudaFree(dout);
  cudaFree(dslot);
  cudaFree(flags);
  cudaFree(err);
  cudaFree(info);
  if (rc == INLA_E_CUDA) cudaGetLastError();
  return rc;
}

// ---- arithmetic peak probes (FMA throughput of the FP64 and FP32 pipes) ----
namespace inla {
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);  // eight independent chains per thread
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1.2345) sink[0] = s;  // never true for these inputs; keeps the chains live
}
}  // namespace inla

// Best-of-`reps` FMA throughput in TFLOP/s (2 flops per FMA) of the FP64 (kind 0) or FP32
// (kind 1) pipes over every SM of the current device, timed with CUDA events.
extern "C" int inla_test_fma_peak(int32_t kind, int32_t reps, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1) || reps <= 0) return INLA_E_BADARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return INLA_E_CUDA;
  void* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) return INLA_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  const int iters = kind == 0 ? 2048 : 65536;
  double best = 0.0;
  int rc = INLA_OK;
  for (int r = 0; r < reps + 1 && rc == INLA_OK; ++r) {  // first run: warm-up
    cudaEventRecord(e0);
    if (kind == 0) k_fma_probe<double><<<blocks, threads>>>((double*)sink, iters, 0.9999999, 1e-7);
    else k_fma_probe<float><<<blocks, threads>>>((float*)sink, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = INLA_E_CUDA;
    const double fl = 2.0 * 8.0 * iters * (double)threads * blocks;
    if (r > 0 && ms > 0.f) best = std::max(best, fl / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc != INLA_OK) cudaGetLastError();
  *tflops = best;
  return rc;
}

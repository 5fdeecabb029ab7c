// FP64 blocked dense linear algebra on 64 x 64 tiles, batched over slots (grid.z / grid.y).
//
// These kernels implement the dense factorisation the paper names as the bottleneck of
// every theta evaluation (Section 4: Cholesky per Newton step of Algorithm 1) and the
// quantities read from the factor (log-determinant for Eq. (41), the diagonal of the
// inverse for the Gaussian marginals of Appendix A.2.1).  Right-looking blocked Cholesky:
// factor the diagonal tile, solve the panel against its inverse, update the trailing
// lower triangle.  Every matrix is row-major with a leading dimension; only the lower
// triangle of a symmetric matrix is read.
#include "kernels.h"
#include "device_util.cuh"
#include <cmath>
#include <climits>

namespace inla {

struct MatRef {
  double* A;
  double* Linv;
  int n;
  int ld;
};

__device__ __forceinline__ MatRef mat_ref(const Slot& s, int sel) {
  if (sel == SEL_L) return MatRef{s.L, s.Linv, s.n_pad, s.n_pad};
  if (sel == SEL_COV) return MatRef{s.Wk, s.Wd, s.nd_pad, s.n_pad};
  return MatRef{s.S, s.SLinv, s.k_pad, s.k_pad};
}

__device__ __forceinline__ double* vec_ref(const Slot& s, int v) {
  switch (v) {
    case 0: return s.g;
    case 1: return s.t1;
    case 2: return s.t2;
    case 3: return s.kv1;
    default: return s.kv2;
  }
}

// ------------------------------------------------------------------------------------
// diagonal tile: Cholesky and triangular inverse in shared memory (FP64)
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_potrf_diag(Slot* slots, int sel, int kt) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  MatRef M = mat_ref(s, sel);
  if (kt * TB >= M.n) return;
  extern __shared__ double smem[];
  double(*a)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(smem);
  double(*inv)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(smem + TB * (TB + 1));
  __shared__ int bad;
  const int tid = threadIdx.x;
  double* base = M.A + (size_t)kt * TB * M.ld + (size_t)kt * TB;
  for (int e = tid; e < TB * TB; e += blockDim.x) a[e / TB][e % TB] = base[(size_t)(e / TB) * M.ld + e % TB];
  if (tid == 0) bad = 0;
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  for (int j = 0; j < TB; ++j) {
    if (tid == 0) {
      double d = a[j][j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (!bad) {
          bad = 1;
          atomicOr(&s.info[0], INFO_NOT_SPD);
          atomicMin(&s.info[1], kt * TB + j);
        }
        d = 1.0;
      }
      a[j][j] = sqrt(d);
    }
    __syncthreads();
    const double djj = a[j][j];
    for (int i = j + 1 + tid; i < TB; i += blockDim.x) a[i][j] = a[i][j] / djj;
    __syncthreads();
    for (int i = j + 1 + ty; i < TB; i += 16)
      for (int c = j + 1 + tx; c <= i; c += 16) a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
    __syncthreads();
  }
  // inverse of the lower-triangular tile: thread c solves column c
  if (tid < TB) {
    const int c = tid;
    for (int i = 0; i < c; ++i) inv[i][c] = 0.0;
    inv[c][c] = 1.0 / a[c][c];
    for (int i = c + 1; i < TB; ++i) {
      double acc0 = 0.0, acc1 = 0.0;
      int k = c;
      for (; k + 1 < i; k += 2) {
        acc0 = fma(a[i][k], inv[k][c], acc0);
        acc1 = fma(a[i][k + 1], inv[k + 1][c], acc1);
      }
      if (k < i) acc0 = fma(a[i][k], inv[k][c], acc0);
      inv[i][c] = -(acc0 + acc1) / a[i][i];
    }
  }
  __syncthreads();
  double* linv = M.Linv + (size_t)kt * TB * TB;
  for (int e = tid; e < TB * TB; e += blockDim.x) {
    int r = e / TB, c = e % TB;
    base[(size_t)r * M.ld + c] = (c <= r) ? a[r][c] : 0.0;
    linv[e] = (c <= r) ? inv[r][c] : 0.0;
  }
}

// ------------------------------------------------------------------------------------
// 64 x 64 tile product  acc = sum_k opA(r,k) opB(c,k)
//   opA(r,k) = TA ? A[k*lda + r] : A[r*lda + k]   (likewise B)
// ------------------------------------------------------------------------------------
template <bool TA, bool TBt>
__device__ __forceinline__ void tile_mm(double (&acc)[4][4], const double* __restrict__ A, int lda,
                                        const double* __restrict__ B, int ldb, int k0, int k1) {
  __shared__ double As[16][TB];
  __shared__ double Bs[16][TB];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k = k0; k < k1; k += 16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      if (!TA) {
        const int r = e >> 4, kk = e & 15;
        As[kk][r] = A[(size_t)r * lda + k + kk];
      } else {
        const int kk = e >> 6, r = e & 63;
        As[kk][r] = A[(size_t)(k + kk) * lda + r];
      }
      if (!TBt) {
        const int r = e >> 4, kk = e & 15;
        Bs[kk][r] = B[(size_t)r * ldb + k + kk];
      } else {
        const int kk = e >> 6, r = e & 63;
        Bs[kk][r] = B[(size_t)(k + kk) * ldb + r];
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// C = alpha * C + beta * acc on the elements with (row < rlim, col < clim)
__device__ __forceinline__ void tile_store(double* C, int ldc, const double (&acc)[4][4], double alpha,
                                           double beta, int rlim = TB, int clim = TB) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < rlim && c < clim) {
        double* p = C + (size_t)r * ldc + c;
        *p = (alpha != 0.0) ? fma(beta, acc[i][j], alpha * *p) : beta * acc[i][j];
      }
    }
}

__device__ __forceinline__ void zero_acc(double (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
}

// panel: tile (i, kt) <- tile (i, kt) * Linv_kt^T  for i > kt
__global__ void __launch_bounds__(256) k_trsm_panel(Slot* slots, int sel, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  MatRef M = mat_ref(s, sel);
  const int T = M.n / TB, i = kt + 1 + blockIdx.x;
  if (i >= T) return;
  double acc[4][4];
  zero_acc(acc);
  double* C = M.A + (size_t)i * TB * M.ld + (size_t)kt * TB;
  tile_mm<false, false>(acc, C, M.ld, M.Linv + (size_t)kt * TB * TB, TB, 0, TB);
  tile_store(C, M.ld, acc, 0.0, 1.0);
}

// trailing update: tile (i, j) -= tile (i, kt) * tile (j, kt)^T, kt < j <= i
__global__ void __launch_bounds__(256) k_syrk_update(Slot* slots, int sel, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  MatRef M = mat_ref(s, sel);
  const int T = M.n / TB;
  int ii, jj;
  tri_decode(blockIdx.x, ii, jj);
  const int i = kt + 1 + ii, j = kt + 1 + jj;
  if (i >= T) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<false, false>(acc, M.A + (size_t)i * TB * M.ld + (size_t)kt * TB, M.ld,
                        M.A + (size_t)j * TB * M.ld + (size_t)kt * TB, M.ld, 0, TB);
  tile_store(M.A + (size_t)i * TB * M.ld + (size_t)j * TB, M.ld, acc, 1.0, -1.0);
}

// triangular inverse W = F^-1, block column jt (descending order), phase A:
//   W_ij = sum_{k = jt+1}^{i} W_ik F_k,jt   for i > jt
__global__ void __launch_bounds__(256) k_trtri_gemm(Slot* slots, int sel, int dst, int jt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  MatRef F = mat_ref(s, sel);
  double* W = dst == DST_L ? s.L : s.Wk;
  const int T = F.n / TB, i = jt + 1 + blockIdx.x;
  if (i >= T) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<false, true>(acc, W + (size_t)i * TB * F.ld, F.ld, F.A + (size_t)jt * TB, F.ld, (jt + 1) * TB,
                       (i + 1) * TB);
  tile_store(W + (size_t)i * TB * F.ld + (size_t)jt * TB, F.ld, acc, 0.0, 1.0);
}
// phase B: W_ij <- -W_ij * Finv_jt (i > jt);  W_jt,jt = Finv_jt
__global__ void __launch_bounds__(256) k_trtri_scale(Slot* slots, int sel, int dst, int jt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  MatRef F = mat_ref(s, sel);
  double* W = dst == DST_L ? s.L : s.Wk;
  const int T = F.n / TB, i = jt + blockIdx.x;
  if (i >= T) return;
  const double* finv = F.Linv + (size_t)jt * TB * TB;
  double* C = W + (size_t)i * TB * F.ld + (size_t)jt * TB;
  if (i == jt) {
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) C[(size_t)(e / TB) * F.ld + e % TB] = finv[e];
    return;
  }
  double acc[4][4];
  zero_acc(acc);
  tile_mm<false, true>(acc, C, F.ld, finv, TB, 0, TB);
  tile_store(C, F.ld, acc, 0.0, -1.0);
}

// Q_p[0:nd, 0:nd] lower tiles = W^T W, W = inverse covariance factor (held in L)
__global__ void __launch_bounds__(256) k_lauum_cov(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.nd == 0) return;
  const int Td = s.nd_pad / TB;
  int i, j;
  tri_decode(blockIdx.x, i, j);
  if (i >= Td) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<true, true>(acc, s.L + (size_t)i * TB, s.n_pad, s.L + (size_t)j * TB, s.n_pad, i * TB, s.nd_pad);
  tile_store(s.Qp + (size_t)(s.nd_off + i * TB) * s.n_pad + (size_t)(s.nd_off + j * TB), s.n_pad, acc, 0.0, 1.0,
             s.nd - i * TB, s.nd - j * TB);
}

// multi-RHS forward substitution L Z' = Z (Z: n_pad x k_pad), step kt
__global__ void __launch_bounds__(256) k_fwd_rhs_diag(Slot* slots, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int c = blockIdx.x;
  if (c >= s.k_pad / TB) return;
  double acc[4][4];
  zero_acc(acc);
  double* Zt = s.Z + (size_t)kt * TB * s.k_pad + (size_t)c * TB;
  tile_mm<false, true>(acc, s.Linv + (size_t)kt * TB * TB, TB, Zt, s.k_pad, 0, TB);
  tile_store(Zt, s.k_pad, acc, 0.0, 1.0);
}
__global__ void __launch_bounds__(256) k_fwd_rhs_upd(Slot* slots, int kt, int tk) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int i = kt + 1 + blockIdx.x / tk, c = blockIdx.x % tk;
  if (i >= s.n_pad / TB || c >= s.k_pad / TB) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<false, true>(acc, s.L + (size_t)i * TB * s.n_pad + (size_t)kt * TB, s.n_pad,
                       s.Z + (size_t)kt * TB * s.k_pad + (size_t)c * TB, s.k_pad, 0, TB);
  tile_store(s.Z + (size_t)i * TB * s.k_pad + (size_t)c * TB, s.k_pad, acc, 1.0, -1.0);
}

// S = Z^T Z (lower tiles), identity on the padded diagonal
__global__ void __launch_bounds__(256) k_schur_syrk(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  int i, j;
  tri_decode(blockIdx.x, i, j);
  if (i >= s.k_pad / TB) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<true, true>(acc, s.Z + (size_t)i * TB, s.k_pad, s.Z + (size_t)j * TB, s.k_pad, 0, s.n_pad);
  double* C = s.S + (size_t)i * TB * s.k_pad + (size_t)j * TB;
  tile_store(C, s.k_pad, acc, 0.0, 1.0);
  if (i == j) {
    __syncthreads();
    for (int r = threadIdx.x; r < TB; r += blockDim.x)
      if (i * TB + r >= s.k) C[(size_t)r * s.k_pad + r] = 1.0;
  }
}

// G^T = Z^T W  (k_pad x n_pad into L), W = Q*^-1 factor inverse (lower) in Wk
__global__ void __launch_bounds__(256) k_zt_w(Slot* slots, int tn) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int i = blockIdx.x / tn, j = blockIdx.x % tn;
  if (i >= s.k_pad / TB || j >= s.n_pad / TB) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<true, true>(acc, s.Z + (size_t)i * TB, s.k_pad, s.Wk + (size_t)j * TB, s.n_pad, j * TB, s.n_pad);
  tile_store(s.L + (size_t)i * TB * s.n_pad + (size_t)j * TB, s.n_pad, acc, 0.0, 1.0);
}

// forward substitution with the factor of S on X (k_pad x n_pad in L), step kt
__global__ void __launch_bounds__(256) k_fwd_s_diag(Slot* slots, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int c = blockIdx.x;
  if (c >= s.n_pad / TB) return;
  double acc[4][4];
  zero_acc(acc);
  double* X = s.L + (size_t)kt * TB * s.n_pad + (size_t)c * TB;
  tile_mm<false, true>(acc, s.SLinv + (size_t)kt * TB * TB, TB, X, s.n_pad, 0, TB);
  tile_store(X, s.n_pad, acc, 0.0, 1.0);
}
__global__ void __launch_bounds__(256) k_fwd_s_upd(Slot* slots, int kt, int tn) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int i = kt + 1 + blockIdx.x / tn, c = blockIdx.x % tn;
  if (i >= s.k_pad / TB || c >= s.n_pad / TB) return;
  double acc[4][4];
  zero_acc(acc);
  tile_mm<false, true>(acc, s.S + (size_t)i * TB * s.k_pad + (size_t)kt * TB, s.k_pad,
                       s.L + (size_t)kt * TB * s.n_pad + (size_t)c * TB, s.n_pad, 0, TB);
  tile_store(s.L + (size_t)i * TB * s.n_pad + (size_t)c * TB, s.n_pad, acc, 1.0, -1.0);
}

// ------------------------------------------------------------------------------------
// vector triangular solves (one launch per tile step; src is consumed, dst receives)
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_trsv_fwd(Slot* slots, int sel, int src, int dst, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  MatRef M = mat_ref(s, sel);
  const int T = M.n / TB, i = kt + blockIdx.x;
  if (i >= T) return;
  double* r = vec_ref(s, src);
  double* out = vec_ref(s, dst);
  __shared__ double rk[TB], y[TB];
  const double* linv = M.Linv + (size_t)kt * TB * TB;
  const int tid = threadIdx.x;
  if (tid < TB) rk[tid] = r[kt * TB + tid];
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  // y = Linv_kt * r_kt : warp w computes rows 8w..8w+7
  for (int row = warp * 8; row < warp * 8 + 8; ++row) {
    double v = linv[row * TB + lane] * rk[lane] + linv[row * TB + lane + 32] * rk[lane + 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) y[row] = v;
  }
  __syncthreads();
  if (i == kt) {
    if (tid < TB) out[kt * TB + tid] = y[tid];
    return;
  }
  const double* Lik = M.A + (size_t)i * TB * M.ld + (size_t)kt * TB;
  for (int row = warp * 8; row < warp * 8 + 8; ++row) {
    double v = Lik[(size_t)row * M.ld + lane] * y[lane] + Lik[(size_t)row * M.ld + lane + 32] * y[lane + 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) r[i * TB + row] -= v;
  }
}
__global__ void __launch_bounds__(256) k_trsv_bwd(Slot* slots, int sel, int src, int dst, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  MatRef M = mat_ref(s, sel);
  const int i = kt - (int)blockIdx.x;
  if (kt >= M.n / TB || i < 0) return;
  double* r = vec_ref(s, src);
  double* out = vec_ref(s, dst);
  __shared__ double rk[TB], y[TB];
  __shared__ double part[4][TB];
  const double* linv = M.Linv + (size_t)kt * TB * TB;
  const int tid = threadIdx.x;
  if (tid < TB) rk[tid] = r[kt * TB + tid];
  __syncthreads();
  // y = Linv_kt^T r_kt : y[c] = sum_k linv[k][c] r[k]; 4 groups of 16 k
  {
    const int c = tid & 63, g = tid >> 6;
    double v = 0.0;
    for (int k = g * 16; k < g * 16 + 16; ++k) v = fma(linv[k * TB + c], rk[k], v);
    part[g][c] = v;
  }
  __syncthreads();
  if (tid < TB) y[tid] = ((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid];
  __syncthreads();
  if (i == kt) {
    if (tid < TB) out[kt * TB + tid] = y[tid];
    return;
  }
  // r_i[c] -= sum_k L[kt*TB + k][i*TB + c] y[k]
  const double* Lki = M.A + (size_t)kt * TB * M.ld + (size_t)i * TB;
  {
    const int c = tid & 63, g = tid >> 6;
    double v = 0.0;
    for (int k = g * 16; k < g * 16 + 16; ++k) v = fma(Lki[(size_t)k * M.ld + c], y[k], v);
    part[g][c] = v;
  }
  __syncthreads();
  if (tid < TB) r[i * TB + tid] -= ((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid];
}

// ------------------------------------------------------------------------------------
// reductions
// ------------------------------------------------------------------------------------
// t1[j] = sum_{i >= j} Wk[i][j]^2 (lower triangular)
__global__ void __launch_bounds__(256) k_colsumsq_wk(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int jt = blockIdx.x;
  if (jt >= s.n_pad / TB) return;
  __shared__ double part[4][TB];
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  double v = 0.0;
  for (int i = jt * TB + g; i < s.n_pad; i += 4) {
    const double w = s.Wk[(size_t)i * s.n_pad + jt * TB + c];
    v = fma(w, w, v);
  }
  part[g][c] = v;
  __syncthreads();
  if (threadIdx.x < TB)
    s.t1[jt * TB + threadIdx.x] = ((part[0][threadIdx.x] + part[1][threadIdx.x]) + part[2][threadIdx.x]) +
                                  part[3][threadIdx.x];
}
// t2[j] = sum_{r < k_pad} L[r][j]^2   (the k_pad x n_pad matrix held in L)
__global__ void __launch_bounds__(256) k_colsumsq_gt(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int jt = blockIdx.x;
  if (jt >= s.n_pad / TB) return;
  __shared__ double part[4][TB];
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  double v = 0.0;
  for (int r = g; r < s.k_pad; r += 4) {
    const double w = s.L[(size_t)r * s.n_pad + jt * TB + c];
    v = fma(w, w, v);
  }
  part[g][c] = v;
  __syncthreads();
  if (threadIdx.x < TB)
    s.t2[jt * TB + threadIdx.x] = ((part[0][threadIdx.x] + part[1][threadIdx.x]) + part[2][threadIdx.x]) +
                                  part[3][threadIdx.x];
}

__global__ void __launch_bounds__(256) k_logdet(Slot* slots, int sel, int out_idx) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  MatRef M = mat_ref(s, sel);
  if (M.n == 0) {
    if (threadIdx.x == 0) s.out[out_idx] = 0.0;
    return;
  }
  double v = 0.0;
  for (int i = threadIdx.x; i < M.n; i += 256) v += log(M.A[(size_t)i * M.ld + i]);
  v = block_sum_256(v);
  if (threadIdx.x == 0) s.out[out_idx] = 2.0 * v;
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
static int tri(int t) { return t * (t + 1) / 2; }

void launch_potrf_diag(Slot* slots, int nslots, int sel, int kt, int max_t, cudaStream_t st) {
  (void)max_t;
  static DeviceFlags attr_set;  // the shared-memory limit is a per-device attribute
  const int smem = 2 * TB * (TB + 1) * (int)sizeof(double);
  const int dev = current_device();
  if (!attr_set.test(dev) &&
      cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess)
    attr_set.set(dev);
  count_launch("k_potrf_diag"), k_potrf_diag<<<nslots, 256, smem, st>>>(slots, sel, kt);
}
void launch_trsm_panel(Slot* slots, int nslots, int sel, int kt, int max_t, cudaStream_t st) {
  if (max_t - kt - 1 <= 0) return;
  count_launch("k_trsm_panel"), k_trsm_panel<<<dim3(max_t - kt - 1, nslots), 256, 0, st>>>(slots, sel, kt);
}
void launch_syrk_update(Slot* slots, int nslots, int sel, int kt, int max_t, cudaStream_t st) {
  const int t = max_t - kt - 1;
  if (t <= 0) return;
  count_launch("k_syrk_update"), k_syrk_update<<<dim3(tri(t), nslots), 256, 0, st>>>(slots, sel, kt);
}
void launch_trtri_step(Slot* slots, int nslots, int sel, int dst, int jt, int max_t, cudaStream_t st) {
  if (max_t - jt - 1 > 0) count_launch("k_trtri_gemm"), k_trtri_gemm<<<dim3(max_t - jt - 1, nslots), 256, 0, st>>>(slots, sel, dst, jt);
  count_launch("k_trtri_scale"), k_trtri_scale<<<dim3(max_t - jt, nslots), 256, 0, st>>>(slots, sel, dst, jt);
}
void launch_lauum_cov(Slot* slots, int nslots, int max_td, cudaStream_t st) {
  if (max_td <= 0) return;
  count_launch("k_lauum_cov"), k_lauum_cov<<<dim3(tri(max_td), nslots), 256, 0, st>>>(slots);
}
void launch_fwd_rhs_step(Slot* slots, int nslots, int kt, int max_t, int max_tk, cudaStream_t st) {
  count_launch("k_fwd_rhs_diag"), k_fwd_rhs_diag<<<dim3(max_tk, nslots), 256, 0, st>>>(slots, kt);
  if (max_t - kt - 1 > 0)
    count_launch("k_fwd_rhs_upd"), k_fwd_rhs_upd<<<dim3((max_t - kt - 1) * max_tk, nslots), 256, 0, st>>>(slots, kt, max_tk);
}
void launch_schur_syrk(Slot* slots, int nslots, int max_tk, int max_t, cudaStream_t st) {
  (void)max_t;
  count_launch("k_schur_syrk"), k_schur_syrk<<<dim3(tri(max_tk), nslots), 256, 0, st>>>(slots);
}
void launch_zt_w(Slot* slots, int nslots, int max_tk, int max_t, cudaStream_t st) {
  count_launch("k_zt_w"), k_zt_w<<<dim3(max_tk * max_t, nslots), 256, 0, st>>>(slots, max_t);
}
void launch_fwd_s_rhs_step(Slot* slots, int nslots, int kt, int max_tk, int max_t, cudaStream_t st) {
  count_launch("k_fwd_s_diag"), k_fwd_s_diag<<<dim3(max_t, nslots), 256, 0, st>>>(slots, kt);
  if (max_tk - kt - 1 > 0)
    count_launch("k_fwd_s_upd"), k_fwd_s_upd<<<dim3((max_tk - kt - 1) * max_t, nslots), 256, 0, st>>>(slots, kt, max_t);
}
void launch_trsv_fwd_step(Slot* slots, int nslots, int sel, int src, int dst, int kt, int max_t,
                          cudaStream_t st) {
  count_launch("k_trsv_fwd"), k_trsv_fwd<<<dim3(max_t - kt, nslots), 256, 0, st>>>(slots, sel, src, dst, kt);
}
void launch_trsv_bwd_step(Slot* slots, int nslots, int sel, int src, int dst, int kt, int max_t,
                          cudaStream_t st) {
  (void)max_t;
  count_launch("k_trsv_bwd"), k_trsv_bwd<<<dim3(kt + 1, nslots), 256, 0, st>>>(slots, sel, src, dst, kt);
}
void launch_colsumsq_wk(Slot* slots, int nslots, int max_t, cudaStream_t st) {
  count_launch("k_colsumsq_wk"), k_colsumsq_wk<<<dim3(max_t, nslots), 256, 0, st>>>(slots);
}
void launch_colsumsq_gt(Slot* slots, int nslots, int max_tk, int max_t, cudaStream_t st) {
  (void)max_tk;
  count_launch("k_colsumsq_gt"), k_colsumsq_gt<<<dim3(max_t, nslots), 256, 0, st>>>(slots);
}
void launch_logdet(Slot* slots, int nslots, int sel, int out_idx, cudaStream_t st) {
  count_launch("k_logdet"), k_logdet<<<nslots, 256, 0, st>>>(slots, sel, out_idx);
}

}  // namespace inla

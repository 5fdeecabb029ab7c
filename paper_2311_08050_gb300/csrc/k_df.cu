// Double-float (df64) variants of the O(n^2) kernels of the mixed path: conversions, the
// structured prior, A^T D A pair sums, Q_p x, triangular solves with the double-float
// factor, log-determinants and column sums of squares.  Arithmetic on the factor runs on
// the FP32 pipes (df64 operations); vectors and scalars stay FP64 (O(n) work).
#include "df64.cuh"
#include "device_util.cuh"
#include "kernels.h"
#include "mixed.h"

namespace inla {

__device__ __forceinline__ float2* dfm(double* p) { return reinterpret_cast<float2*>(p); }

struct DfRef {
  float2* A;
  double* Linv;
  int n, ld;
};
__device__ __forceinline__ DfRef df_ref(const Slot& s, int sel) {
  if (sel == SEL_L) return DfRef{dfm(s.L), s.Linv, s.n_pad, s.n_pad};
  if (sel == SEL_COV) return DfRef{dfm(s.Wk), s.Wd, s.nd_pad, s.n_pad};
  return DfRef{dfm(s.S), s.SLinv, s.k_pad, s.k_pad};
}
__device__ __forceinline__ double* vec_ref_df(const Slot& s, int v) {
  switch (v) {
    case 0: return s.g;
    case 1: return s.t1;
    case 2: return s.t2;
    case 3: return s.kv1;
    default: return s.kv2;
  }
}

// in-place FP64 -> df64 on the lower tiles of the dense covariance block (Wk)
__global__ void __launch_bounds__(256) k_cov_to_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.nd == 0) return;
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  if (ti >= s.nd_pad / TB) return;
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    double* p = s.Wk + (size_t)(ti * TB + e / TB) * s.n_pad + tj * TB + e % TB;
    const df v = df_from_double(*p);
    *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo);
  }
}

__global__ void k_prior_entries_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < md.nentries; e += (int64_t)gridDim.x * blockDim.x) {
    const PriorEntry pe = md.entries[e];
    const double v = pe.t >= 0 ? pe.a + pe.b * exp(s.theta[pe.t]) : pe.a;
    df_store(dfm(s.Qp) + (size_t)pe.row * s.n_pad + pe.col, df_from_double(v));
  }
}

// L[row][col] += sum w c  (pair sums in FP64, added in df64)
__global__ void __launch_bounds__(256) k_add_pairs_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp0; p < md.npairs; p += nwarps) {
    const int64_t lo = md.pair_ptr[p], hi = md.pair_ptr[p + 1];
    double v = 0.0;
    for (int64_t c = lo + lane; c < hi; c += 32) v = fma(s.w[md.pc_obs[c]], md.pc_coef[c], v);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      float2* q = dfm(s.L) + (size_t)md.pair_row[p] * s.n_pad + md.pair_col[p];
      df_store(q, df_add(df_load(q), df_from_double(v)));
    }
  }
}

// vd = double-float copy of x (which = 0) or xn (which = 1)
__global__ void __launch_bounds__(256) k_vec_to_df(Slot* slots, int which) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const double* v = which ? s.xn : s.x;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < s.n_pad; j += gridDim.x * 256) df_store(dfm(s.vd) + j, df_from_double(v[j]));
}

// t1 = Q_p v (df64 Q_p, full symmetric; v from vd), one warp per row
__global__ void __launch_bounds__(256) k_qp_gemv_df(Slot* slots, int which) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  (void)which;
  const float2* vd = dfm(s.vd);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = s.n_pad;
  for (int row = blockIdx.x * 8 + warp; row < n; row += gridDim.x * 8) {
    const float2* q = dfm(s.Qp) + (size_t)row * n;
    df acc = df_make(0.f, 0.f);
    for (int c = lane; c < n; c += 32) acc = df_fma(acc, df_load(q + c), df_load(vd + c));
    double r = df_to_double(acc);
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) s.t1[row] = r;
  }
}

// t2 = Z kv1 (df64 Z, n_pad x k_pad)
__global__ void __launch_bounds__(256) k_z_gemv_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row = blockIdx.x * 8 + warp; row < s.n_pad; row += gridDim.x * 8) {
    const float2* z = dfm(s.Z) + (size_t)row * s.k_pad;
    df acc = df_make(0.f, 0.f);
    for (int c = lane; c < s.k_pad; c += 32) acc = df_fma(acc, df_load(z + c), df_from_double(s.kv1[c]));
    double r = df_to_double(acc);
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) s.t2[row] = r;
  }
}

// Z = dense C^T in df64 (caller zeroed Z)
__global__ void __launch_bounds__(256) k_ct_fill_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const ModelDev& md = *s.md;
  for (int r = blockIdx.x * 256 + threadIdx.x; r < s.k; r += gridDim.x * 256)
    for (int64_t e = md.C_rowptr[r]; e < md.C_rowptr[r + 1]; ++e)
      df_store(dfm(s.Z) + (size_t)md.C_col[e] * s.k_pad + r, df_from_double(md.C_val[e]));
}

// identity on the padded diagonal of S
__global__ void k_s_pad_identity(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  for (int r = s.k + blockIdx.x * 256 + threadIdx.x; r < s.k_pad; r += gridDim.x * 256)
    df_store(dfm(s.S) + (size_t)r * s.k_pad + r, df_make(1.f, 0.f));
}

// identity on the lower triangle of an n_pad x n_pad df64 matrix (W before the inverse)
__global__ void __launch_bounds__(256) k_set_identity_df(Slot* slots, int which_wk, int size_sel) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int n = size_sel == SEL_COV ? s.nd_pad : s.n_pad;
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  if (ti >= n / TB) return;
  float2* W = dfm(which_wk ? s.Wk : s.L);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int r = ti * TB + e / TB, c = tj * TB + e % TB;
    W[(size_t)r * s.n_pad + c] = make_float2(r == c ? 1.f : 0.f, 0.f);
  }
}

// diagonal 64-tile: load df64, Cholesky + triangular inverse in FP64 (shared memory),
// store the factor tile in df64 (upper part zeroed) and its inverse in FP64
__global__ void __launch_bounds__(256) k_potrf_diag_df(Slot* slots, int sel, int kt) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  DfRef M = df_ref(s, sel);
  if (kt * TB >= M.n) return;
  extern __shared__ double smem[];
  double(*a)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(smem);
  double(*inv)[TB + 1] = reinterpret_cast<double(*)[TB + 1]>(smem + TB * (TB + 1));
  __shared__ int bad;
  const int tid = threadIdx.x;
  float2* base = M.A + (size_t)kt * TB * M.ld + (size_t)kt * TB;
  for (int e = tid; e < TB * TB; e += blockDim.x) a[e / TB][e % TB] = df_to_double(df_load(base + (size_t)(e / TB) * M.ld + e % TB));
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
    const double rdjj = 1.0 / a[j][j];
    for (int i = j + 1 + tid; i < TB; i += blockDim.x) a[i][j] = a[i][j] * rdjj;
    __syncthreads();
    for (int i = j + 1 + ty; i < TB; i += 16)
      for (int c = j + 1 + tx; c <= i; c += 16) a[i][c] = fma(-a[i][j], a[c][j], a[i][c]);
    __syncthreads();
  }
  __shared__ double rdiag[TB];
  if (tid < TB) rdiag[tid] = 1.0 / a[tid][tid];
  __syncthreads();
  if (tid < TB) {
    const int c = tid;
    for (int i = 0; i < c; ++i) inv[i][c] = 0.0;
    inv[c][c] = rdiag[c];
    for (int i = c + 1; i < TB; ++i) {
      double acc0 = 0.0, acc1 = 0.0;
      int k = c;
      for (; k + 1 < i; k += 2) {
        acc0 = fma(a[i][k], inv[k][c], acc0);
        acc1 = fma(a[i][k + 1], inv[k + 1][c], acc1);
      }
      if (k < i) acc0 = fma(a[i][k], inv[k][c], acc0);
      inv[i][c] = -(acc0 + acc1) * rdiag[i];
    }
  }
  __syncthreads();
  double* linv = M.Linv + (size_t)kt * TB * TB;
  for (int e = tid; e < TB * TB; e += blockDim.x) {
    const int r = e / TB, c = e % TB;
    df_store(base + (size_t)r * M.ld + c, c <= r ? df_from_double(a[r][c]) : df_make(0.f, 0.f));
    linv[e] = (c <= r) ? inv[r][c] : 0.0;
  }
}

// vector triangular solves with a df64 factor (FP64 Linv tiles, FP64 vectors)
__global__ void __launch_bounds__(256) k_trsv_fwd_df(Slot* slots, int sel, int src, int dst, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  DfRef M = df_ref(s, sel);
  const int T = M.n / TB, i = kt + blockIdx.x;
  if (i >= T) return;
  double* r = vec_ref_df(s, src);
  double* out = vec_ref_df(s, dst);
  __shared__ double rk[TB], y[TB];
  __shared__ float2 yd[TB];
  const double* linv = M.Linv + (size_t)kt * TB * TB;
  const int tid = threadIdx.x;
  if (tid < TB) rk[tid] = r[kt * TB + tid];
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
  for (int row = warp * 8; row < warp * 8 + 8; ++row) {
    double v = linv[row * TB + lane] * rk[lane] + linv[row * TB + lane + 32] * rk[lane + 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      y[row] = v;
      const df t = df_from_double(v);
      yd[row] = make_float2(t.hi, t.lo);
    }
  }
  __syncthreads();
  if (i == kt) {
    if (tid < TB) out[kt * TB + tid] = y[tid];
    return;
  }
  const float2* Lik = M.A + (size_t)i * TB * M.ld + (size_t)kt * TB;
  for (int row = warp * 8; row < warp * 8 + 8; ++row) {
    df acc = df_mul(df_load(Lik + (size_t)row * M.ld + lane), df_make(yd[lane].x, yd[lane].y));
    acc = df_fma(acc, df_load(Lik + (size_t)row * M.ld + lane + 32), df_make(yd[lane + 32].x, yd[lane + 32].y));
    double v = df_to_double(acc);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) r[i * TB + row] -= v;
  }
}
__global__ void __launch_bounds__(256) k_trsv_bwd_df(Slot* slots, int sel, int src, int dst, int kt) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  DfRef M = df_ref(s, sel);
  const int i = kt - (int)blockIdx.x;
  if (kt >= M.n / TB || i < 0) return;
  double* r = vec_ref_df(s, src);
  double* out = vec_ref_df(s, dst);
  __shared__ double rk[TB], y[TB];
  __shared__ float2 yd[TB];
  __shared__ double part[4][TB];
  const double* linv = M.Linv + (size_t)kt * TB * TB;
  const int tid = threadIdx.x;
  if (tid < TB) rk[tid] = r[kt * TB + tid];
  __syncthreads();
  {
    const int c = tid & 63, g = tid >> 6;
    double v = 0.0;
    for (int k = g * 16; k < g * 16 + 16; ++k) v = fma(linv[k * TB + c], rk[k], v);
    part[g][c] = v;
  }
  __syncthreads();
  if (tid < TB) {
    y[tid] = ((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid];
    const df t = df_from_double(y[tid]);
    yd[tid] = make_float2(t.hi, t.lo);
  }
  __syncthreads();
  if (i == kt) {
    if (tid < TB) out[kt * TB + tid] = y[tid];
    return;
  }
  const float2* Lki = M.A + (size_t)kt * TB * M.ld + (size_t)i * TB;
  {
    const int c = tid & 63, g = tid >> 6;
    df acc = df_make(0.f, 0.f);
    for (int k = g * 16; k < g * 16 + 16; ++k) acc = df_fma(acc, df_load(Lki + (size_t)k * M.ld + c), df_make(yd[k].x, yd[k].y));
    part[g][c] = df_to_double(acc);
  }
  __syncthreads();
  if (tid < TB) r[i * TB + tid] -= ((part[0][tid] + part[1][tid]) + part[2][tid]) + part[3][tid];
}

__global__ void __launch_bounds__(256) k_logdet_df(Slot* slots, int sel, int out_idx) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) return;
  DfRef M = df_ref(s, sel);
  double v = 0.0;
  for (int i = threadIdx.x; i < M.n; i += 256) v += log(df_to_double(df_load(M.A + (size_t)i * M.ld + i)));
  v = block_sum_256(v);
  if (threadIdx.x == 0) s.out[out_idx] = 2.0 * v;
}

// t1[j] = sum_{i >= j} Wk[i][j]^2 (df64 W, lower)
__global__ void __launch_bounds__(256) k_colsumsq_wk_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int jt = blockIdx.x;
  if (jt >= s.n_pad / TB) return;
  __shared__ double part[4][TB];
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  df acc = df_make(0.f, 0.f);
  const float2* W = dfm(s.Wk);
  for (int i = jt * TB + g; i < s.n_pad; i += 4) {
    const df w = df_load(W + (size_t)i * s.n_pad + jt * TB + c);
    acc = df_fma(acc, w, w);
  }
  part[g][c] = df_to_double(acc);
  __syncthreads();
  if (threadIdx.x < TB)
    s.t1[jt * TB + threadIdx.x] = ((part[0][threadIdx.x] + part[1][threadIdx.x]) + part[2][threadIdx.x]) + part[3][threadIdx.x];
}
// t2[j] = sum_{r < k_pad} L[r][j]^2 (df64 k_pad x n_pad held in L)
__global__ void __launch_bounds__(256) k_colsumsq_gt_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const int jt = blockIdx.x;
  if (jt >= s.n_pad / TB) return;
  __shared__ double part[4][TB];
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  df acc = df_make(0.f, 0.f);
  const float2* X = dfm(s.L);
  for (int r = g; r < s.k_pad; r += 4) {
    const df w = df_load(X + (size_t)r * s.n_pad + jt * TB + c);
    acc = df_fma(acc, w, w);
  }
  part[g][c] = df_to_double(acc);
  __syncthreads();
  if (threadIdx.x < TB)
    s.t2[jt * TB + threadIdx.x] = ((part[0][threadIdx.x] + part[1][threadIdx.x]) + part[2][threadIdx.x]) + part[3][threadIdx.x];
}

// ---------------- launchers ----------------
static int tri(int t) { return t * (t + 1) / 2; }
static int vgrid(int n) { return std::min(1024, std::max(1, (n + 255) / 256)); }

void launch_cov_to_df(Slot* slots, int nslots, int max_td, cudaStream_t st) {
  if (max_td > 0) count_launch("k_cov_to_df"), k_cov_to_df<<<dim3(tri(max_td), nslots), 256, 0, st>>>(slots);
}
void launch_prior_entries_df(Slot* slots, int nslots, int64_t max_entries, cudaStream_t st) {
  if (max_entries > 0)
    count_launch("k_prior_entries_df"), k_prior_entries_df<<<dim3((unsigned)std::min<int64_t>(2048, (max_entries + 255) / 256), nslots), 256, 0, st>>>(slots);
}
void launch_add_pairs_df(Slot* slots, int nslots, int64_t max_pairs, cudaStream_t st) {
  if (max_pairs > 0)
    count_launch("k_add_pairs_df"), k_add_pairs_df<<<dim3((unsigned)std::min<int64_t>(4096, (max_pairs + 7) / 8), nslots), 256, 0, st>>>(slots);
}
void launch_qp_gemv_df(Slot* slots, int nslots, int which, int max_n, cudaStream_t st) {
  count_launch("k_vec_to_df"), k_vec_to_df<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots, which);
  count_launch("k_qp_gemv_df"), k_qp_gemv_df<<<dim3(std::min(4096, (max_n + 7) / 8), nslots), 256, 0, st>>>(slots, which);
}
void launch_z_gemv_df(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_z_gemv_df"), k_z_gemv_df<<<dim3(std::min(4096, (max_n + 7) / 8), nslots), 256, 0, st>>>(slots);
}
void launch_ct_fill_df(Slot* slots, int nslots, int max_k, cudaStream_t st) {
  count_launch("k_ct_fill_df"), k_ct_fill_df<<<dim3(vgrid(max_k), nslots), 256, 0, st>>>(slots);
}
void launch_s_pad_identity(Slot* slots, int nslots, int max_k, cudaStream_t st) {
  count_launch("k_s_pad_identity"), k_s_pad_identity<<<dim3(vgrid(max_k), nslots), 256, 0, st>>>(slots);
}
void launch_set_identity_df(Slot* slots, int nslots, int which_wk, int size_sel, int max_t, cudaStream_t st) {
  count_launch("k_set_identity_df"), k_set_identity_df<<<dim3(tri(max_t), nslots), 256, 0, st>>>(slots, which_wk, size_sel);
}
void launch_potrf_diag_df(Slot* slots, int nslots, int sel, int kt, cudaStream_t st) {
  static bool init = false;
  const int smem = 2 * TB * (TB + 1) * (int)sizeof(double);
  if (!init) {
    cudaFuncSetAttribute(k_potrf_diag_df, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    init = true;
  }
  count_launch("k_potrf_diag_df"), k_potrf_diag_df<<<nslots, 256, smem, st>>>(slots, sel, kt);
}
void launch_trsv_fwd_df(Slot* slots, int nslots, int sel, int src, int dst, int kt, int max_t, cudaStream_t st) {
  count_launch("k_trsv_fwd_df"), k_trsv_fwd_df<<<dim3(max_t - kt, nslots), 256, 0, st>>>(slots, sel, src, dst, kt);
}
void launch_trsv_bwd_df(Slot* slots, int nslots, int sel, int src, int dst, int kt, cudaStream_t st) {
  count_launch("k_trsv_bwd_df"), k_trsv_bwd_df<<<dim3(kt + 1, nslots), 256, 0, st>>>(slots, sel, src, dst, kt);
}
void launch_logdet_df(Slot* slots, int nslots, int sel, int out_idx, cudaStream_t st) {
  count_launch("k_logdet_df"), k_logdet_df<<<nslots, 256, 0, st>>>(slots, sel, out_idx);
}
void launch_colsumsq_wk_df(Slot* slots, int nslots, int max_t, cudaStream_t st) {
  count_launch("k_colsumsq_wk_df"), k_colsumsq_wk_df<<<dim3(max_t, nslots), 256, 0, st>>>(slots);
}
void launch_colsumsq_gt_df(Slot* slots, int nslots, int max_t, cudaStream_t st) {
  count_launch("k_colsumsq_gt_df"), k_colsumsq_gt_df<<<dim3(max_t, nslots), 256, 0, st>>>(slots);
}

}  // namespace inla

namespace inla {
__global__ void k_add_cct_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.k == 0) return;
  const ModelDev& md = *s.md;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < md.ncct; e += (int64_t)gridDim.x * blockDim.x) {
    const PriorEntry pe = md.cct[e];
    float2* q = dfm(s.L) + (size_t)pe.row * s.n_pad + pe.col;
    df_store(q, df_add(df_load(q), df_from_double(md.gamma_c * pe.a)));
  }
}
void launch_add_cct_df(Slot* slots, int nslots, cudaStream_t st) {
  count_launch("k_add_cct_df"), k_add_cct_df<<<dim3(1024, nslots), 256, 0, st>>>(slots);
}
}  // namespace inla

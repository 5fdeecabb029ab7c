// Double-float (df64) variants of the O(n^2) kernels of the mixed path: conversions, the
// structured prior, A^T D A pair sums, Q_p x, triangular solves with the double-float
// factor, log-determinants and column sums of squares.  Arithmetic on the factor runs on
// the FP32 pipes (df64 operations); vectors and scalars stay FP64 (O(n) work).
#include "df64.cuh"
#include "df_exp.cuh"
#include "device_util.cuh"
#include "kernels.h"
#include "mixed.h"
#include "oz_slice.cuh"

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
  if (sel == SEL_AUX) return DfRef{dfm(s.Qp), s.Linv, s.aux_n, s.n_pad};
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

// Dense covariance block Sigma_ij = sigma^2 exp(-d_ij) (+ the diagonal term), written in
// double-float straight into Wk (lower tiles; identity on the padding): the distance
// d = sqrt((dx / rho_x)^2 + (dy / rho_y)^2) and the exponential run in double-float on the
// FP32 pipes.  The tile's 2 x 64 points are converted once per block (shared memory).
__device__ __forceinline__ df cov_entry_df(df xi, df yi, df xj, df yj, df irx, df iry, df sigma2) {
  const df dx = df_mul(df_add(xi, df_neg(xj)), irx);
  const df dy = df_mul(df_add(yi, df_neg(yj)), iry);
  const df d2 = df_add(df_mul(dx, dx), df_mul(dy, dy));
  if (!(d2.hi > 0.f)) return sigma2;
  return df_mul(sigma2, df_exp_neg(df_sqrt(d2)));
}

__global__ void __launch_bounds__(256) k_cov_build_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active || s.nd == 0) return;
  const ModelDev& md = *s.md;
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  if (ti >= s.nd_pad / TB) return;
  __shared__ float2 px[2][TB], py[2][TB];  // [0]: row points, [1]: column points
  const double* P = md.points;
  if (threadIdx.x < 2 * TB) {
    const int side = threadIdx.x / TB, e = threadIdx.x % TB;
    const int idx = (side ? tj : ti) * TB + e;
    df x = df_make(0.f, 0.f), y = df_make(0.f, 0.f);
    if (idx < s.nd) {
      x = df_from_double(P[2 * idx]);
      y = df_from_double(P[2 * idx + 1]);
    }
    px[side][e] = make_float2(x.hi, x.lo);
    py[side][e] = make_float2(y.hi, y.lo);
  }
  __syncthreads();
  const df sigma2 = df_from_double(exp(2.0 * s.theta[md.theta_sigma]));
  const df irx = df_from_double(exp(-s.theta[md.theta_rx]));
  const df iry = df_from_double(exp(-s.theta[md.theta_ry]));
  double diag_add = md.nugget;
  if (md.theta_iid >= 0) diag_add += exp(-s.theta[md.theta_iid]);
  const df dadd = df_from_double(diag_add);
  for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
    const int a = e / TB, b = e % TB;
    const int i = ti * TB + a, j = tj * TB + b;
    df v;
    if (i < s.nd && j < s.nd) {
      v = cov_entry_df(df_make(px[0][a].x, px[0][a].y), df_make(py[0][a].x, py[0][a].y), df_make(px[1][b].x, px[1][b].y),
                       df_make(py[1][b].x, py[1][b].y), irx, iry, sigma2);
      if (i == j) v = df_add(v, dadd);
    } else {
      v = df_make(i == j ? 1.f : 0.f, 0.f);
    }
    df_store(dfm(s.Wk) + (size_t)i * s.n_pad + j, v);
  }
}

// test hook support: Sigma entries for raw points (row-major n x 2) in double-float, as FP64
__global__ void k_cov_points_df(const double* P, int n, double sigma2, double irx, double iry, double* out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const df v = cov_entry_df(df_from_double(P[2 * i]), df_from_double(P[2 * i + 1]), df_from_double(P[2 * j]),
                              df_from_double(P[2 * j + 1]), df_from_double(irx), df_from_double(iry),
                              df_from_double(sigma2));
    out[e] = df_to_double(v);
  }
}
void launch_cov_points_df(const double* P, int n, double sigma2, double irx, double iry, double* out, cudaStream_t st) {
  count_launch("k_cov_points_df"), k_cov_points_df<<<256, 256, 0, st>>>(P, n, sigma2, irx, iry, out);
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
  if (blockIdx.x < HEAVY_BLOCKS) {  // heavy pairs: a whole block each (fixed-order tree)
    for (int h = blockIdx.x; h < md.n_heavy_pairs; h += HEAVY_BLOCKS) {
      const int64_t p = md.heavy_pairs[h];
      double v = 0.0;
      for (int64_t c = md.pair_ptr[p] + threadIdx.x; c < md.pair_ptr[p + 1]; c += 256)
        v = fma(s.w[md.pc_obs[c]], md.pc_coef[c], v);
      v = block_sum_256(v);
      if (threadIdx.x == 0) {
        float2* q = dfm(s.L) + (size_t)md.pair_row[p] * s.n_pad + md.pair_col[p];
        df_store(q, df_add(df_load(q), df_from_double(v)));
      }
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

// t1 = Q_p v from the lower triangle of the symmetric Q_p (df64, stored mirrored; v from vd), so
// that each element below the diagonal tiles is read once.  Block (tile row I, slot), the longest
// rows first: each 64 x 64 tile (I, J <= I) is staged in shared memory; its row sums Q_IJ v_J
// accumulate into t1's tile I (the diagonal tile in full), and for J < I its column sums
// Q_IJ^T v_I go to qpart[I][tile J], which k_qp_symv_sum_df adds to t1's tile J in a fixed order.
// Thread (row or column tid & 63, 16-wide quarter tid >> 6); the next tile is loaded into
// registers while the current one is summed.
__global__ void __launch_bounds__(256) k_qp_symv_part_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int n = s.n_pad, T = n / TB;
  const int I = T - 1 - (int)blockIdx.x;
  if (I < 0) return;
  __shared__ float2 tile[TB][TB + 1];
  __shared__ float2 vi[TB], vj[TB];
  __shared__ float2 cpart[4][TB];
  const int tid = threadIdx.x, r = tid & 63, q = tid >> 6;
  const float2* Q = dfm(s.Qp);
  const float2* vd = dfm(s.vd);
  if (tid < TB) vi[tid] = vd[I * TB + tid];
  float2 nxt[16];
  auto load = [&](int J) {
#pragma unroll
    for (int k = 0; k < 16; ++k) nxt[k] = Q[(size_t)(I * TB + k * 4 + q) * n + J * TB + r];
  };
  load(0);
  df rowacc = df_make(0.f, 0.f);
  for (int J = 0; J <= I; ++J) {
    __syncthreads();  // the previous tile and its column sums are consumed
#pragma unroll
    for (int k = 0; k < 16; ++k) tile[k * 4 + q][r] = nxt[k];
    if (tid < TB) vj[tid] = vd[J * TB + tid];
    __syncthreads();
    if (J < I) load(J + 1);
    df a = df_make(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < 16; ++c) a = df_add_fast(a, df_mul(df_load(&tile[r][q * 16 + c]), df_load(&vj[q * 16 + c])));
    rowacc = df_add(rowacc, a);
    if (J < I) {
      df b = df_make(0.f, 0.f);
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) b = df_add_fast(b, df_mul(df_load(&tile[q * 16 + rr][r]), df_load(&vi[q * 16 + rr])));
      cpart[q][r] = make_float2(b.hi, b.lo);
      __syncthreads();
      if (tid < TB) {
        df c2 = df_load(&cpart[0][tid]);
        for (int h = 1; h < 4; ++h) c2 = df_add(c2, df_load(&cpart[h][tid]));
        s.qpart[(size_t)I * n + J * TB + tid] = df_to_double(c2);
      }
    }
  }
  __syncthreads();
  cpart[q][r] = make_float2(rowacc.hi, rowacc.lo);
  __syncthreads();
  if (tid < TB) {
    df t = df_load(&cpart[0][tid]);
    for (int h = 1; h < 4; ++h) t = df_add(t, df_load(&cpart[h][tid]));
    s.t1[I * TB + tid] = df_to_double(t);
  }
}
// t1_j += sum over the tile rows I below j's tile of qpart[I][j], in increasing I
__global__ void __launch_bounds__(256) k_qp_symv_sum_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int n = s.n_pad, T = n / TB;
  for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256) {
    double a = 0.0;
    for (int I = j / TB + 1; I < T; ++I) a += s.qpart[(size_t)I * n + j];
    s.t1[j] += a;
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

// Diagonal 64-tile: Cholesky factor and its inverse in double-float on the FP32 pipes (this
// GPU's FP64 rate is ~2 FMA/clock/SM).  One CTA of DG_THREADS threads per tile, the tile in shared
// memory (row pitch 65 cells).  Factor: right-looking elimination A = L1 D L1^T, step j
// subtracting (a_ij / a_jj) a_cj from every a_ic with i >= c > j.  The lower triangle is listed by
// column, last column first, rows ascending, so the elements step j updates are the first
// (63 - j)(64 - j) / 2 positions of the list and column j + 1 is the last 64 - (j + 1) of them.
// Thread t owns positions t, t + DG_THREADS, .. and keeps those elements in registers for the
// whole elimination: at step j it reads a_ij and a_cj (column j, final) from shared memory, and
// publishes an element there once it is final (when its column is j + 1); the owner of the next
// pivot a_{j+1,j+1} also publishes its reciprocal, so one barrier per step closes it and warps
// whose positions are all past the step's prefix only meet the barrier.  Then L = L1 D^1/2 is
// written out and L1 is inverted in place by levels (s = 1, 2, .., 32: two inverted diagonal
// blocks of size s and the block below them give the inverse of the 2s block, -Y22 L21 Y11), so
// L^-1 = D^-1/2 Y.  Stores the factor tile (double-float, upper part zeroed) and the inverse tile
// (double-float, in the FP64-sized cells of the inverse-tile array).  With `pb.planes` set it also
// slices the inverse tile as the 64-row, K = 64 operand pb (one exponent per row, 8 values per
// lane), exactly as the row slicer would from the stored tile; a slot that is inactive or has no
// tile kt gets zero slices, so the product adds nothing to it.
constexpr int DG_LD = TB + 1;
constexpr int DG_THREADS = 1024;
// 1 / a for the tile's pivot chain: the PTX approximate reciprocal (within 1 ulp over the whole
// FP32 range) refined by one Newton step r0 + r0 (1 - a r0) in double-float, ~2^-44 relative;
// ~17 cycles shorter than an IEEE-rounded seed on every elimination step
__device__ __forceinline__ df dg_recip(df a) {
  float r0;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r0) : "f"(a.hi));
  const float e = __fmaf_rn(-a.lo, r0, __fmaf_rn(-a.hi, r0, 1.0f));
  float s, t;
  fast_two_sum(r0, r0 * e, s, t);
  return df{s, t};
}
__device__ __forceinline__ df dg_ld(const float2* t, int i, int c) { return df_make(t[i * DG_LD + c].x, t[i * DG_LD + c].y); }
__device__ __forceinline__ void dg_st(float2* t, int i, int c, df v) { t[i * DG_LD + c] = make_float2(v.hi, v.lo); }

__device__ __forceinline__ void dg_zero_slices(const OzOperand& pb, int S) {
  if (!pb.planes) return;
  const int slot = blockIdx.x;
  uint16_t* planes = pb.planes + (int64_t)slot * S * pb.plane_stride;
  for (int e = threadIdx.x; e < S * TB * (TB / 8); e += blockDim.x) {
    const int sl = e / (TB * (TB / 8)), rem = e % (TB * (TB / 8)), i = rem >> 3, g = rem & 7;
    *reinterpret_cast<uint4*>(planes + sl * pb.plane_stride + (int64_t)i * pb.ld_k + 8 * g) = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x < TB) pb.exps[slot * pb.exp_slot_stride + threadIdx.x] = 0;
}

__global__ void __launch_bounds__(DG_THREADS) k_potrf_diag_df(Slot* slots, int sel, int kt, OzOperand pb, int S) {
  const Slot& s = slots[blockIdx.x];
  if (!s.active) {
    dg_zero_slices(pb, S);
    return;
  }
  DfRef M = df_ref(s, sel);
  if (kt * TB >= M.n) {
    dg_zero_slices(pb, S);
    return;
  }
  constexpr int NTRI = TB * (TB + 1) / 2;  // 2080 lower-triangle elements (diagonal included)
  constexpr int NQ = (NTRI + DG_THREADS - 1) / DG_THREADS;  // positions per thread
  __shared__ float2 t[TB * DG_LD];
  __shared__ float2 rpa[TB];               // 1 / a_jj
  __shared__ float2 dsq[TB], rdq[TB];      // sqrt(a_jj), 1 / sqrt(a_jj)
  __shared__ int bad_sh;
  const int tid = threadIdx.x;
  float2* base = M.A + (size_t)kt * TB * M.ld + (size_t)kt * TB;
  if (tid == 0) bad_sh = 0;
  for (int e = tid; e < TB * TB; e += DG_THREADS) {
    const int i = e >> 6, c = e & 63;
    if (c <= i) t[i * DG_LD + c] = base[(size_t)i * M.ld + c];
  }
  __syncthreads();
  auto pivot_recip = [&](df p, int j) {
    if (!(p.hi > 0.f) || !isfinite(p.hi)) {
      bad_sh = 1;
      atomicMin(&s.info[1], kt * TB + j);
      p = df_make(1.f, 0.f);
    }
    const df r = dg_recip(p);
    rpa[j] = make_float2(r.hi, r.lo);
  };
  // owned elements: position p = tid + DG_THREADS q lies in column c = 63 - w, w the largest
  // integer with w (w + 1) / 2 <= p, at row c + p - w (w + 1) / 2
  df av[NQ];
  int pq[NQ], rof[NQ], cof[NQ], col[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int p = tid + DG_THREADS * q;
    pq[q] = p < NTRI ? p : NTRI;           // NTRI: never in a step's prefix
    int w = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    if (w > TB - 1) w = TB - 1;
    if (w < 0) w = 0;
    if ((w + 1) * (w + 2) / 2 <= p && w < TB - 1) ++w;
    if (w * (w + 1) / 2 > p && w > 0) --w;
    const int c = TB - 1 - w, i = min(c + p - w * (w + 1) / 2, TB - 1);
    rof[q] = i * DG_LD;
    cof[q] = c * DG_LD;
    col[q] = c;
    av[q] = p < NTRI ? dg_ld(t, i, c) : df_make(0.f, 0.f);
  }
  if (tid == 0) pivot_recip(dg_ld(t, 0, 0), 0);
  __syncthreads();
  // ---- factor: 63 elimination steps, one barrier each ----
  for (int j = 0; j < TB - 1; ++j) {
    const int w = TB - 1 - j;                // columns j+1 .. 63: w of them
    const int cnt = w * (w + 1) / 2;         // the step's prefix of the list
    const int nxt = cnt - w;                 // column j+1 starts here, with its pivot
    if (tid < cnt) {
      const df r = df_make(rpa[j].x, rpa[j].y);
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (pq[q] < cnt) {
          const df u = dg_ld(t, 0, rof[q] + j), b = dg_ld(t, 0, cof[q] + j);
          av[q] = df_add_fast(av[q], df_neg(df_mul(df_mul(u, r), b)));
          if (pq[q] >= nxt) {                // column j+1: final now
            dg_st(t, 0, rof[q] + col[q], av[q]);
            if (pq[q] == nxt) pivot_recip(av[q], j + 1);
          }
        }
    }
    __syncthreads();
  }
  if (bad_sh && tid == 0) atomicOr(&s.info[0], INFO_NOT_SPD);
  // ---- unit factor L1 (in place below the diagonal), sqrt of the pivots ----
  if (tid < TB) {
    df p = dg_ld(t, tid, tid);
    if (!(p.hi > 0.f) || !isfinite(p.hi)) p = df_make(1.f, 0.f);
    const df d = df_sqrt(p), rd = dg_recip(d);
    dsq[tid] = make_float2(d.hi, d.lo);
    rdq[tid] = make_float2(rd.hi, rd.lo);
  }
  for (int e = tid; e < TB * TB; e += DG_THREADS) {
    const int i = e >> 6, c = e & 63;
    if (i > c) dg_st(t, i, c, df_mul(dg_ld(t, i, c), df_make(rpa[c].x, rpa[c].y)));
  }
  __syncthreads();
  // ---- L = L1 D^1/2 to global (upper part zeroed) ----
  for (int e = tid; e < TB * TB; e += DG_THREADS) {
    const int i = e >> 6, c = e & 63;
    df v = df_make(0.f, 0.f);
    if (c < i) v = df_mul(dg_ld(t, i, c), df_make(dsq[c].x, dsq[c].y));
    else if (c == i) v = df_make(dsq[i].x, dsq[i].y);
    base[(size_t)i * M.ld + c] = make_float2(v.hi, v.lo);
  }
  // ---- Y = L1^-1 in place, level by level (unit diagonal implicit); level s has 64 / (2 s)
  // blocks of s x s outputs, 32 s in all, OPT = 1024 / DG_THREADS of them per thread at most.
  // In T the sum's length depends on the column, in Y21 on the row: the index that sets it is
  // the slow one (one value per warp at s = 32), so a warp's lanes run equal loops; each sum
  // runs in two interleaved accumulators ----
  constexpr int OPT = (32 * 32 + DG_THREADS - 1) / DG_THREADS;
  for (int sz = 1; sz < TB; sz <<= 1) {
    const int lg = __ffs(sz) - 1;          // sz = 2^lg
    const int nel = 32 * sz;
    df tv[OPT];
    // T = L21 Y11: T_rc = L21_rc + sum_{k = c+1}^{sz-1} L21_rk Y11_kc
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int e = tid + DG_THREADS * q;
      if (e < nel) {
        const int blk = e >> (2 * lg), rem = e & (sz * sz - 1), r = rem & (sz - 1), c = rem >> lg;
        const int p = blk * 2 * sz, row = p + sz + r;
        df acc = dg_ld(t, row, p + c), acc2 = df_make(0.f, 0.f);
        int k = c + 1;
        for (; k + 1 < sz; k += 2) {
          acc = df_add_fast(acc, df_mul(dg_ld(t, row, p + k), dg_ld(t, p + k, p + c)));
          acc2 = df_add_fast(acc2, df_mul(dg_ld(t, row, p + k + 1), dg_ld(t, p + k + 1, p + c)));
        }
        if (k < sz) acc = df_add_fast(acc, df_mul(dg_ld(t, row, p + k), dg_ld(t, p + k, p + c)));
        tv[q] = df_add_fast(acc, acc2);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int e = tid + DG_THREADS * q;
      if (e < nel) {
        const int blk = e >> (2 * lg), rem = e & (sz * sz - 1), r = rem & (sz - 1), c = rem >> lg;
        const int p = blk * 2 * sz;
        dg_st(t, p + sz + r, p + c, tv[q]);
      }
    }
    __syncthreads();
    // Y21 = -Y22 T: -(T_rc + sum_{k < r} Y22_rk T_kc)
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int e = tid + DG_THREADS * q;
      if (e < nel) {
        const int blk = e >> (2 * lg), rem = e & (sz * sz - 1), r = rem >> lg, c = rem & (sz - 1);
        const int p = blk * 2 * sz, row = p + sz + r;
        df acc = dg_ld(t, row, p + c), acc2 = df_make(0.f, 0.f);
        int k = 0;
        for (; k + 1 < r; k += 2) {
          acc = df_add_fast(acc, df_mul(dg_ld(t, row, p + sz + k), dg_ld(t, p + sz + k, p + c)));
          acc2 = df_add_fast(acc2, df_mul(dg_ld(t, row, p + sz + k + 1), dg_ld(t, p + sz + k + 1, p + c)));
        }
        if (k < r) acc = df_add_fast(acc, df_mul(dg_ld(t, row, p + sz + k), dg_ld(t, p + sz + k, p + c)));
        tv[q] = df_neg(df_add_fast(acc, acc2));
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < OPT; ++q) {
      const int e = tid + DG_THREADS * q;
      if (e < nel) {
        const int blk = e >> (2 * lg), rem = e & (sz * sz - 1), r = rem >> lg, c = rem & (sz - 1);
        const int p = blk * 2 * sz;
        dg_st(t, p + sz + r, p + c, tv[q]);
      }
    }
    __syncthreads();
  }
  // ---- L^-1 = D^-1/2 Y: lane (row i, group g) holds columns 8g .. 8g + 7 of row i ----
  float2* linv = reinterpret_cast<float2*>(M.Linv) + (size_t)kt * TB * TB;
  static_assert(DG_THREADS >= TB * (TB / 8), "one lane per 8 values of the tile");
  if (tid < TB * (TB / 8)) {
    const int i = tid >> 3, g = tid & 7;
    const df ri = df_make(rdq[i].x, rdq[i].y);
    df x[8];
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = 8 * g + k;
      df v = df_make(0.f, 0.f);
      if (c < i) v = df_mul(dg_ld(t, i, c), ri);
      else if (c == i) v = ri;
      x[k] = v;
      mx = fmaxf(mx, fabsf(v.hi));
    }
    float4* dst = reinterpret_cast<float4*>(linv + i * TB + 8 * g);  // 64-byte aligned
#pragma unroll
    for (int k = 0; k < 8; k += 2) dst[k / 2] = make_float4(x[k].hi, x[k].lo, x[k + 1].hi, x[k + 1].lo);
    if (pb.planes) {
      // the row's exponent over its 8 lanes (aligned groups of 8 within the warp)
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      // |x| <= |hi| (1 + 2^-24): round the bound up so that |x| 2^-e <= 1 holds
      const int e = chunk_exponent(mx * (1.0f + 1.2e-7f));
      const int slot = blockIdx.x;
      if (g == 0) pb.exps[slot * pb.exp_slot_stride + i] = e;
      slice_and_store(x, e, pb.planes + (int64_t)slot * S * pb.plane_stride, pb.plane_stride, S,
                      (int64_t)i * pb.ld_k + 8 * g, true);
    }
  }
}

// Triangular solves with the double-float factor, one cooperative launch per solve:
// forward dst = L^-1 src (tiles in increasing order), backward dst = L^-T src (decreasing).
// Work items are (slot, tile) pairs in processing order, tile outermost; each block takes its
// items in increasing order (alternating direction across blocks for balance) and, for each
// tile its item depends on (every earlier tile of the slot), waits for that tile's ready
// flag, then subtracts the tile's contribution.  Items only wait on earlier items, so the
// launch makes progress when all blocks are resident (cooperative launch).  The dependency's
// factor tile is loaded into registers before its flag is awaited.  Every wait is bounded: on
// a timeout the block records the failure in *err and returns.  In place (src == dst) is
// allowed: an item reads its own src tile before writing its dst tile.
__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ df df_shfl_xor_sum(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df w = df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    v = df_add_fast(v, w);
  }
  return v;
}

__global__ void __launch_bounds__(256) k_trsv_df(TrsvArgs p) {
  __shared__ float2 vk[2][TB];
  __shared__ float2 part[4][TB];
  __shared__ float2 av[TB];
  __shared__ int abort_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = tid & 63, g = tid >> 6;  // backward layout: column c, 16-row group g
  const int P = p.T * p.nslots, G = gridDim.x;
  if (tid == 0) abort_sh = 0;
  __syncthreads();
  for (int round = 0;; ++round) {
    const int idx = (round & 1) ? (round + 1) * G - 1 - (int)blockIdx.x : round * G + (int)blockIdx.x;
    if (idx >= P) break;
    const int t = idx / p.nslots, sl = idx - t * p.nslots;
    const Slot& s = p.slots[sl];
    if (!s.active) continue;
    const DfRef M = df_ref(s, p.sel);
    const int Ts = M.n / TB;
    if (t >= Ts) continue;
    const int i = p.backward ? Ts - 1 - t : t;
    const double* src = vec_ref_df(s, p.src);
    double* dst = vec_ref_df(s, p.dst);
    int32_t* flg = p.flags + (size_t)sl * p.T;
    const float2* Li = reinterpret_cast<const float2*>(M.Linv) + (size_t)i * TB * TB;
    // the diagonal-tile inverse and this tile of src, read now: off the chain of ready flags
    float2 liv[16];
    if (!p.backward) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        liv[2 * r] = Li[(warp * 8 + r) * TB + lane];
        liv[2 * r + 1] = Li[(warp * 8 + r) * TB + lane + 32];
      }
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) liv[r] = Li[(g * 16 + r) * TB + c];
    }
    const double srcv = tid < TB ? src[(size_t)i * TB + tid] : 0.0;
    df acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = df_make(0.f, 0.f);
    for (int u = 0; u < t; ++u) {
      const int k = p.backward ? Ts - 1 - u : u;
      // this dependency's factor tile: L_ik (forward, rows of tile i) or L_ki (backward)
      float2 lv[16];
      if (!p.backward) {
        const float2* Lik = M.A + (size_t)i * TB * M.ld + (size_t)k * TB;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          lv[2 * r] = Lik[(size_t)(warp * 8 + r) * M.ld + lane];
          lv[2 * r + 1] = Lik[(size_t)(warp * 8 + r) * M.ld + lane + 32];
        }
      } else {
        const float2* Lki = M.A + (size_t)k * TB * M.ld + (size_t)i * TB;
#pragma unroll
        for (int r = 0; r < 16; ++r) lv[r] = Lki[(size_t)(g * 16 + r) * M.ld + c];
      }
      if (tid == 0) {
        bool ok = false;
        for (int64_t it = 0; it < p.spin_limit; ++it) {
          if (ld_acquire_gpu(flg + k) != 0) {
            ok = true;
            break;
          }
          __nanosleep(32);
        }
        if (!ok) {
          abort_sh = 1;
          atomicExch(p.err, 1);
        }
      }
      __syncthreads();
      if (abort_sh) return;
      float2* vb = vk[u & 1];
      if (tid < TB) {
        const df v = df_from_double(dst[(size_t)k * TB + tid]);
        vb[tid] = make_float2(v.hi, v.lo);
      }
      __syncthreads();
      if (!p.backward) {
        const df v0 = df_make(vb[lane].x, vb[lane].y), v1 = df_make(vb[lane + 32].x, vb[lane + 32].y);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          acc[r] = df_add_fast(acc[r], df_mul(df_make(lv[2 * r].x, lv[2 * r].y), v0));
          acc[r] = df_add_fast(acc[r], df_mul(df_make(lv[2 * r + 1].x, lv[2 * r + 1].y), v1));
        }
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r)
          acc[r & 7] = df_add_fast(acc[r & 7], df_mul(df_make(lv[r].x, lv[r].y), df_make(vb[g * 16 + r].x, vb[g * 16 + r].y)));
      }
    }
    // a = src_i - (sum of the dependencies)
    if (!p.backward) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const df v = df_shfl_xor_sum(acc[r]);
        if (lane == 0) part[0][warp * 8 + r] = make_float2(v.hi, v.lo);
      }
    } else {
      df v = acc[0];
#pragma unroll
      for (int r = 1; r < 8; ++r) v = df_add_fast(v, acc[r]);
      part[g][c] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    if (tid < TB) {
      df sum = df_make(part[0][tid].x, part[0][tid].y);
      if (p.backward)
        for (int q = 1; q < 4; ++q) sum = df_add_fast(sum, df_make(part[q][tid].x, part[q][tid].y));
      const df a = df_add_fast(df_from_double(srcv), df_neg(sum));
      av[tid] = make_float2(a.hi, a.lo);
    }
    __syncthreads();
    // diagonal tile: dst_i = Linv_i a (forward) or Linv_i^T a (backward)
    if (!p.backward) {
      const df a0 = df_make(av[lane].x, av[lane].y), a1 = df_make(av[lane + 32].x, av[lane + 32].y);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = warp * 8 + r;
        df v = df_mul(df_make(liv[2 * r].x, liv[2 * r].y), a0);
        v = df_add_fast(v, df_mul(df_make(liv[2 * r + 1].x, liv[2 * r + 1].y), a1));
        v = df_shfl_xor_sum(v);
        if (lane == 0) dst[(size_t)i * TB + row] = df_to_double(v);
      }
    } else {
      df v = df_make(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        v = df_add_fast(v, df_mul(df_make(liv[r].x, liv[r].y), df_make(av[g * 16 + r].x, av[g * 16 + r].y)));
      }
      part[g][c] = make_float2(v.hi, v.lo);
      __syncthreads();
      if (tid < TB) {
        df sum = df_make(part[0][tid].x, part[0][tid].y);
        for (int q = 1; q < 4; ++q) sum = df_add_fast(sum, df_make(part[q][tid].x, part[q][tid].y));
        dst[(size_t)i * TB + tid] = df_to_double(sum);
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release_gpu(flg + i, 1);
  }
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
// t1[j] = sum_{k >= j} Wk[j][k]^2 (df64 Y = W^T, upper): the column sums of squares of W read
// along rows of Y, one warp per row (coalesced)
__global__ void __launch_bounds__(256) k_rowsumsq_wk_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int lane = threadIdx.x & 31;
  const float2* Y = dfm(s.Wk);
  for (int j = (blockIdx.x * 256 + threadIdx.x) >> 5; j < s.n_pad; j += (gridDim.x * 256) >> 5) {
    df acc = df_make(0.f, 0.f);
    const float2* row = Y + (size_t)j * s.n_pad;
    for (int k = j + lane; k < s.n_pad; k += 32) {
      const df w = df_load(row + k);
      acc = df_fma(acc, w, w);
    }
    double r = df_to_double(acc);
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) s.t1[j] = r;
  }
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

void launch_cov_build_df(Slot* slots, int nslots, int max_td, cudaStream_t st) {
  if (max_td > 0) count_launch("k_cov_build_df"), k_cov_build_df<<<dim3(tri(max_td), nslots), 256, 0, st>>>(slots);
}
void launch_prior_entries_df(Slot* slots, int nslots, int64_t max_entries, cudaStream_t st) {
  if (max_entries > 0)
    count_launch("k_prior_entries_df"), k_prior_entries_df<<<dim3((unsigned)std::min<int64_t>(2048, (max_entries + 255) / 256), nslots), 256, 0, st>>>(slots);
}
void launch_add_pairs_df(Slot* slots, int nslots, int64_t max_pairs, cudaStream_t st) {
  if (max_pairs > 0)
    count_launch("k_add_pairs_df"), k_add_pairs_df<<<dim3(HEAVY_BLOCKS + (unsigned)std::min<int64_t>(4096, (max_pairs + 7) / 8), nslots), 256, 0, st>>>(slots);
}
void launch_qp_gemv_df(Slot* slots, int nslots, int which, int max_n, cudaStream_t st) {
  count_launch("k_vec_to_df"), k_vec_to_df<<<dim3(vgrid(max_n), nslots), 256, 0, st>>>(slots, which);
  (void)which;
  count_launch("k_qp_symv_part_df"), k_qp_symv_part_df<<<dim3(max_n / TB, nslots), 256, 0, st>>>(slots);
  count_launch("k_qp_symv_sum_df"), k_qp_symv_sum_df<<<dim3(std::min(1024, (max_n + 255) / 256), nslots), 256, 0, st>>>(slots);
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
void launch_potrf_diag_df(Slot* slots, int nslots, int sel, int kt, const OzOperand* slices, int S, cudaStream_t st) {
  OzOperand pb{};
  if (slices) pb = *slices;
  count_launch("k_potrf_diag_df"), k_potrf_diag_df<<<nslots, DG_THREADS, 0, st>>>(slots, sel, kt, pb, S);
}
int launch_trsv_df(const TrsvArgs& a, cudaStream_t st) {
  // resident blocks per SM and SM count, per device (the cooperative grid must fit at once)
  static std::atomic<int> geo[64][2];
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return INLA_E_CUDA;
  int per_sm = geo[dev][0].load(), sms = geo[dev][1].load();
  if (per_sm <= 0 || sms <= 0) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trsv_df, 256, 0) != cudaSuccess || per_sm <= 0 ||
        sms <= 0)
      return INLA_E_CUDA;
    geo[dev][0].store(per_sm);
    geo[dev][1].store(sms);
  }
  const int items = a.T * a.nslots;
  if (items <= 0) return INLA_OK;
  if (cudaMemsetAsync(a.flags, 0, sizeof(int32_t) * (size_t)items, st) != cudaSuccess) return INLA_E_CUDA;
  const int grid = std::min(items, per_sm * sms);
  TrsvArgs args = a;
  void* params[] = {&args};
  count_launch("k_trsv_df");
  if (cudaLaunchCooperativeKernel((const void*)k_trsv_df, dim3(grid), dim3(256), params, 0, st) != cudaSuccess)
    return note_launch_error("k_trsv_df cooperative launch");
  return INLA_OK;
}
void launch_logdet_df(Slot* slots, int nslots, int sel, int out_idx, cudaStream_t st) {
  count_launch("k_logdet_df"), k_logdet_df<<<nslots, 256, 0, st>>>(slots, sel, out_idx);
}
void launch_colsumsq_wk_df(Slot* slots, int nslots, int max_t, cudaStream_t st) {
  count_launch("k_colsumsq_wk_df"), k_colsumsq_wk_df<<<dim3(max_t, nslots), 256, 0, st>>>(slots);
}
void launch_rowsumsq_wk_df(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_rowsumsq_wk_df"), k_rowsumsq_wk_df<<<dim3(std::min(2048, (max_n + 7) / 8), nslots), 256, 0, st>>>(slots);
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

namespace inla {

// ---- Moore-Penrose / Woodbury route (Section 3.1, Eq. (woodeqn)) ----

// Q+ entry (i, j), internal indices: 0 across blocks; fixed 1 / prec and iid exp(-theta) on the
// diagonal; the dense block's covariance (double-float distance and exp, as the prior build);
// Kronecker blocks exp(-theta) times the product of the factors' pseudo-inverse entries (last
// factor fastest); 0 on the padding.
__device__ df pinv_prior_entry(const Slot& s, const ModelDev& md, int i, int j) {
  if (i >= s.n || j >= s.n) return df_make(0.f, 0.f);
  int bi = -1;
  for (int b = 0; b < md.nblk; ++b)
    if (i >= md.blk[b].off && i < md.blk[b].off + md.blk[b].size) bi = b;
  const BlockInfo& B = md.blk[bi];
  if (j < B.off || j >= B.off + B.size) return df_make(0.f, 0.f);
  const int li = i - B.off, lj = j - B.off;
  switch (B.kind) {
    case INLA_BLOCK_FIXED:
      return li == lj ? df_from_double(1.0 / B.prec) : df_make(0.f, 0.f);
    case INLA_BLOCK_IID:
      return li == lj ? df_from_double(exp(-s.theta[B.theta_idx])) : df_make(0.f, 0.f);
    case INLA_BLOCK_DENSE_EXP: {
      const double* P = md.points;
      df v = cov_entry_df(df_from_double(P[2 * li]), df_from_double(P[2 * li + 1]), df_from_double(P[2 * lj]),
                          df_from_double(P[2 * lj + 1]), df_from_double(exp(-s.theta[md.theta_rx])),
                          df_from_double(exp(-s.theta[md.theta_ry])), df_from_double(exp(2.0 * s.theta[md.theta_sigma])));
      if (li == lj) {
        double diag_add = md.nugget;
        if (md.theta_iid >= 0) diag_add += exp(-s.theta[md.theta_iid]);
        v = df_add(v, df_from_double(diag_add));
      }
      return v;
    }
    default: {  // Kronecker
      double prod = exp(-s.theta[B.theta_idx]);
      int ri = li, rj = lj;
      for (int f = B.nf - 1; f >= 0; --f) {
        const int fs = B.fsize[f];
        const int a = ri % fs, c = rj % fs;
        ri /= fs;
        rj /= fs;
        prod *= md.factor_pinv[B.pinv_off[f] + (int64_t)a * fs + c];
      }
      return df_from_double(prod);
    }
  }
}

__global__ void __launch_bounds__(256) k_woodbury_qplus_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  const int n = s.n_pad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    df_store(dfm(s.Wk) + e, pinv_prior_entry(s, md, i, j));
  }
}

// G row r = sqrt(w_r) sum_{e in row r of A} a_e Q+[col_e, :] (rows r >= m zero), into L
__global__ void __launch_bounds__(256) k_woodbury_g_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  const int n = s.n_pad;
  for (int r = blockIdx.x; r < s.aux_n; r += gridDim.x) {
    float2* G = dfm(s.L) + (size_t)r * n;
    if (r >= s.m) {
      for (int c = threadIdx.x; c < n; c += blockDim.x) G[c] = make_float2(0.f, 0.f);
      continue;
    }
    const double sw = sqrt(s.w[r]);
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      df acc = df_make(0.f, 0.f);
      for (int64_t e = md.A_rowptr[r]; e < md.A_rowptr[r + 1]; ++e)
        acc = df_add(acc, df_mul(df_from_double(sw * md.A_val[e]), df_load(dfm(s.Wk) + (size_t)md.A_col[e] * n + c)));
      df_store(G + c, acc);
    }
  }
}

// M = I + G B^T (lower triangle, aux_n x aux_n, identity on the padding), into Qp
__global__ void __launch_bounds__(256) k_woodbury_m_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const ModelDev& md = *s.md;
  const int n = s.n_pad, na = s.aux_n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)na * na; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / na), l = (int)(e % na);
    if (l > i) continue;
    df v = df_make(i == l ? 1.f : 0.f, 0.f);
    if (i < s.m && l < s.m) {
      const double sw = sqrt(s.w[l]);
      const float2* G = dfm(s.L) + (size_t)i * n;
      for (int64_t q = md.A_rowptr[l]; q < md.A_rowptr[l + 1]; ++q)
        v = df_add(v, df_mul(df_from_double(sw * md.A_val[q]), df_load(G + md.A_col[q])));
    }
    df_store(dfm(s.Qp) + (size_t)i * n + l, v);
  }
}

// t1[j] = Q+_jj - sum_{r < aux_n} Z[r][j]^2 with Z = L_M^-1 G held in L
__global__ void __launch_bounds__(256) k_woodbury_var_df(Slot* slots) {
  const Slot& s = slots[blockIdx.y];
  if (!s.active) return;
  const int jt = blockIdx.x;
  if (jt >= s.n_pad / TB) return;
  __shared__ double part[4][TB];
  const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
  df acc = df_make(0.f, 0.f);
  const float2* Z = dfm(s.L);
  for (int r = g; r < s.aux_n; r += 4) {
    const df z = df_load(Z + (size_t)r * s.n_pad + jt * TB + c);
    acc = df_fma(acc, z, z);
  }
  part[g][c] = df_to_double(acc);
  __syncthreads();
  if (threadIdx.x < TB) {
    const int j = jt * TB + threadIdx.x;
    const double t2 = ((part[0][threadIdx.x] + part[1][threadIdx.x]) + part[2][threadIdx.x]) + part[3][threadIdx.x];
    s.t1[j] = df_to_double(df_load(dfm(s.Wk) + (size_t)j * s.n_pad + j)) - t2;
  }
}

void launch_woodbury_terms_df(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_woodbury_qplus_df"), k_woodbury_qplus_df<<<dim3(4096, nslots), 256, 0, st>>>(slots);
  count_launch("k_woodbury_g_df"), k_woodbury_g_df<<<dim3(std::min(max_n, 8192), nslots), 256, 0, st>>>(slots);
  count_launch("k_woodbury_m_df"), k_woodbury_m_df<<<dim3(4096, nslots), 256, 0, st>>>(slots);
}
void launch_woodbury_var_df(Slot* slots, int nslots, int max_n, cudaStream_t st) {
  count_launch("k_woodbury_var_df"), k_woodbury_var_df<<<dim3(max_n / TB, nslots), 256, 0, st>>>(slots);
}

}  // namespace inla

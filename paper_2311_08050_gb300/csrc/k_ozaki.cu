// tcgen05 / TMA implementation of the Ozaki-split GEMM declared in ozaki.h.
//
// One CTA computes one 128 x 128 output tile with 10 warps:
//   warp 0      TMA producer: B slices of a 64-wide K step stay resident (2 stages),
//               A slices stream through a 2-stage ring;
//   warp 1      owns the TMEM allocation; lane 0 issues tcgen05.mma (M=128, N=128, K=16,
//               BF16 x BF16 -> FP32) into S accumulators, one per slice-order d = i + j;
//   warps 2..9  epilogue: after each 256-wide K chunk, read the accumulators (tcgen05.ld),
//               combine them exactly in double-float, scale by 2^(eA + eB - 14) and add the
//               chunk into C (double-float) in global memory.
// Every mbarrier wait is bounded by spin_limit; on a timeout the CTA records the failure in
// *err, stops issuing work, drains what it issued and returns.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstdio>
#include "df64.cuh"
#include "ozaki.h"

namespace inla {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int64_t limit) {
  const uint32_t a = smem_u32(bar);
  for (int64_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int A_BYTES = OZ_BM * OZ_BK * 2;  // 16 KB
constexpr int B_BYTES = OZ_BN * OZ_BK * 2;  // 16 KB

__device__ __forceinline__ void tile_coords(const OzArgs& p, int& tm, int& tn) {
  const int x = blockIdx.x;
  if (p.lower) {
    int t = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while (t * (t + 1) / 2 > x) --t;
    while ((t + 1) * (t + 2) / 2 <= x) ++t;
    tm = t;
    tn = x - t * (t + 1) / 2;
  } else {
    tm = x / p.tiles_n;
    tn = x % p.tiles_n;
  }
}

}  // namespace

template <int S>
__global__ void __launch_bounds__(320, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const OzArgs p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* Bbuf = smem;                       // 2 stages x S slices x 16 KB
  uint8_t* Abuf = smem + 2 * S * B_BYTES;     // 2 stages x 16 KB
  __shared__ __align__(8) uint64_t fullB[2], emptyB[2], fullA[2], emptyA[2], acc_full, acc_empty, done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh_;
  volatile int& abort_sh = abort_sh_;

  int tm, tn;
  tile_coords(p, tm, tn);
  if (tm >= p.tiles_m || tn >= p.tiles_n) return;
  const int m0 = tm * OZ_BM, n0 = tn * OZ_BN;
  const int slot = blockIdx.z;
  int k_lo = 0;
  if (p.k_mode == 1) k_lo = max(m0, n0);
  else if (p.k_mode == 2) k_lo = n0;
  else if (p.k_mode == 3) k_lo = m0;
  k_lo = (k_lo / OZ_BK) * OZ_BK;
  const int n_kc = k_lo < p.K ? (p.K - k_lo) / OZ_BK : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&fullB[s], 1);
      mbar_init(&emptyB[s], 1);
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 256);
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // slice-order groups d = i + j >= NACC-1 share the last accumulator (see ozaki.h)
  constexpr int NACC = S < OZ_NACC ? S : OZ_NACC;
  constexpr uint32_t TMEM_COLS = NACC * OZ_BN <= 256 ? 256 : 512;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  const int64_t lim = p.spin_limit;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0 && n_kc > 0) {
      int issued_b = 0, issued_a = 0;
      for (int kc = 0; kc < n_kc && !abort_sh; ++kc) {
        const int k = k_lo + kc * OZ_BK;
        const int b = kc & 1;
        if (kc >= 2 && !mbar_wait(&emptyB[b], ((kc >> 1) - 1) & 1, lim)) {
          abort_sh = 1;
          break;
        }
        mbar_expect_tx(&fullB[b], S * B_BYTES);
        for (int j = 0; j < S; ++j) tma_load_3d(Bbuf + (b * S + j) * B_BYTES, &tmB, k, n0, slot * S + j, &fullB[b]);
        issued_b = kc + 1;
        for (int i = 0; i < S; ++i) {
          const int a = kc * S + i, sa = a & 1;
          if (a >= 2 && !mbar_wait(&emptyA[sa], ((a >> 1) - 1) & 1, lim)) {
            abort_sh = 1;
            break;
          }
          mbar_expect_tx(&fullA[sa], A_BYTES);
          tma_load_3d(Abuf + sa * A_BYTES, &tmA, k, m0, slot * S + i, &fullA[sa]);
          issued_a = a + 1;
        }
      }
      if (abort_sh) {
        // drain the copies already issued before leaving (bounded)
        for (int kc = max(0, issued_b - 2); kc < issued_b; ++kc) mbar_wait(&fullB[kc & 1], (kc >> 1) & 1, lim);
        for (int a = max(0, issued_a - 2); a < issued_a; ++a) mbar_wait(&fullA[a & 1], (a >> 1) & 1, lim);
        atomicExch(p.err, 1);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0 && n_kc > 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) |
                             ((uint32_t)(OZ_BM >> 4) << 24);
      int chunk_no = 0;
      bool first_in_chunk = true;
      for (int kc = 0; kc < n_kc && !abort_sh; ++kc) {
        const int k = k_lo + kc * OZ_BK;
        if (first_in_chunk && chunk_no > 0) {
          if (!mbar_wait(&acc_empty, (chunk_no - 1) & 1, lim)) {
            abort_sh = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        const int b = kc & 1;
        if (!mbar_wait(&fullB[b], (kc >> 1) & 1, lim)) {
          abort_sh = 1;
          break;
        }
        bool ok = true;
        for (int i = 0; i < S; ++i) {
          const int a = kc * S + i, sa = a & 1;
          if (!mbar_wait(&fullA[sa], (a >> 1) & 1, lim)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a_addr = smem_u32(Abuf + sa * A_BYTES);
          for (int j = 0; j < S - i; ++j) {
            const uint32_t b_addr = smem_u32(Bbuf + (b * S + j) * B_BYTES);
            const int acc_idx = (i + j) < NACC ? (i + j) : NACC - 1;
            const uint32_t d_tmem = tmem + (uint32_t)(acc_idx * OZ_BN);
#pragma unroll
            for (int kk = 0; kk < OZ_BK / 16; ++kk) {
              // the first write of accumulator a in a chunk is the pair (0, a), kk = 0
              const uint32_t accum = (first_in_chunk && i == 0 && kk == 0 && j < NACC) ? 0u : 1u;
              mma_bf16(d_tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), idesc, accum);
            }
          }
          mma_commit(&emptyA[sa]);
        }
        if (!ok) {
          abort_sh = 1;
          break;
        }
        mma_commit(&emptyB[b]);
        first_in_chunk = false;
        const bool chunk_end = ((k + OZ_BK) % OZ_CHUNK == 0) || (kc == n_kc - 1);
        if (chunk_end) {
          mma_commit(&acc_full);
          ++chunk_no;
          first_in_chunk = true;
        }
      }
      // all issued MMAs complete before the TMEM is released
      mma_commit(&done_bar);
      mbar_wait(&done_bar, 0, lim);
      if (abort_sh) atomicExch(p.err, 1);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int row = q * 32 + lane;
    const int gr = m0 + row;
    const int32_t* eA = p.expA + slot * p.expA_slot_stride;
    const int32_t* eB = p.expB + slot * p.expB_slot_stride;
    float2* C = p.C + slot * p.C_slot_stride;
    if (n_kc == 0 && p.alpha == 0.f && gr < p.M)
      for (int c = h * 64; c < h * 64 + 64; ++c) {
        const int gc = n0 + c;
        if (gc < p.N && !(p.lower_elems && gc > gr)) df_store(C + (int64_t)gr * p.ldc + gc, df_make(0.f, 0.f));
      }
    int chunk_no = 0;
    for (int k = k_lo; k < p.K && !abort_sh;) {
      const int k_end = min(p.K, (k / OZ_CHUNK + 1) * OZ_CHUNK);
      const int chunk = k / OZ_CHUNK;
      if (!mbar_wait(&acc_full, chunk_no & 1, lim)) {
        abort_sh = 1;
        atomicExch(p.err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int ea = gr < p.M ? eA[(int64_t)chunk * p.expA_chunk_stride + gr] : 0;
      const bool first = (chunk_no == 0);
#pragma unroll 1
      for (int blk = 0; blk < 4; ++blk) {
        const int c0 = h * 64 + blk * 16;
        float D[NACC][16];
#pragma unroll
        for (int d = 0; d < NACC; ++d)
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(d * OZ_BN + c0), D[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (gr < p.M) {
          float2* crow = C + (int64_t)gr * p.ldc + n0 + c0;
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int gc = n0 + c0 + c;
            if (gc >= p.N || (p.lower_elems && gc > gr)) continue;
            // slices carry their 2^(-7i) scale, so the groups add directly
            df v = df_make(D[0][c], 0.f);
#pragma unroll
            for (int d = 1; d < NACC; ++d) v = df_add_f(v, D[d][c]);
            const int eb = eB[(int64_t)chunk * p.expB_chunk_stride + gc];
            v = df_scale(v, pow2f(ea + eb - 14));
            if (p.beta < 0.f) v = df_neg(v);
            if (first && p.alpha == 0.f) {
              df_store(crow + c, v);
            } else {
              df_store(crow + c, df_add(df_load(crow + c), v));
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(&acc_empty);
      ++chunk_no;
      k = k_end;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
  }
}

// ------------------------------------------------------------------------------------
// slicing: per (row, 256-chunk) power-of-two scale and S slices of 7 bits
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ df load_df(const T* p);
template <>
__device__ __forceinline__ df load_df<float2>(const float2* p) {
  return df_load(p);
}
template <>
__device__ __forceinline__ df load_df<double>(const double* p) {
  return df_from_double(*p);
}

// slice the 8 values of one lane (already loaded) given the warp-wide exponent; write S planes
__device__ __forceinline__ void slice_and_store(const df (&x)[8], int e, uint16_t* planes, int64_t plane_stride,
                                                int S, int64_t base, bool valid) {
  const float sc = pow2f(7 - e);  // t * 2^7 with t = x 2^-e, |t| <= 1
  df r[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = df_scale(x[i], sc);
  for (int s = 0; s < S; ++s) {
    uint16_t out[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = rintf(r[i].hi + r[i].lo);
      // remainder (exact): (hi - v) + lo, then scaled by 2^7 for the next slice
      df rem = df_add_f(df_make(r[i].hi - v, 0.f), r[i].lo);
      r[i] = df_scale(rem, 128.f);
      // slice s is stored as v_s 2^(-7s) (exact: a power-of-two scaling of an integer <= 2^8)
      const __nv_bfloat16 bv = __float2bfloat16_rn(v * pow2f(-7 * s));
      out[i] = *reinterpret_cast<const uint16_t*>(&bv);
    }
    if (valid) {
      uint4 pk;
      pk.x = (uint32_t)out[0] | ((uint32_t)out[1] << 16);
      pk.y = (uint32_t)out[2] | ((uint32_t)out[3] << 16);
      pk.z = (uint32_t)out[4] | ((uint32_t)out[5] << 16);
      pk.w = (uint32_t)out[6] | ((uint32_t)out[7] << 16);
      *reinterpret_cast<uint4*>(planes + s * plane_stride + base) = pk;
    }
  }
}

__device__ __forceinline__ int chunk_exponent(float m) {
  // smallest e with m <= 2^e  (m > 0); e = 0 for an all-zero chunk
  if (!(m > 0.f)) return 0;
  int e;
  const float f = frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  (void)f;
  return e;
}

// untransposed source: one warp per (operand row, chunk); lane covers k = lane*8 .. +7
template <typename T>
__global__ void __launch_bounds__(256) k_slice_rows(const T* src, int64_t src_slot_stride, int ld, int row0, int col0,
                                                    int R, int K, OzOperand dst, int S) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nchunks = (K + OZ_CHUNK - 1) / OZ_CHUNK;
  if (warp >= R * nchunks) return;
  const int r = warp / nchunks, ch = warp % nchunks;
  const int slot = blockIdx.y;
  const T* s = src + slot * src_slot_stride + (int64_t)(row0 + r) * ld + col0;
  const int k0 = ch * OZ_CHUNK + lane * 8;
  const bool valid = k0 < K;
  df x[8];
  float mx = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    x[i] = valid ? load_df<T>(s + k0 + i) : df_make(0.f, 0.f);
    mx = fmaxf(mx, fabsf(x[i].hi));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // |x| <= |hi| (1 + 2^-24): round the bound up so that |x| 2^-e <= 1 holds
  const int e = chunk_exponent(mx * (1.0f + 1.2e-7f));
  if (lane == 0) dst.exps[slot * dst.exp_slot_stride + (int64_t)ch * dst.exp_chunk_stride + r] = e;
  uint16_t* planes = dst.planes + (int64_t)slot * S * dst.plane_stride;
  slice_and_store(x, e, planes, dst.plane_stride, S, (int64_t)r * dst.ld_k + k0, valid);
}

// transposed source: a block handles 16 operand rows x one 256-chunk through shared memory
template <typename T>
__global__ void __launch_bounds__(256) k_slice_cols(const T* src, int64_t src_slot_stride, int ld, int row0, int col0,
                                                    int R, int K, OzOperand dst, int S) {
  __shared__ float2 tile[OZ_CHUNK][17];
  const int r0 = blockIdx.x * 16, ch = blockIdx.z, slot = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* s = src + slot * src_slot_stride;
  for (int kk = warp * 2 + (lane >> 4); kk < OZ_CHUNK; kk += 16) {
    const int k = ch * OZ_CHUNK + kk, r = r0 + (lane & 15);
    df v = df_make(0.f, 0.f);
    if (k < K && r < R) v = load_df<T>(s + (int64_t)(row0 + k) * ld + col0 + r);
    tile[kk][lane & 15] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  for (int rr = warp * 2; rr < warp * 2 + 2; ++rr) {
    const int r = r0 + rr;
    if (r >= R) break;
    const int k0 = ch * OZ_CHUNK + lane * 8;
    const bool valid = k0 < K;
    df x[8];
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 t = tile[lane * 8 + i][rr];
      x[i] = df_make(t.x, t.y);
      mx = fmaxf(mx, fabsf(t.x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = chunk_exponent(mx * (1.0f + 1.2e-7f));
    if (lane == 0) dst.exps[slot * dst.exp_slot_stride + (int64_t)ch * dst.exp_chunk_stride + r] = e;
    uint16_t* planes = dst.planes + (int64_t)slot * S * dst.plane_stride;
    slice_and_store(x, e, planes, dst.plane_stride, S, (int64_t)r * dst.ld_k + k0, valid);
  }
}

// ------------------------------------------------------------------------------------
// host
// ------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int get_encode() {
  if (g_encode) return INLA_OK;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return INLA_E_CUDA;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return INLA_OK;
}

int oz_make_map(CUtensorMap* map, const OzOperand& op, int nplanes) {
  INLA_TRY(get_encode());
  if ((op.ld_k % OZ_BK) != 0 || (op.K % OZ_BK) != 0 || ((uintptr_t)op.planes & 15) != 0) return INLA_E_BADARG;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)op.ld_k * 2, (cuuint64_t)op.plane_stride * 2};
  cuuint32_t box[3] = {OZ_BK, OZ_BM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op.planes, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? INLA_OK : INLA_E_BADARG;
}

template <int S>
static int launch_oz(const CUtensorMap& ma, const CUtensorMap& mb, const OzArgs& a, int nslots, cudaStream_t st) {
  const int smem = 2 * S * B_BYTES + 2 * A_BYTES + 1024;
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_ozaki_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return INLA_E_CUDA;
    init = true;
  }
  const int tiles = a.lower ? a.tiles_m * (a.tiles_m + 1) / 2 : a.tiles_m * a.tiles_n;
  if (tiles <= 0) return INLA_OK;
  count_launch("k_ozaki_gemm<S>"), k_ozaki_gemm<S><<<dim3(tiles, 1, nslots), 320, smem, st>>>(ma, mb, a);
  if (debug_sync_enabled()) {
    char site[200];
    snprintf(site, sizeof(site), "ozaki S=%d M=%d N=%d K=%d kmode=%d lower=%d slots=%d", S, a.M, a.N, a.K, a.k_mode,
             a.lower, nslots);
    return debug_check(st, site);
  }
  return INLA_OK;
}

// ---- optional launch statistics (CUDA events around every GEMM launch) ----
struct OzStats {
  bool on = false;
  int64_t launches = 0;
  double alg_flops = 0.0;     // 2 * (needed output elements) * K, per the tile k-ranges
  double tensor_flops = 0.0;  // alg_flops * S (S + 1) / 2 BF16 passes
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};
static OzStats g_stats;

static double oz_alg_flops(const OzArgs& a, int nslots) {
  double f = 0.0;
  const int tiles = a.lower ? a.tiles_m * (a.tiles_m + 1) / 2 : a.tiles_m * a.tiles_n;
  for (int x = 0; x < tiles; ++x) {
    int tm, tn;
    if (a.lower) {
      int t = 0;
      while ((t + 1) * (t + 2) / 2 <= x) ++t;
      tm = t;
      tn = x - t * (t + 1) / 2;
    } else {
      tm = x / a.tiles_n;
      tn = x % a.tiles_n;
    }
    const int m0 = tm * OZ_BM, n0 = tn * OZ_BN;
    int k_lo = a.k_mode == 1 ? std::max(m0, n0) : a.k_mode == 2 ? n0 : a.k_mode == 3 ? m0 : 0;
    k_lo = (k_lo / OZ_BK) * OZ_BK;
    const double rows = std::min(OZ_BM, a.M - m0), cols = std::min(OZ_BN, a.N - n0);
    double elems = rows * cols;
    if (a.lower && tm == tn) elems = rows * (rows + 1) / 2;
    if (k_lo < a.K) f += 2.0 * elems * (a.K - k_lo);
  }
  return f * nslots;
}

int oz_gemm(const OzOperand& A, const OzOperand& B, const OzArgs& args_in, int nslots, cudaStream_t st) {
  OzArgs a = args_in;
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return INLA_OK;
  if (a.K % OZ_BK) return INLA_E_BADARG;
  if (a.lower && a.M != a.N) return INLA_E_BADARG;
  a.expA = A.exps;
  a.expB = B.exps;
  a.expA_chunk_stride = A.exp_chunk_stride;
  a.expB_chunk_stride = B.exp_chunk_stride;
  a.expA_slot_stride = A.exp_slot_stride;
  a.expB_slot_stride = B.exp_slot_stride;
  a.tiles_m = (a.M + OZ_BM - 1) / OZ_BM;
  a.tiles_n = (a.N + OZ_BN - 1) / OZ_BN;
  CUtensorMap ma, mb;
  INLA_TRY(oz_make_map(&ma, A, a.S * nslots));
  INLA_TRY(oz_make_map(&mb, B, a.S * nslots));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g_stats.on) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  int rc;
  switch (a.S) {
    case 2: rc = launch_oz<2>(ma, mb, a, nslots, st); break;
    case 3: rc = launch_oz<3>(ma, mb, a, nslots, st); break;
    case 4: rc = launch_oz<4>(ma, mb, a, nslots, st); break;
    case 5: rc = launch_oz<5>(ma, mb, a, nslots, st); break;
    default: rc = INLA_E_BADARG;
  }
  if (g_stats.on) {
    cudaEventRecord(e1, st);
    g_stats.ev.push_back({e0, e1});
    g_stats.launches += 1;
    const double f = oz_alg_flops(a, nslots);
    g_stats.alg_flops += f;
    g_stats.tensor_flops += f * a.S * (a.S + 1) / 2;
  }
  return rc;
}

}  // namespace inla

// test hooks: launch statistics of the Ozaki GEMM
extern "C" void inla_test_stats_enable(int on) {
  using namespace inla;
  g_stats.on = on != 0;
}
extern "C" int inla_test_stats_read(double* out) {
  using namespace inla;
  if (!out) return INLA_E_BADARG;
  double ms = 0.0;
  for (auto& p : g_stats.ev) {
    float t = 0.f;
    if (cudaEventSynchronize(p.second) == cudaSuccess && cudaEventElapsedTime(&t, p.first, p.second) == cudaSuccess)
      ms += t;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  g_stats.ev.clear();
  out[0] = (double)g_stats.launches;
  out[1] = g_stats.alg_flops;
  out[2] = g_stats.tensor_flops;
  out[3] = ms;
  g_stats.launches = 0;
  g_stats.alg_flops = g_stats.tensor_flops = 0.0;
  return INLA_OK;
}

namespace inla {

template <typename T>
static void slice_impl(const T* src, int64_t sss, int ld, int row0, int col0, int R, int K, bool transposed,
                       const OzOperand& dst, int S, int nslots, cudaStream_t st) {
  if (R <= 0 || K <= 0) return;
  const int nchunks = (K + OZ_CHUNK - 1) / OZ_CHUNK;
  if (!transposed) {
    const int64_t warps = (int64_t)R * nchunks;
    count_launch("k_slice_rows<T>"), k_slice_rows<T><<<dim3((unsigned)((warps + 7) / 8), nslots), 256, 0, st>>>(src, sss, ld, row0, col0, R, K, dst, S);
  } else {
    count_launch("k_slice_cols<T>"), k_slice_cols<T><<<dim3((R + 15) / 16, nslots, nchunks), 256, 0, st>>>(src, sss, ld, row0, col0, R, K, dst, S);
  }
  if (debug_sync_enabled()) {
    char site[200];
    snprintf(site, sizeof(site), "slice R=%d K=%d t=%d row0=%d col0=%d ld=%d", R, K, (int)transposed, row0, col0, ld);
    debug_check(st, site);
  }
}

void oz_slice_df(const float2* src, int64_t sss, int ld, int row0, int col0, int R, int K, bool transposed,
                 const OzOperand& dst, int S, int nslots, cudaStream_t st) {
  slice_impl<float2>(src, sss, ld, row0, col0, R, K, transposed, dst, S, nslots, st);
}
void oz_slice_f64(const double* src, int64_t sss, int ld, int row0, int col0, int R, int K, bool transposed,
                  const OzOperand& dst, int S, int nslots, cudaStream_t st) {
  slice_impl<double>(src, sss, ld, row0, col0, R, K, transposed, dst, S, nslots, st);
}

}  // namespace inla

// tcgen05 / TMA implementation of the Ozaki-split GEMM declared in ozaki.h.
//
// Persistent kernel: one CTA per SM walks 128 x BN output tiles (slot-major; BN = 128, or 64
// for narrow or short-K products) with 12 warps (warpgroup 0 gives registers up to warpgroups
// 1-2 with setmaxnreg):
//   warp 0      TMA producer: a stage is the S slices of A and of B for 32 values of k
//               (two 3-D boxes, 64-byte swizzle); 2..6 stages depending on S and BN;
//   warp 1      owns the TMEM allocation; lane 0 issues tcgen05.mma (M=128, N=BN, K=16,
//               BF16 x BF16 -> FP32) into min(S, 4) accumulators, slice-order d = i + j
//               (groups d >= 3 share the last one); with BN = 64 two accumulator sets
//               alternate by chunk, so the MMAs run on while the epilogue reads the other set;
//   warps 4..11 epilogue: after each 512-wide K chunk, read the accumulators (tcgen05.ld),
//               combine them in double-float, scale by 2^(eA + eB - 14) and add the chunk
//               into a register tile, then release the TMEM so that the next chunk (or tile)
//               runs on the tensor cores while the finished tile is added into C (double-float,
//               global) with coalesced row segments.
// Every mbarrier wait is bounded by spin_limit; on a timeout the CTA records the failure in
// *err, stops issuing work, drains what it issued and returns.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cstdio>
#include "df64.cuh"
#include "ozaki.h"
#include "oz_slice.cuh"

namespace inla {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
// Bounded wait for a phase; try_wait with a short (32 ns) suspend-time hint: the hand-offs
// between the MMA issuer and the epilogue then resume promptly.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int64_t limit) {
  const uint32_t a = smem_u32(bar);
  for (int64_t it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 32; selp.u32 %0, 1, 0, p; }"
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
// Pipeline geometry: a stage holds the S slices of both operands for OZ_KS values of k;
// the stage count fills the shared memory left after the epilogue staging buffers.  The TMEM
// holds NBUF sets of NACC accumulators of BN columns: with two sets (the narrow tile) the MMAs
// of the next chunk run while the epilogue reads the previous one.
template <int S, int BN>
struct OzCfg {
  static constexpr int A_SLICE = OZ_BM * OZ_KS * 2;
  static constexpr int B_SLICE = BN * OZ_KS * 2;
  static constexpr int STAGE_BYTES = S * (A_SLICE + B_SLICE);
  static constexpr int NST_FIT = (OZ_SMEM_BUDGET - 1024 - OZ_STAGING_BYTES - OZ_COLSC_BYTES) / STAGE_BYTES;
  static constexpr int NST = NST_FIT > 6 ? 6 : NST_FIT;
  static constexpr int SMEM = 1024 + NST * STAGE_BYTES + OZ_STAGING_BYTES + OZ_COLSC_BYTES;  // 1024: alignment
  static constexpr int NACC = S < OZ_NACC ? S : OZ_NACC;
  static constexpr int ACC_COLS = NACC * BN;                 // one accumulator set
  static constexpr int NBUF = 2 * ACC_COLS <= 512 ? 2 : 1;
  static constexpr int USED = NBUF * ACC_COLS;
  static constexpr uint32_t TMEM_COLS = USED <= 32 ? 32 : USED <= 64 ? 64 : USED <= 128 ? 128 : USED <= 256 ? 256 : 512;
  static constexpr int CPT = BN / 2;                         // columns per epilogue thread
  static_assert(BN == OZ_BN || BN == OZ_BN_NARROW, "tile width");
  static_assert(STAGE_BYTES % 1024 == 0, "stages keep the 64-byte swizzle atoms aligned");
};

// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)4 << 61);
}
// Double-float sum without the second error-free step on the low words: its error, ~2^-44 of
// |a| + |b|, stays far below the slice truncation of the products it accumulates.
__device__ __forceinline__ float2 df2_add_fast(float2 a, float2 b) {
  float s, t;
  two_sum(a.x, b.x, s, t);
  t = __fadd_rn(t, __fadd_rn(a.y, b.y));
  fast_two_sum(s, t, s, t);
  return make_float2(s, t);
}
// Packed FP32 pairs (f32x2: two lanes of arithmetic per instruction on the FP32 pipe).
__device__ __forceinline__ uint64_t f2pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 f2unpack(uint64_t v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return make_float2(a, b);
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Load 16 consecutive TMEM columns of NA accumulators (columns col + a * stride), wait for the
// loads, and return them as packed column pairs d[a][m] = (column 2m, column 2m + 1).  One asm
// statement: the registers are read only after tcgen05.wait::ld.
template <int NA>
__device__ __forceinline__ void tmem_ld16_pairs(uint32_t taddr, uint32_t stride, uint64_t (&d)[NA][8]);
template <>
__device__ __forceinline__ void tmem_ld16_pairs<2>(uint32_t t, uint32_t stride, uint64_t (&d)[2][8]) {
  asm volatile(
      "{\n.reg .b32 a<32>;\n"
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a0,a1,a2,a3,a4,a5,a6,a7,a8,a9,a10,a11,a12,a13,a14,a15}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a16,a17,a18,a19,a20,a21,a22,a23,a24,a25,a26,a27,a28,a29,a30,a31}, [%17];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "mov.b64 %0, {a0,a1}; mov.b64 %1, {a2,a3}; mov.b64 %2, {a4,a5}; mov.b64 %3, {a6,a7}; mov.b64 %4, {a8,a9}; mov.b64 %5, {a10,a11}; mov.b64 %6, {a12,a13}; mov.b64 %7, {a14,a15}; mov.b64 %8, {a16,a17}; mov.b64 %9, {a18,a19}; mov.b64 %10, {a20,a21}; mov.b64 %11, {a22,a23}; mov.b64 %12, {a24,a25}; mov.b64 %13, {a26,a27}; mov.b64 %14, {a28,a29}; mov.b64 %15, {a30,a31};\n}"
      : "=l"(d[0][0]), "=l"(d[0][1]), "=l"(d[0][2]), "=l"(d[0][3]), "=l"(d[0][4]), "=l"(d[0][5]), "=l"(d[0][6]), "=l"(d[0][7]), "=l"(d[1][0]), "=l"(d[1][1]), "=l"(d[1][2]), "=l"(d[1][3]), "=l"(d[1][4]), "=l"(d[1][5]), "=l"(d[1][6]), "=l"(d[1][7])
      : "r"(t), "r"(t + 1 * stride)
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld16_pairs<3>(uint32_t t, uint32_t stride, uint64_t (&d)[3][8]) {
  asm volatile(
      "{\n.reg .b32 a<48>;\n"
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a0,a1,a2,a3,a4,a5,a6,a7,a8,a9,a10,a11,a12,a13,a14,a15}, [%24];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a16,a17,a18,a19,a20,a21,a22,a23,a24,a25,a26,a27,a28,a29,a30,a31}, [%25];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a32,a33,a34,a35,a36,a37,a38,a39,a40,a41,a42,a43,a44,a45,a46,a47}, [%26];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "mov.b64 %0, {a0,a1}; mov.b64 %1, {a2,a3}; mov.b64 %2, {a4,a5}; mov.b64 %3, {a6,a7}; mov.b64 %4, {a8,a9}; mov.b64 %5, {a10,a11}; mov.b64 %6, {a12,a13}; mov.b64 %7, {a14,a15}; mov.b64 %8, {a16,a17}; mov.b64 %9, {a18,a19}; mov.b64 %10, {a20,a21}; mov.b64 %11, {a22,a23}; mov.b64 %12, {a24,a25}; mov.b64 %13, {a26,a27}; mov.b64 %14, {a28,a29}; mov.b64 %15, {a30,a31}; mov.b64 %16, {a32,a33}; mov.b64 %17, {a34,a35}; mov.b64 %18, {a36,a37}; mov.b64 %19, {a38,a39}; mov.b64 %20, {a40,a41}; mov.b64 %21, {a42,a43}; mov.b64 %22, {a44,a45}; mov.b64 %23, {a46,a47};\n}"
      : "=l"(d[0][0]), "=l"(d[0][1]), "=l"(d[0][2]), "=l"(d[0][3]), "=l"(d[0][4]), "=l"(d[0][5]), "=l"(d[0][6]), "=l"(d[0][7]), "=l"(d[1][0]), "=l"(d[1][1]), "=l"(d[1][2]), "=l"(d[1][3]), "=l"(d[1][4]), "=l"(d[1][5]), "=l"(d[1][6]), "=l"(d[1][7]), "=l"(d[2][0]), "=l"(d[2][1]), "=l"(d[2][2]), "=l"(d[2][3]), "=l"(d[2][4]), "=l"(d[2][5]), "=l"(d[2][6]), "=l"(d[2][7])
      : "r"(t), "r"(t + 1 * stride), "r"(t + 2 * stride)
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_ld16_pairs<4>(uint32_t t, uint32_t stride, uint64_t (&d)[4][8]) {
  asm volatile(
      "{\n.reg .b32 a<64>;\n"
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a0,a1,a2,a3,a4,a5,a6,a7,a8,a9,a10,a11,a12,a13,a14,a15}, [%32];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a16,a17,a18,a19,a20,a21,a22,a23,a24,a25,a26,a27,a28,a29,a30,a31}, [%33];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a32,a33,a34,a35,a36,a37,a38,a39,a40,a41,a42,a43,a44,a45,a46,a47}, [%34];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {a48,a49,a50,a51,a52,a53,a54,a55,a56,a57,a58,a59,a60,a61,a62,a63}, [%35];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "mov.b64 %0, {a0,a1}; mov.b64 %1, {a2,a3}; mov.b64 %2, {a4,a5}; mov.b64 %3, {a6,a7}; mov.b64 %4, {a8,a9}; mov.b64 %5, {a10,a11}; mov.b64 %6, {a12,a13}; mov.b64 %7, {a14,a15}; mov.b64 %8, {a16,a17}; mov.b64 %9, {a18,a19}; mov.b64 %10, {a20,a21}; mov.b64 %11, {a22,a23}; mov.b64 %12, {a24,a25}; mov.b64 %13, {a26,a27}; mov.b64 %14, {a28,a29}; mov.b64 %15, {a30,a31}; mov.b64 %16, {a32,a33}; mov.b64 %17, {a34,a35}; mov.b64 %18, {a36,a37}; mov.b64 %19, {a38,a39}; mov.b64 %20, {a40,a41}; mov.b64 %21, {a42,a43}; mov.b64 %22, {a44,a45}; mov.b64 %23, {a46,a47}; mov.b64 %24, {a48,a49}; mov.b64 %25, {a50,a51}; mov.b64 %26, {a52,a53}; mov.b64 %27, {a54,a55}; mov.b64 %28, {a56,a57}; mov.b64 %29, {a58,a59}; mov.b64 %30, {a60,a61}; mov.b64 %31, {a62,a63};\n}"
      : "=l"(d[0][0]), "=l"(d[0][1]), "=l"(d[0][2]), "=l"(d[0][3]), "=l"(d[0][4]), "=l"(d[0][5]), "=l"(d[0][6]), "=l"(d[0][7]), "=l"(d[1][0]), "=l"(d[1][1]), "=l"(d[1][2]), "=l"(d[1][3]), "=l"(d[1][4]), "=l"(d[1][5]), "=l"(d[1][6]), "=l"(d[1][7]), "=l"(d[2][0]), "=l"(d[2][1]), "=l"(d[2][2]), "=l"(d[2][3]), "=l"(d[2][4]), "=l"(d[2][5]), "=l"(d[2][6]), "=l"(d[2][7]), "=l"(d[3][0]), "=l"(d[3][1]), "=l"(d[3][2]), "=l"(d[3][3]), "=l"(d[3][4]), "=l"(d[3][5]), "=l"(d[3][6]), "=l"(d[3][7])
      : "r"(t), "r"(t + 1 * stride), "r"(t + 2 * stride), "r"(t + 3 * stride)
      : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
// Tile t of the launch (slots outermost): its slot, origin and K range in 32-wide stages.
// Lower launches enumerate row-major the tiles that reach the diagonal or below: with R = 128 / BN
// tiles per 128 columns, tile row u holds R (u + 1) of them and starts at R u (u + 1) / 2.
struct OzTile {
  int slot, m0, n0, k_lo, n_st;
};
template <int BN>
__device__ __forceinline__ OzTile oz_tile(const OzArgs& p, int t) {
  constexpr int R = OZ_BM / BN;
  OzTile r;
  r.slot = t / p.tiles_per_slot;
  const int x = t - r.slot * p.tiles_per_slot;
  int tm, tn;
  if (p.lower) {
    const int xr = x / R;  // R u (u + 1) / 2 <= x  <=>  u (u + 1) / 2 <= floor(x / R)
    int u = (int)((sqrtf(8.0f * (float)xr + 1.0f) - 1.0f) * 0.5f);  // corrected below (no FP64 on this GPU's hot path)
    while (u * (u + 1) / 2 > xr) --u;
    while ((u + 1) * (u + 2) / 2 <= xr) ++u;
    tm = u;
    tn = x - R * (u * (u + 1) / 2);
  } else {
    tm = x / p.tiles_n;
    tn = x - tm * p.tiles_n;
  }
  r.m0 = tm * OZ_BM;
  r.n0 = tn * BN;
  int k_lo = 0;
  if (p.k_mode == 1) k_lo = max(r.m0, r.n0);
  else if (p.k_mode == 2) k_lo = r.n0;
  else if (p.k_mode == 3) k_lo = r.m0;
  k_lo = (k_lo / OZ_BK) * OZ_BK;
  r.k_lo = k_lo;
  r.n_st = k_lo < p.K ? (p.K - k_lo) / OZ_KS : 0;
  return r;
}

}  // namespace

template <int S, int BN>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const OzArgs p) {
  using Cfg = OzCfg<S, BN>;
  constexpr int NST = Cfg::NST, NACC = Cfg::NACC, NBUF = Cfg::NBUF, CPT = Cfg::CPT;
  constexpr uint32_t STAGE_BYTES = Cfg::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float2* staging = reinterpret_cast<float2*>(smem + NST * STAGE_BYTES);
  float* colsc_all = reinterpret_cast<float*>(smem + NST * STAGE_BYTES + OZ_STAGING_BYTES);
  __shared__ __align__(8) uint64_t full[NST], empty[NST], acc_full[NBUF], acc_empty[NBUF], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh_;
  volatile int& abort_sh = abort_sh_;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], OZ_EPI_WARPS * 32);
    }
    mbar_init(&done_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "n"(Cfg::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  const int64_t lim = p.spin_limit;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(OZ_ROLE_REGS));
    // one stage = the S slices of A and of B for 32 values of k (two 3-D boxes)
    if (lane == 0) {
      int g = 0;  // stages issued by this CTA
      for (int t = blockIdx.x; t < p.tiles_total && !abort_sh; t += gridDim.x) {
        const OzTile ti = oz_tile<BN>(p, t);
        for (int s = 0; s < ti.n_st; ++s, ++g) {
          const int st = g % NST, u = g / NST;
          if (u > 0 && !mbar_wait(&empty[st], (u - 1) & 1, lim)) {
            abort_sh = 1;
            break;
          }
          uint8_t* dst = smem + st * STAGE_BYTES;
          const int k = ti.k_lo + s * OZ_KS;
          mbar_expect_tx(&full[st], STAGE_BYTES);
          tma_load_3d(dst, &tmA, k, ti.m0, ti.slot * S, &full[st]);
          tma_load_3d(dst + S * Cfg::A_SLICE, &tmB, k, ti.n0, ti.slot * S, &full[st]);
        }
      }
      if (abort_sh) {
        // drain the copies already issued before leaving (bounded)
        for (int h = max(0, g - NST); h < g; ++h) mbar_wait(&full[h % NST], (h / NST) & 1, lim);
        atomicExch(p.err, 1);
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(OZ_ROLE_REGS));
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(OZ_BM >> 4) << 24);
      int g = 0, c = 0;  // stages consumed, chunks completed
      bool ok = true;
      for (int t = blockIdx.x; t < p.tiles_total && ok && !abort_sh; t += gridDim.x) {
        const OzTile ti = oz_tile<BN>(p, t);
        bool first_in_chunk = true;
        for (int s = 0; s < ti.n_st; ++s, ++g) {
          const int k = ti.k_lo + s * OZ_KS;
          if (first_in_chunk && c >= NBUF) {
            // the epilogue has read the chunk that last used this accumulator set
            if (!mbar_wait(&acc_empty[c % NBUF], (c / NBUF - 1) & 1, lim)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
          }
          const int st = g % NST, u = g / NST;
          if (!mbar_wait(&full[st], u & 1, lim)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t base = smem_u32(smem + st * STAGE_BYTES);
          const uint32_t set = tmem + (uint32_t)((c % NBUF) * Cfg::ACC_COLS);
#pragma unroll
          for (int i = 0; i < S; ++i) {
#pragma unroll
            for (int j = 0; j < S - i; ++j) {
              const int acc_idx = (i + j) < NACC ? (i + j) : NACC - 1;
              const uint32_t d_tmem = set + (uint32_t)(acc_idx * BN);
              const uint32_t a_addr = base + i * Cfg::A_SLICE, b_addr = base + S * Cfg::A_SLICE + j * Cfg::B_SLICE;
#pragma unroll
              for (int kk = 0; kk < OZ_KS / 16; ++kk) {
                // the first write of accumulator a in a chunk is the pair (0, a), kk = 0
                const uint32_t accum = (first_in_chunk && i == 0 && kk == 0 && j < NACC) ? 0u : 1u;
                mma_bf16(d_tmem, sw64_desc(a_addr + kk * 32), sw64_desc(b_addr + kk * 32), idesc, accum);
              }
            }
          }
          mma_commit(&empty[st]);
          first_in_chunk = false;
          if (((k + OZ_KS) % OZ_CHUNK) == 0 || s == ti.n_st - 1) {
            mma_commit(&acc_full[c % NBUF]);
            ++c;
            first_in_chunk = true;
          }
        }
      }
      // all issued MMAs complete before the TMEM is released
      mma_commit(&done_bar);
      mbar_wait(&done_bar, 0, lim);
      if (!ok || abort_sh) {
        abort_sh = 1;
        atomicExch(p.err, 1);
      }
    }
  } else if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(OZ_ROLE_REGS));
  } else {
    // ------------------------------ epilogue ------------------------------
    // Thread = one row of the tile and CPT = BN / 2 columns (warp half h).  Per chunk: drain the
    // group accumulators into a double-float register tile and release the TMEM, so that the
    // next chunk's (or tile's) MMAs start at once.  After the tile's last chunk, add the tile into C
    // through a per-warp staging buffer: each store instruction writes 64-byte row segments.
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(OZ_EPI_REGS));
    const int ew = warp - 4;
    const int q = warp & 3, h = ew >> 2;
    const int row = q * 32 + lane;
    float2* stg = staging + ew * (32 * OZ_STG_LD);
    float* colsc = colsc_all + ew * CPT;
    const uint32_t t_lane = tmem + ((uint32_t)(q * 32) << 16);
    const bool neg = p.beta < 0.f;
    const bool accumulate = p.alpha != 0.f;
    constexpr float kRound = 12582912.f;  // 1.5 * 2^23
    int c = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.tiles_total && ok; t += gridDim.x) {
      const OzTile ti = oz_tile<BN>(p, t);
      const int gr = ti.m0 + row;
      const int col0 = ti.n0 + h * CPT;
      float2* C = p.C + ti.slot * p.C_slot_stride;
      float2 acc[CPT];  // the register tile: (hi, lo) of the thread's CPT columns
      if (ti.n_st == 0) {
        if (p.alpha != 0.f) continue;
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[j] = make_float2(0.f, 0.f);
      } else {
        if (p.alpha != 0.f && gr < p.M)
          for (int j = 0; j < CPT; j += 16)
            if (col0 + j < p.N) prefetch_l2(C + (int64_t)gr * p.ldc + col0 + j);
        const int32_t* eA = p.expA + ti.slot * p.expA_slot_stride;
        const int32_t* eB = p.expB + ti.slot * p.expB_slot_stride;
        for (int k = ti.k_lo; k < p.K;) {
          const int chunk = k / OZ_CHUNK;
          const int k_end = min(p.K, (chunk + 1) * OZ_CHUNK);
          // scales of this chunk: +-2^(eA - 14) for the thread's row (sign of beta); 2^eB for the
          // warp's CPT columns in a per-warp shared array (read as broadcast pairs)
          float rs = pow2f(gr < p.M ? eA[(int64_t)chunk * p.expA_chunk_stride + gr] - 14 : 0);
          if (neg) rs = -rs;
          const uint64_t rs2 = f2pack(rs, rs);
          const int64_t eb_base = (int64_t)chunk * p.expB_chunk_stride;
          __syncwarp();
#pragma unroll
          for (int jj = lane; jj < CPT; jj += 32) colsc[jj] = pow2f(col0 + jj < p.N ? eB[eb_base + col0 + jj] : 0);
          __syncwarp();
          const int buf = c % NBUF;
          bool got = mbar_wait(&acc_full[buf], (c / NBUF) & 1, lim);
          got = __all_sync(0xffffffffu, got);
          if (!got) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const bool first = (k == ti.k_lo);
#pragma unroll
          for (int blk2 = 0; blk2 < CPT / 16; ++blk2) {
            uint64_t D[NACC][8];
            tmem_ld16_pairs<NACC>(t_lane + (uint32_t)(buf * Cfg::ACC_COLS + h * CPT + blk2 * 16), (uint32_t)BN, D);
            // Group 0 holds integers of magnitude <= 2^23, groups 1 and 2 multiples of 2^-7 and
            // 2^-14 of magnitude <= 2^16 and 640: the integer parts add exactly in FP32 (below
            // 2^24), the fractions exactly into the low word (multiples of 2^-14 below 1), and the
            // rounded tail group (d >= 3) costs ~2^-24 of a value below 2^3.  Integer parts by the
            // 1.5 * 2^23 shift (exact for |x| < 2^22); two columns per f32x2 instruction.
            const uint64_t KR2 = f2pack(kRound, kRound);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              const int j2 = blk2 * 8 + m;  // column pair (2 j2, 2 j2 + 1) of the thread's CPT
              const uint64_t d1 = D[1][m];
              const uint64_t t1 = sub2(add2(d1, KR2), KR2);
              uint64_t sv = add2(D[0][m], t1);
              uint64_t ev = sub2(d1, t1);
              if (NACC >= 3) {
                const uint64_t d2 = D[2][m];
                const uint64_t t2 = sub2(add2(d2, KR2), KR2);
                sv = add2(sv, t2);
                ev = add2(ev, sub2(d2, t2));
              }
              if (NACC >= 4) ev = add2(ev, D[NACC - 1][m]);
              const uint64_t sc = mul2(rs2, *reinterpret_cast<const uint64_t*>(colsc + 2 * j2));
              const uint64_t hi = mul2(sv, sc), lo = mul2(ev, sc);
              const float2 hh = f2unpack(hi), ll = f2unpack(lo);
              if (first) {
                acc[2 * j2] = make_float2(hh.x, ll.x);
                acc[2 * j2 + 1] = make_float2(hh.y, ll.y);
              } else {
                acc[2 * j2] = df2_add_fast(acc[2 * j2], make_float2(hh.x, ll.x));
                acc[2 * j2 + 1] = df2_add_fast(acc[2 * j2 + 1], make_float2(hh.y, ll.y));
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(&acc_empty[buf]);
          ++c;
          k = k_end;
        }
        if (!ok) break;
      }
      const int cc = lane & 7;
      int grow[8];
      float2* crow[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        grow[i] = ti.m0 + q * 32 + i * 4 + (lane >> 3);
        crow[i] = C + (int64_t)grow[i] * p.ldc;
      }
#pragma unroll
      for (int blk = 0; blk < CPT / 8; ++blk) {
        __syncwarp();
#pragma unroll
        for (int u = 0; u < 8; ++u) stg[lane * OZ_STG_LD + u] = acc[blk * 8 + u];
        __syncwarp();
        const int gcol = col0 + blk * 8 + cc;
        bool valid[8];
        float2 old[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          valid[i] = grow[i] < p.M && gcol < p.N && !(p.lower_elems && gcol > grow[i]);
          old[i] = make_float2(0.f, 0.f);
          if (accumulate && valid[i]) old[i] = __ldcg(crow[i] + gcol);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float2 v = stg[(i * 4 + (lane >> 3)) * OZ_STG_LD + cc];
          if (accumulate) {
            v = df2_add_fast(old[i], v);
          } else {
            float hi, lo;
            two_sum(v.x, v.y, hi, lo);
            v = make_float2(hi, lo);
          }
          if (valid[i]) crow[i][gcol] = v;
        }
      }
    }
    if (!ok) {
      abort_sh = 1;
      atomicExch(p.err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(Cfg::TMEM_COLS));
  }
}

// ------------------------------------------------------------------------------------
// slicing: per (row, 512-chunk) power-of-two scale and S slices of 7 bits
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

// Untransposed source: a group of G lanes (8, 16 or 32) per (operand row, chunk); lane g of the
// group covers the NSEG segments k = chunk * OZ_CHUNK + 8 (G seg + g) .. +7 (G * 8 * NSEG is
// the chunk width, or K when K is shorter).
template <typename T, int G, int NSEG>
__global__ void __launch_bounds__(256) k_slice_rows(const T* src, int64_t src_slot_stride, int ld, int row0, int col0,
                                                    int R, int K, OzOperand dst, int S) {
  const int lane = threadIdx.x & 31, gl = lane & (G - 1);
  const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int nchunks = (K + OZ_CHUNK - 1) / OZ_CHUNK;
  const bool active = grp < (int64_t)R * nchunks;
  const int r = active ? (int)(grp / nchunks) : 0, ch = active ? (int)(grp % nchunks) : 0;
  const int slot = blockIdx.y;
  const T* s = src + slot * src_slot_stride + (int64_t)(row0 + r) * ld + col0;
  df x[NSEG][8];
  int k0[NSEG];
  bool valid[NSEG];
  float mx = 0.f;
#pragma unroll
  for (int g = 0; g < NSEG; ++g) {
    k0[g] = ch * OZ_CHUNK + (g * G + gl) * 8;
    valid[g] = active && k0[g] < K;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      x[g][i] = valid[g] ? load_df<T>(s + k0[g] + i) : df_make(0.f, 0.f);
      mx = fmaxf(mx, fabsf(x[g][i].hi));
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // |x| <= |hi| (1 + 2^-24): round the bound up so that |x| 2^-e <= 1 holds
  const int e = chunk_exponent(mx * (1.0f + 1.2e-7f));
  if (active && gl == 0) dst.exps[slot * dst.exp_slot_stride + (int64_t)ch * dst.exp_chunk_stride + r] = e;
  uint16_t* planes = dst.planes + (int64_t)slot * S * dst.plane_stride;
#pragma unroll
  for (int g = 0; g < NSEG; ++g)
    slice_and_store(x[g], e, planes, dst.plane_stride, S, (int64_t)r * dst.ld_k + k0[g], valid[g]);
}

// Transposed source: a block handles ROWS operand rows (16, or 8 for chunks longer than 256)
// x one chunk through shared memory (dynamic: ROWS x LDT double-float cells, LDT = min(K,
// OZ_CHUNK) + 1, odd so that the rows of a transposing write hit distinct banks; 8 rows keep a
// 512-wide chunk's tile at 33 KB, so that six blocks share an SM).  The tile is stored
// row-major by operand row with the k index swizzled (k ^ ((k >> 3) & 15)), so that both the
// transposing writes (ROWS rows, one k) and the per-lane reads (one row, k = 8 lane + i + 256 g)
// avoid bank conflicts.  Only the chunk's part below K is loaded.
template <typename T, int ROWS>
__global__ void __launch_bounds__(256) k_slice_cols(const T* src, int64_t src_slot_stride, int ld, int row0, int col0,
                                                    int R, int K, OzOperand dst, int S, int LDT) {
  constexpr int NSEG = OZ_CHUNK / 256;
  constexpr int KPW = 32 / ROWS;          // k rows per warp per load instruction
  constexpr int RPW = ROWS / 8;           // operand rows per warp in the slicing phase
  extern __shared__ float2 tile[];
  const int r0 = blockIdx.x * ROWS, ch = blockIdx.z, slot = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kk_end = min(OZ_CHUNK, K - ch * OZ_CHUNK);
  const T* s = src + slot * src_slot_stride;
  const int r = r0 + (lane % ROWS);
  // eight loads in flight per thread before their shared-memory stores
  for (int kb = warp * KPW + lane / ROWS; kb < kk_end; kb += 8 * KPW * 8) {
    df v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int kk = kb + 8 * KPW * u;
      v[u] = df_make(0.f, 0.f);
      if (kk < kk_end && r < R) v[u] = load_df<T>(s + (int64_t)(row0 + ch * OZ_CHUNK + kk) * ld + col0 + r);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int kk = kb + 8 * KPW * u;
      if (kk < kk_end) tile[(lane % ROWS) * LDT + (kk ^ ((kk >> 3) & 15))] = make_float2(v[u].hi, v[u].lo);
    }
  }
  __syncthreads();
  for (int rr = warp * RPW; rr < warp * RPW + RPW; ++rr) {
    const int rw = r0 + rr;
    if (rw >= R) break;
    df x[NSEG][8];
    int k0[NSEG];
    bool valid[NSEG];
    float mx = 0.f;
#pragma unroll
    for (int g = 0; g < NSEG; ++g) {
      const int kb = g * 256 + lane * 8;
      k0[g] = ch * OZ_CHUNK + kb;
      valid[g] = kb < kk_end;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int kk = kb + i;
        float2 t = make_float2(0.f, 0.f);
        if (valid[g]) t = tile[rr * LDT + (kk ^ ((kk >> 3) & 15))];
        x[g][i] = df_make(t.x, t.y);
        mx = fmaxf(mx, fabsf(t.x));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = chunk_exponent(mx * (1.0f + 1.2e-7f));
    if (lane == 0) dst.exps[slot * dst.exp_slot_stride + (int64_t)ch * dst.exp_chunk_stride + rw] = e;
    uint16_t* planes = dst.planes + (int64_t)slot * S * dst.plane_stride;
#pragma unroll
    for (int g = 0; g < NSEG; ++g)
      slice_and_store(x[g], e, planes, dst.plane_stride, S, (int64_t)rw * dst.ld_k + k0[g], valid[g]);
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

int oz_make_map(CUtensorMap* map, const OzOperand& op, int nplanes, int S, int box_rows) {
  INLA_TRY(get_encode());
  if ((op.ld_k % OZ_BK) != 0 || (op.K % OZ_BK) != 0 || ((uintptr_t)op.planes & 15) != 0 || S < 1 ||
      S > OZ_MAX_S || nplanes % S || (box_rows != OZ_BM && box_rows != OZ_BN_NARROW))
    return INLA_E_BADARG;
  cuuint64_t dims[3] = {(cuuint64_t)op.K, (cuuint64_t)op.rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)op.ld_k * 2, (cuuint64_t)op.plane_stride * 2};
  cuuint32_t box[3] = {OZ_KS, (cuuint32_t)box_rows, (cuuint32_t)S};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, op.planes, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? INLA_OK : INLA_E_BADARG;
}

static int num_sms() {
  static std::atomic<int> cached[64];
  const int dev = current_device();
  if (dev < 0 || dev >= 64) return 148;
  int v = cached[dev].load();
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cached[dev].store(v);
  }
  return v;
}

int oz_num_sms() { return num_sms(); }

// Persistent launch: one CTA per SM (shared memory allows no second), tiles round-robin.
template <int S, int BN>
static int launch_oz(const CUtensorMap& ma, const CUtensorMap& mb, const OzArgs& a, int nslots, cudaStream_t st) {
  constexpr int smem = OzCfg<S, BN>::SMEM;
  static DeviceFlags attr_set;  // the shared-memory limit is a per-device attribute
  const int dev = current_device();
  if (!attr_set.test(dev)) {
    if (cudaFuncSetAttribute(k_ozaki_gemm<S, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return INLA_E_CUDA;
    attr_set.set(dev);
  }
  if (a.tiles_total <= 0) return INLA_OK;
  const int sms = num_sms();
  const int grid = std::min(a.tiles_total, a.max_ctas > 0 ? std::min(a.max_ctas, sms) : sms);
  count_launch("k_ozaki_gemm<S>"), k_ozaki_gemm<S, BN><<<grid, OZ_THREADS, smem, st>>>(ma, mb, a);
  if (cudaPeekAtLastError() != cudaSuccess) return note_launch_error("k_ozaki_gemm launch");
  if (debug_sync_enabled()) {
    char site[200];
    snprintf(site, sizeof(site), "ozaki S=%d BN=%d M=%d N=%d K=%d kmode=%d lower=%d slots=%d", S, BN, a.M, a.N, a.K,
             a.k_mode, a.lower, nslots);
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
  double alg_bytes = 0.0;     // compulsory DRAM bytes: slice planes once + C written (and read)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};
static OzStats g_stats;
bool oz_stats_active() { return g_stats.on; }

// Algorithmic flops of a launch: 2 K' per needed output element, K' the tile's k range
// (lower launches need the elements on or below the diagonal).  Also its compulsory DRAM
// bytes: every needed element of the double-float C written once (8 bytes) and, when
// accumulating, read once; the S BF16 slice planes of both operands read once (2 S (M + N) K
// bytes; the same operand for A and B is counted once).
static double oz_alg_flops(const OzArgs& a, int nslots, int bn, bool same_operand, double* bytes) {
  double f = 0.0, elems_all = 0.0;
  for (int tm = 0; tm < a.tiles_m; ++tm) {
    const int tn_end = a.lower ? std::min(a.tiles_n, (tm + 1) * (OZ_BM / bn)) : a.tiles_n;
    for (int tn = 0; tn < tn_end; ++tn) {
      const int m0 = tm * OZ_BM, n0 = tn * bn;
      int k_lo = a.k_mode == 1 ? std::max(m0, n0) : a.k_mode == 2 ? n0 : a.k_mode == 3 ? m0 : 0;
      k_lo = (k_lo / OZ_BK) * OZ_BK;
      if (k_lo >= a.K) continue;
      const int rows = std::min(OZ_BM, a.M - m0), cols = std::min(bn, a.N - n0);
      double elems = 0.0;
      if (a.lower)
        for (int r = m0; r < m0 + rows; ++r) elems += std::max(0, std::min(r, n0 + cols - 1) - n0 + 1);
      else
        elems = (double)rows * cols;
      f += 2.0 * elems * (a.K - k_lo);
      elems_all += elems;
    }
  }
  if (bytes) {
    const double c_bytes = elems_all * (a.alpha != 0.f ? 16.0 : 8.0);
    const double op_bytes = 2.0 * a.S * (double)a.K * (same_operand ? a.M : (double)a.M + a.N);
    *bytes = (c_bytes + op_bytes) * nslots;
  }
  return f * nslots;
}

// Tile width.  The narrow (double-buffered) tile serves products of at most 64 columns, where
// the wide tile would spend half its tensor and epilogue work on padding, and products with
// K <= 64, where a tile is one short chunk and the wide tile's MMAs wait for every drain
// (measured on 147456-row panels of the blocked Cholesky: 1.8x at N = 64, 1.2-1.5x at
// N = 192..448).  Longer K stays on the wide tile: the narrow one loads A twice per 128
// columns and measured ~30% slower there.  A test hook may force one width.
static int g_force_bn = 0;

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
  const int bn = g_force_bn ? g_force_bn : (a.N <= OZ_BN_NARROW || a.K <= OZ_BK ? OZ_BN_NARROW : OZ_BN);
  a.tiles_m = (a.M + OZ_BM - 1) / OZ_BM;
  a.tiles_n = (a.N + bn - 1) / bn;
  a.tiles_per_slot = a.lower ? (OZ_BM / bn) * (a.tiles_m * (a.tiles_m + 1) / 2) : a.tiles_m * a.tiles_n;
  a.tiles_total = a.tiles_per_slot * nslots;
  CUtensorMap ma, mb;
  INLA_TRY(oz_make_map(&ma, A, a.S * nslots, a.S, OZ_BM));
  INLA_TRY(oz_make_map(&mb, B, a.S * nslots, a.S, bn));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g_stats.on) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  int rc;
  const bool narrow = bn == OZ_BN_NARROW;
  switch (a.S) {
    case 2: rc = narrow ? launch_oz<2, OZ_BN_NARROW>(ma, mb, a, nslots, st) : launch_oz<2, OZ_BN>(ma, mb, a, nslots, st); break;
    case 3: rc = narrow ? launch_oz<3, OZ_BN_NARROW>(ma, mb, a, nslots, st) : launch_oz<3, OZ_BN>(ma, mb, a, nslots, st); break;
    case 4: rc = narrow ? launch_oz<4, OZ_BN_NARROW>(ma, mb, a, nslots, st) : launch_oz<4, OZ_BN>(ma, mb, a, nslots, st); break;
    case 5: rc = narrow ? launch_oz<5, OZ_BN_NARROW>(ma, mb, a, nslots, st) : launch_oz<5, OZ_BN>(ma, mb, a, nslots, st); break;
    case 6: rc = narrow ? launch_oz<6, OZ_BN_NARROW>(ma, mb, a, nslots, st) : launch_oz<6, OZ_BN>(ma, mb, a, nslots, st); break;
    default: rc = INLA_E_BADARG;
  }
  if (g_stats.on) {
    cudaEventRecord(e1, st);
    g_stats.ev.push_back({e0, e1});
    g_stats.launches += 1;
    double by = 0.0;
    const double f = oz_alg_flops(a, nslots, bn, A.planes == B.planes, &by);
    g_stats.alg_flops += f;
    g_stats.alg_bytes += by;
    g_stats.tensor_flops += f * a.S * (a.S + 1) / 2;
  }
  return rc;
}

}  // namespace inla

// test hooks: launch statistics of the Ozaki GEMM; forced tile width (0: by shape, 64, 128)
extern "C" int inla_test_gemm_tile_width(int bn) {
  using namespace inla;
  if (bn != 0 && bn != OZ_BN && bn != OZ_BN_NARROW) return INLA_E_BADARG;
  g_force_bn = bn;
  return INLA_OK;
}
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
  out[4] = g_stats.alg_bytes;
  g_stats.launches = 0;
  g_stats.alg_flops = g_stats.tensor_flops = g_stats.alg_bytes = 0.0;
  return INLA_OK;
}

namespace inla {

template <typename T>
static void slice_impl(const T* src, int64_t sss, int ld, int row0, int col0, int R, int K, bool transposed,
                       const OzOperand& dst, int S, int nslots, cudaStream_t st) {
  if (R <= 0 || K <= 0) return;
  const int nchunks = (K + OZ_CHUNK - 1) / OZ_CHUNK;
  if (!transposed) {
    // lanes per (row, chunk): K / 8 up to 32 lanes (K is a multiple of 64), then 2 segments
    static_assert(OZ_CHUNK == 512, "segment choice below");
    const int G = K <= 64 ? 8 : K <= 128 ? 16 : 32;
    const int64_t threads = (int64_t)R * nchunks * G;
    const dim3 grid((unsigned)((threads + 255) / 256), nslots);
    count_launch("k_slice_rows<T>");
    if (G == 8) k_slice_rows<T, 8, 1><<<grid, 256, 0, st>>>(src, sss, ld, row0, col0, R, K, dst, S);
    else if (G == 16) k_slice_rows<T, 16, 1><<<grid, 256, 0, st>>>(src, sss, ld, row0, col0, R, K, dst, S);
    else if (K <= 256) k_slice_rows<T, 32, 1><<<grid, 256, 0, st>>>(src, sss, ld, row0, col0, R, K, dst, S);
    else k_slice_rows<T, 32, 2><<<grid, 256, 0, st>>>(src, sss, ld, row0, col0, R, K, dst, S);
  } else {
    // 16 rows per block up to 256-wide chunks (33 KB), 8 rows for the 512-wide ones (33 KB)
    const int ldt = std::min(K, OZ_CHUNK) + 1;
    if (ldt <= 257) {
      const size_t smem = (size_t)16 * ldt * sizeof(float2);
      count_launch("k_slice_cols<T>"), k_slice_cols<T, 16><<<dim3((R + 15) / 16, nslots, nchunks), 256, smem, st>>>(src, sss, ld, row0, col0, R, K, dst, S, ldt);
    } else {
      const size_t smem = (size_t)8 * ldt * sizeof(float2);
      count_launch("k_slice_cols<T>"), k_slice_cols<T, 8><<<dim3((R + 7) / 8, nslots, nchunks), 256, smem, st>>>(src, sss, ld, row0, col0, R, K, dst, S, ldt);
    }
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

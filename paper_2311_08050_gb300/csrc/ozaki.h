// Ozaki-split GEMM on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA).
//
// Each operand row is scaled by a power of two per 512-wide K chunk and cut into S slices of
// 7 bits (integers held exactly in BF16: |v_0| <= 128, |v_i| <= 64 for i >= 1, each later
// digit being a rounded remainder of magnitude <= 1/2 scaled by 2^7):
// x = 2^e sum_i v_i 2^{-7(i+1)} + r, |r| <= 2^{e-7S-1}.  A chunk's product is then
// sum_{i+j<S} 2^{-7(i+j+2)} (V_i W_j^T), and the FP32 tensor-core sums of the groups
// d = i + j <= 2 are exact over 512 terms: per term |v_0 w_0| <= 2^14,
// |v_0 w_1| + |v_1 w_0| <= 2^14 and |v_0 w_2| + |v_1 w_1| + |v_2 w_0| <= 5 2^12, so every
// partial sum is an integer (in units of its group) below 5 2^21 < 2^24.
// The epilogue combines them in double-float (FP32 pairs) and updates a double-float C.
// (Splitting of floating-point operands into error-free slices: Ozaki, Ogita, Oishi, Rump,
// Numer. Algorithms 59 (2012).)
#pragma once
#include <cuda.h>
#include <cstdint>
#include "internal.h"

namespace inla {

constexpr int OZ_BM = 128;      // tile rows (tcgen05 M)
constexpr int OZ_BN = 128;      // tile columns (tcgen05 N) of the wide tile
constexpr int OZ_BN_NARROW = 64;  // tile columns of the narrow tile (N <= 64 or K <= 64): its
                                  // accumulator sets fit twice in the TMEM (double buffering)
constexpr int OZ_BK = 64;       // K granularity of operands and of the k ranges
constexpr int OZ_KS = 32;       // K per pipeline stage (64-byte swizzled rows of BF16)
constexpr int OZ_CHUNK = 512;   // K per exact accumulation chunk (one exponent per row)
constexpr int OZ_MAX_S = 6;
constexpr int OZ_SLICE_BYTES = OZ_BM * OZ_KS * 2;   // one slice of A (128 rows) for one stage
constexpr int OZ_EPI_WARPS = 8;                     // epilogue warps (two per TMEM lane quarter)
constexpr int OZ_THREADS = 384;                     // warpgroup 0: TMA + MMA; 1-2: epilogue
// Register split: launched at 168 per thread (384 x 168 <= 64K; three warps share each
// sub-partition's 16K registers), then warpgroup 0 drops to OZ_ROLE_REGS and the epilogue
// warpgroups rise to OZ_EPI_REGS, which holds a finished 128 x 128 double-float tile in
// registers (64 columns per thread).  4 * 56 + 8 * 224 = 12 * 168.
constexpr int OZ_ROLE_REGS = 56;
constexpr int OZ_EPI_REGS = 224;
static_assert(4 * OZ_ROLE_REGS + 8 * OZ_EPI_REGS <= 12 * 168, "register split exceeds the launch allocation");
constexpr int OZ_STG_LD = 9;                        // epilogue staging row stride (float2)
constexpr int OZ_STAGING_BYTES = OZ_EPI_WARPS * 32 * OZ_STG_LD * 8;
constexpr int OZ_COLSC_BYTES = OZ_EPI_WARPS * 64 * 4;  // per-warp column scale factors
constexpr int OZ_SMEM_BUDGET = 232448 - 512;        // opt-in maximum less the static barriers
// TMEM accumulators per tile (4 x 128 columns = all 512).  Slice i is stored pre-scaled by
// 2^(-7i), so a product V_i W_j^T arrives with its weight 2^(-7(i+j)): groups d = 0, 1, 2 are
// exact in FP32 (integers times 2^(-7d) with < 24 significant bits over a 512-wide chunk) and
// every group d >= 3 is summed into the fourth accumulator, where FP32 rounding costs
// ~2^-24 of a 2^-21-scaled quantity, i.e. ~2^-45 of the product: negligible against the
// 2^-7S slice truncation.
constexpr int OZ_NACC = 4;

// A sliced operand: planes [plane = slot * S + slice][row][k] (BF16, row stride ld_k
// elements, plane stride plane_stride elements) and exponents [slot][chunk][row] (int32,
// chunk stride exp_chunk_stride, slot stride exp_slot_stride).
struct OzOperand {
  uint16_t* planes;
  int32_t* exps;
  int rows;               // valid rows (TMA zero-fills beyond)
  int K;                  // valid K (multiple of 64)
  int ld_k;               // row stride in elements (multiple of 64)
  int64_t plane_stride;   // elements between planes
  int exp_chunk_stride;   // = rows capacity
  int64_t exp_slot_stride;
};

// C (double-float, row-major) = alpha C + beta (A B^T) over [0, M) x [0, N), per slot.
struct OzArgs {
  int32_t* expA;
  int32_t* expB;
  int expA_chunk_stride, expB_chunk_stride;
  int64_t expA_slot_stride, expB_slot_stride;
  float2* C;
  int64_t C_slot_stride;
  int ldc;
  int M, N, K;
  int k_mode;        // 0: k in [0, K); 1: k >= max(m0, n0); 2: k >= n0; 3: k >= m0
  int tiles_m, tiles_n;
  int tiles_per_slot, tiles_total;   // set by oz_gemm
  int lower;         // only tiles with tile_m >= tile_n
  int lower_elems;   // only elements with row >= col
  float alpha, beta;
  int S;
  int64_t spin_limit;
  int32_t* err;      // device flag: set to nonzero on a timed-out wait
  int max_ctas;      // persistent grid cap (0: one CTA per SM), leaving SMs to concurrent kernels
};

// Host: encode a 3-D tensor map over an operand's planes (box OZ_KS x box_rows x S: all S
// slices of box_rows rows for one pipeline stage; box_rows = 128, or 64 for a narrow B).
int oz_make_map(CUtensorMap* map, const OzOperand& op, int nplanes, int S, int box_rows);
// Host: C = alpha C + beta A B^T for `nslots` slots (grid.z), S slices.
int oz_gemm(const OzOperand& A, const OzOperand& B, const OzArgs& args, int nslots, cudaStream_t st);
// Host: the SM count of the current device (the persistent grid)
int oz_num_sms();

// Slicing kernels (host launchers).  Source element (r, k) of operand row r is
//   rows:  src[(row0 + r) * ld + col0 + k]      cols: src[(row0 + k) * ld + col0 + r]
// for r < R, k < K.  `src_slot_stride` in elements.  Source type: df64 (float2) or FP64.
void oz_slice_df(const float2* src, int64_t src_slot_stride, int ld, int row0, int col0, int R, int K,
                 bool transposed, const OzOperand& dst, int S, int nslots, cudaStream_t st);
void oz_slice_f64(const double* src, int64_t src_slot_stride, int ld, int row0, int col0, int R, int K,
                  bool transposed, const OzOperand& dst, int S, int nslots, cudaStream_t st);

}  // namespace inla

/*
 * inla_testing.h -- test hooks of libinla (not part of the evaluation API).
 *
 * These entry points expose single building blocks of the mixed-precision path so that
 * tests can check them in isolation against plain FP64 arithmetic.  They allocate their own
 * device buffers, copy host arrays in and out, and return INLA_OK or a negative INLA_E_*.
 */
#ifndef INLA_TESTING_H
#define INLA_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* C = alpha C + beta op(A) op(B)^T with the Ozaki-split tensor-core GEMM (S BF16 slices per
 * operand, exact FP32 accumulation per 512-wide K chunk, double-float C).
 * A: row-major M x K (trans_a = 0) or K x M (trans_a = 1); B: N x K or K x N; C: M x N,
 * all host FP64 arrays.  K must be a multiple of 64.  lower = 1 computes only the lower
 * triangle (M == N); k_mode restricts K per 128 x 128 tile (0: all; 1: k >= max(row0, col0);
 * 2: k >= col0; 3: k >= row0).  alpha must be 0 or 1, beta +1 or -1. */
int inla_test_ozaki_gemm(const double *A, const double *B, double *C, int32_t M, int32_t N, int32_t K,
                         int32_t slices, int32_t trans_a, int32_t trans_b, int32_t lower, int32_t k_mode,
                         double alpha, double beta);

/* With the environment variable INLA_DEBUG_SYNC=1 the library synchronizes after each
 * checked step; this returns the first step at which a CUDA error became visible ("" if
 * none).  Static storage, owned by the library. */
const char *inla_test_debug_site(void);

/* Launch statistics of the Ozaki-split tensor-core GEMM (the dominant kernel of the mixed
 * path).  While enabled, CUDA events are recorded around every launch on its stream.
 * inla_test_stats_read fills out[0..4] = {launches, algorithmic flops (2 * needed output
 * elements * K), tensor-pipe flops (algorithmic * S(S+1)/2 BF16 passes), summed launch
 * time in ms, compulsory DRAM bytes (slice planes of both operands read once, the needed
 * double-float C elements written once and, when accumulating, read once)}, synchronizing on
 * the recorded events, and resets the counters. */
void inla_test_stats_enable(int on);
int inla_test_stats_read(double *out);

/* Tile width of the Ozaki-split GEMM: 0 (default) chooses by shape -- the double-buffered
 * 128 x 64 tile for products of at most 64 columns or with K <= 64, 128 x 128 otherwise; 64 or 128 forces
 * one for every later launch.  INLA_E_BADARG for any other value. */
int inla_test_gemm_tile_width(int bn);

/* Number of CUDA kernels the library launched since the previous call (then reset). */
int64_t inla_test_launch_count(void);

/* Per-kernel profile: while enabled, a CUDA event is recorded on the evaluation stream
 * before every launch.  inla_test_profile_read writes "name launches total_ms" lines
 * (largest total first) into buf and resets; it returns the bytes written. */
void inla_test_profile_enable(int on);
int inla_test_profile_read(char *buf, int len);
/* Phase profile of the same recording: "name count total_ms" lines in order of first appearance
 * for the phases of a batch (prior, Newton of the leading points, their factor at the mode,
 * Newton of the points that start from another point's mode, their factor, and the
 * log-determinants, variances and log pi~); resets and returns the bytes written. */
int inla_test_phase_read(char *buf, int len);
/* The n-point Gauss-Hermite rule (weight e^{-x^2}, n <= 32) the variational Bayes correction
 * uses: nodes ascending, weights summing to sqrt(pi).  Host computation, no GPU needed. */
int inla_test_gauss_hermite(int32_t n, double *nodes, double *weights);
/* As inla_test_profile_read, the lines keyed "phase/kernel" (the phase in force at the launch). */
int inla_test_profile_read_by_phase(char *buf, int len);

/* Dense covariance entries sigma2 * exp(-sqrt((dx * inv_rx)^2 + (dy * inv_ry)^2)) for n <= 8192
 * host points (row-major n x 2), computed by the mixed path's double-float device code (its own
 * exp and sqrt on the FP32 pipes) and returned in out (n x n host doubles). */
int inla_test_cov_df(const double *points, int32_t n, double sigma2, double inv_rx, double inv_ry, double *out);

/* The last batch's Newton iterations (this host thread's most recent inla_eval_batch): for each
 * iteration the largest step over the points still iterating and whether the factor was
 * computed afresh (1) or reused (0).  Writes up to cap entries; returns the iteration count. */
int inla_test_newton_trace(double *steps, int32_t *refactored, int32_t cap);

/* The outer block (panel width) the mixed Cholesky chose for matrices of padded size n_pad
 * factored with `slices` slices (tuned per batch size; this returns the choice for the largest
 * batch decided): 256 or 512 once its two timed candidate runs are complete, 0 while undecided
 * (sizes below 1024 always use 256).  With the environment variable
 * INLA_OUTER_BLOCK=256 or 512 (read once) every size and every tuned routine uses that block,
 * untuned (for profiler captures, whose timings would mislead the tuner), and this returns it. */
int inla_test_outer_block(int32_t n_pad, int32_t slices);

/* The same for the mixed transposed inverse of a factor (Y = F^-T: the inverse of the prior
 * covariance's factor and, for the marginal variances, of the factor at the mode). */
int inla_test_inverse_block(int32_t n_pad, int32_t slices);

/* One cooperative double-float triangular solve of the mixed path on a caller-given lower
 * factor L (host, row-major n x n FP64, n a multiple of 64): x = L^-1 b (backward = 0) or
 * x = L^-T b (backward = 1).  Every wait of a tile on an earlier tile's ready flag gives up
 * after spin_limit polls (0: at once); a wait that gave up makes the call return
 * INLA_E_TIMEOUT (x untouched) with the device still usable. */
int inla_test_trsv_df(const double *L, const double *b, int32_t n, int32_t backward, int64_t spin_limit, double *x);

/* Arithmetic peak probe: best of `reps` timed launches (after one warm-up) of a kernel running
 * eight independent FMA chains per thread on every SM, FP64 (kind 0) or FP32 (kind 1); writes
 * the rate in TFLOP/s (2 flops per FMA).  Changes no device setting. */
int inla_test_fma_peak(int32_t kind, int32_t reps, double *tflops);

#ifdef __cplusplus
}
#endif
#endif /* INLA_TESTING_H */

// Launchers of the CUDA kernels (host-callable), grouped by file.
#pragma once
#include "internal.h"

namespace inla {

// Which matrix of a slot a blocked routine works on.
enum MatSel {
  SEL_L = 0,      // Q / its factor (n_pad), diagonal-tile inverses in Linv
  SEL_COV = 1,    // dense-block covariance / its factor in Wk (nd_pad), inverses in Wd
  SEL_S = 2,      // constraint Schur matrix S (k_pad), inverses in SLinv
  SEL_AUX = 3,    // the Moore-Penrose route's m x m system (aux_n, held in Qp), inverses in Linv
};
// Destination of a triangular inverse.
enum InvDst { DST_L = 0, DST_WK = 1 };

// ---- k_fp64.cu : FP64 tile kernels (64 x 64 tiles) ----
void launch_potrf_diag(Slot* slots, int nslots, int sel, int kt, int max_t, cudaStream_t st);
void launch_trsm_panel(Slot* slots, int nslots, int sel, int kt, int max_t, cudaStream_t st);
void launch_syrk_update(Slot* slots, int nslots, int sel, int kt, int max_t, cudaStream_t st);
// W = F^-1 for the factor selected by `sel`, written to `dst`: step j (descending)
void launch_trtri_step(Slot* slots, int nslots, int sel, int dst, int jt, int max_t, cudaStream_t st);
// Q_p[0:nd, 0:nd] (lower tiles) = W^T W with W the inverse covariance factor held in L
void launch_lauum_cov(Slot* slots, int nslots, int max_td, cudaStream_t st);
// multi-RHS forward substitution on X = Z (n_pad x k_pad) with the factor L: step kt
void launch_fwd_rhs_step(Slot* slots, int nslots, int kt, int max_t, int max_tk, cudaStream_t st);
// S = Z^T Z (lower tiles), identity on the padded diagonal
void launch_schur_syrk(Slot* slots, int nslots, int max_tk, int max_t, cudaStream_t st);
// G^T = Z^T W (k_pad x n_pad, written into L), W = L^-1 held in Wk
void launch_zt_w(Slot* slots, int nslots, int max_tk, int max_t, cudaStream_t st);
// forward substitution with S on the k_pad x n_pad matrix held in L: step kt
void launch_fwd_s_rhs_step(Slot* slots, int nslots, int kt, int max_tk, int max_t, cudaStream_t st);
// vector triangular solves with the selected factor, one tile step; vectors:
// 0 g, 1 t1, 2 t2, 3 kv1, 4 kv2; src is consumed, the solution lands in dst (dst != src)
void launch_trsv_fwd_step(Slot* slots, int nslots, int sel, int src, int dst, int kt, int max_t, cudaStream_t st);
void launch_trsv_bwd_step(Slot* slots, int nslots, int sel, int src, int dst, int kt, int max_t, cudaStream_t st);
// column sums of squares of the lower-triangular matrix held in Wk -> t1 (n_pad)
void launch_colsumsq_wk(Slot* slots, int nslots, int max_t, cudaStream_t st);
// column sums of squares of the k_pad x n_pad matrix held in L -> t2 (n_pad)
void launch_colsumsq_gt(Slot* slots, int nslots, int max_tk, int max_t, cudaStream_t st);
// out[idx] = 2 * sum_i log(diag_i) of the selected factor (deterministic)
void launch_logdet(Slot* slots, int nslots, int sel, int out_idx, cudaStream_t st);

// ---- k_model.cu : prior, likelihood, vectors ----
void launch_cov_build(Slot* slots, int nslots, int max_td, cudaStream_t st);
void launch_prior_entries(Slot* slots, int nslots, int64_t max_entries, cudaStream_t st);
void launch_mirror_qp(Slot* slots, int nslots, int max_t, cudaStream_t st);
void launch_copy_qp_to_l(Slot* slots, int nslots, int max_t, cudaStream_t st);
void launch_add_pairs(Slot* slots, int nslots, int64_t max_pairs, cudaStream_t st);
void launch_prior_logdet(Slot* slots, int nslots, cudaStream_t st);
// eta = A x + o, likelihood sums; mode 0: at x, 1: at xn.  Writes w, r (in eta), OUT_LOGLIK
void launch_eval_lik(Slot* slots, int nslots, int which, int max_m, cudaStream_t st);
// t1 = Q_p v (v = x or xn), OUT_QUAD = v^T t1
void launch_qp_gemv(Slot* slots, int nslots, int which, int max_n, cudaStream_t st);
// OUT_QUAD = v^T t1 only
void launch_quad(Slot* slots, int nslots, int which, cudaStream_t st);
// g = A^T r - t1   (r held in eta)
void launch_gradient(Slot* slots, int nslots, int max_n, cudaStream_t st);
// w, r (in eta) of the weighted least-squares start system, t1 = 0 (mixed Newton's start)
void launch_wls_start(Slot* slots, int nslots, int max_m, int max_n, cudaStream_t st);
// xn = x + g ; kv1 = C xn (if k > 0)
void launch_newton_xu(Slot* slots, int nslots, int max_n, cudaStream_t st);
void launch_cx(Slot* slots, int nslots, int max_k, cudaStream_t st);
// t2 = Z kv1
void launch_z_gemv(Slot* slots, int nslots, int max_n, cudaStream_t st);
// xn -= g
void launch_krige_apply(Slot* slots, int nslots, int max_n, cudaStream_t st);
// OUT_STEP = max |xn - x|
void launch_step_norm(Slot* slots, int nslots, int max_n, cudaStream_t st);
// xn = x + 0.5 (xn - x) for slots flagged in `flags` (device int array)
void launch_halve(Slot* slots, int nslots, const int* flags, int max_n, cudaStream_t st);
// x = xn
void launch_accept(Slot* slots, int nslots, int max_n, cudaStream_t st);
void launch_zero_vec(Slot* slots, int nslots, int which, int max_n, cudaStream_t st);
void launch_ct_fill(Slot* slots, int nslots, int max_k, cudaStream_t st);
void launch_theta_prior(Slot* slots, int nslots, cudaStream_t st);
// var = t1 - t2 (t2 only with constraints) -> t1
void launch_var_finish(Slot* slots, int nslots, int max_n, cudaStream_t st);
void launch_assemble(Slot* slots, int nslots, cudaStream_t st);
// Q* += gamma_c C^T C (lower) for constrained models
void launch_add_cct(Slot* slots, int nslots, cudaStream_t st);

}  // namespace inla

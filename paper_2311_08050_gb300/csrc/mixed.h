// Mixed-precision path: double-float matrices, Ozaki-split tensor-core GEMMs, double-float
// 64 x 64 diagonal tiles.  Declarations shared by eval.cu, eval_mixed.cu and k_df.cu.
#pragma once
#include "kernels.h"
#include "ozaki.h"

namespace inla {

// ---- k_df.cu launchers ----
void launch_cov_build_df(Slot* slots, int nslots, int max_td, cudaStream_t st);
void launch_cov_points_df(const double* P, int n, double sigma2, double irx, double iry, double* out, cudaStream_t st);
void launch_prior_entries_df(Slot* slots, int nslots, int64_t max_entries, cudaStream_t st);
void launch_add_pairs_df(Slot* slots, int nslots, int64_t max_pairs, cudaStream_t st);
void launch_add_cct_df(Slot* slots, int nslots, cudaStream_t st);
void launch_qp_gemv_df(Slot* slots, int nslots, int which, int max_n, cudaStream_t st);
void launch_z_gemv_df(Slot* slots, int nslots, int max_n, cudaStream_t st);
void launch_ct_fill_df(Slot* slots, int nslots, int max_k, cudaStream_t st);
void launch_s_pad_identity(Slot* slots, int nslots, int max_k, cudaStream_t st);
// factor diagonal tile kt of every slot; with `slices` non-null, also write the tile inverse's S
// slices into that operand (64 rows, K = 64): the B operand of the panel product X = A L^-T
void launch_potrf_diag_df(Slot* slots, int nslots, int sel, int kt, const OzOperand* slices, int S, cudaStream_t st);
// triangular solve with a double-float factor (one cooperative launch; see k_df.cu)
struct TrsvArgs {
  Slot* slots;
  int sel, src, dst;
  int nslots, T;        // slots, tile rows of the largest factor
  int backward;         // 0: dst = L^-1 src; 1: dst = L^-T src
  int32_t* flags;       // nslots x T ready flags (zeroed by the launcher)
  int32_t* err;         // set on a timed-out wait
  int64_t spin_limit;
};
int launch_trsv_df(const TrsvArgs& a, cudaStream_t st);
void launch_logdet_df(Slot* slots, int nslots, int sel, int out_idx, cudaStream_t st);
void launch_colsumsq_wk_df(Slot* slots, int nslots, int max_t, cudaStream_t st);
void launch_rowsumsq_wk_df(Slot* slots, int nslots, int max_n, cudaStream_t st);
void launch_colsumsq_gt_df(Slot* slots, int nslots, int max_t, cudaStream_t st);
void launch_diag_ones_df(float2* base, int64_t slot_stride, int ld, int n, int nslots, cudaStream_t st);

// Outer block of the mixed blocked routines: the trailing updates have K = outer block (C is
// read and written n^3 / (3 NB) times per factorisation).  512 (one exact 512-wide chunk per
// update) halves that traffic but deepens the recursive panel factorisation inside each outer
// panel (Cholesky) or doubles the 64-wide steps inside each outer block (triangular routines);
// each routine picks between 256 and 512 per shape (eval_mixed.cu's tuner).
constexpr int MIXED_NB_MAX = 512;   // workspace capacity (largest candidate)

// A batch of slots with identical shapes (uniform per-slot strides).
struct Batch {
  Slot* d_slots;
  std::vector<Slot> h;
  int n;
  int max_t, max_td, max_tk, max_m, max_n, max_k;
  int64_t max_entries, max_pairs;
  cudaStream_t st;
  // uniform layout (slot 0 bases and strides, in elements)
  int np, ndp, kp;
  int64_t mat_stride, z_stride, s_stride, linv_stride, wd_stride, slinv_stride;
  // mixed-path workspace
  bool mixed;
  int S;                 // slices of the GEMMs being issued (set per phase)
  int S_exact = 0;       // prior inversion and the factor at the mode
  int S_newton = 0;      // Newton-step factorisations
  int S_prior = 0;       // prior covariance factorisation, inverse and W^T W
  int S_var = 0;         // inverse of the factor at the mode (marginal variances)
  int S_gram = 0;        // the prior precision W^T W
  uint16_t *PA, *PB, *PBIG;
  int32_t *EA, *EB, *EBIG;
  int64_t pa_cap, pb_cap, pbig_cap;   // elements per slot
  int64_t ea_cap, eb_cap, ebig_cap;   // exponents per slot
  int32_t* err;
  int32_t* flags;        // ready flags of the cooperative triangular solves (slots x tiles)
  int64_t spin_limit;
};

// variational Bayes mean correction (vb.cu): (Q*^-1)_kl for the A^T A pairs and the linear
// predictor's variances (needs the inverse factor in Wk); the correction's residual and weights
void launch_vb_prepare(Slot* slots, int nslots, int mixed, int64_t max_pairs, int max_m, cudaStream_t st);
int launch_vb_terms(Slot* slots, int nslots, int max_m, cudaStream_t st);

// mixed blocked routines (eval_mixed.cu)
int mixed_potrf(Batch& B, int sel);          // replays a captured CUDA graph for a known layout
void mixed_graphs_clear();                   // drop every captured graph (workspace reallocated)
int mixed_nb_choice(int n, int S);           // the Cholesky's tuned outer block for (n, S), 0 if undecided
int mixed_inverse_nb_choice(int n, int S);   // the transposed inverse's, likewise
int mixed_inverse_factor(Batch& B, int sel, bool into_wk);   // Y = F^-T (upper), F by sel
int mixed_lauum_cov(Batch& B);                                // Q_p[0:nd,0:nd] = Y Y^T (Y in L)
int mixed_schur(Batch& B);                                    // Z = L^-1 C^T, S = Z^T Z, factor S
int mixed_var_constraint(Batch& B);                           // t2 = diag(Q^-1 C^T S^-1 C Q^-1)
int mixed_woodbury_variances(Batch& B);                       // t1 = diag(Sigma*) of Eq. (woodeqn)
// Moore-Penrose route kernels (k_df.cu): Q+ into Wk, G = D^1/2 A Q+ into L, M = I + G (D^1/2 A)^T
// into Qp; then t1 = diag(Q+) - column sums of squares of the first aux_n rows of L
void launch_woodbury_terms_df(Slot* slots, int nslots, int max_n, cudaStream_t st);
void launch_woodbury_var_df(Slot* slots, int nslots, int max_n, cudaStream_t st);

}  // namespace inla

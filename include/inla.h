/*
 * inla.h -- C ABI of libinla: the per-hyperparameter evaluation of dense-matrix INLA
 * (INLA+, arXiv 2311.08050) on one GB300 GPU (sm_103a).
 *
 * Model (Section 1, LGM statement):  y_i | x, theta ~ f(eta_i, theta),  eta = A x + offset,
 * x | theta ~ N(0, Q_prior(theta)^-1) (optionally conditioned on C x = 0), theta ~ pi(theta).
 * For one theta the library returns (Eq. (41) of Appendix A.1.1, evaluated at the mode):
 *   log pi~(theta|y) = log pi(theta) + sum_i log p(y_i|eta_hat_i) - 1/2 x_hat^T Q_p x_hat
 *                      + 1/2 log|Q_p| - 1/2 log|Q*| + 1/2 log|C Q_p^-1 C^T| - 1/2 log|C Q*^-1 C^T|
 * with x_hat the conditional mode from the Gaussian-approximation Newton iteration
 * (Algorithm 1, Appendix A.2.1; constraints by conditioning by kriging, Section 5.2 /
 * Appendix C), Q* = Q_p + A^T D(x_hat) A, and the Gaussian marginals
 * x_i | theta, y ~ N(x_hat_i, (Q*^-1)_ii) corrected for the constraints (Appendix A.2.1).
 *
 * Conventions (every entry point):
 *  - Return value: INLA_OK (0) or a negative INLA_E_* code; inla_status_string() names it.
 *    The library never aborts and never prints.
 *  - Ownership: all pointers in descriptors are caller-owned HOST arrays, read only during
 *    the call that receives them (inla_model_create copies everything it needs to the
 *    device).  Output arrays are caller-owned host arrays unless INLA_OPT_DEVICE_OUT is set,
 *    in which case they are device pointers on the current device.
 *  - Layout: CSR matrices use int64 row pointers (nrows+1), int32 column indices and
 *    double values; point coordinates are row-major (size x 2) doubles; theta batches are
 *    row-major (B x theta_dim).
 *  - Threading: a model may be used by one host thread at a time.
 */
#ifndef INLA_H
#define INLA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define INLA_OK                 0
#define INLA_E_BADARG          -1   /* invalid argument or descriptor */
#define INLA_E_CUDA            -2   /* CUDA runtime error (no device, launch failure) */
#define INLA_E_NOT_SPD         -3   /* a Cholesky pivot was not positive */
#define INLA_E_NO_CONVERGENCE  -4   /* Newton did not reach the tolerance in newton_max steps */
#define INLA_E_TIMEOUT         -5   /* a bounded device-side wait gave up */
#define INLA_E_UNSUPPORTED     -6   /* model shape this build does not handle */
#define INLA_E_NOMEM           -7   /* device allocation failed */

/* ---- enumerations ---- */
#define INLA_LIK_POISSON   0   /* y ~ Poisson(exp(eta)), log link, offset = log(expected) */
#define INLA_LIK_GAUSSIAN  1   /* y ~ N(eta, 1/lik_prec) */

#define INLA_BLOCK_FIXED      0  /* precision prec * I (e.g. an intercept, prec = 1e-3) */
#define INLA_BLOCK_IID        1  /* precision exp(theta[theta_idx]) * I */
#define INLA_BLOCK_DENSE_EXP  2  /* covariance sigma^2 exp(-d) + (1/tau_iid + nugget) I on 2-D
                                    points, d = sqrt((dx/rho_x)^2 + (dy/rho_y)^2),
                                    sigma = exp(theta[theta_sigma]), rho_* = exp(theta[..]),
                                    tau_iid = exp(theta[theta_iid]) (theta_iid < 0: absent) */
#define INLA_BLOCK_KRON       3  /* precision exp(theta[theta_idx]) * (R_1 kron ... kron R_f)
                                    + eps I  (Section 5.1 structures) */

#define INLA_FACTOR_ICAR  0   /* Besag: R = D - W of a neighbourhood graph */
#define INLA_FACTOR_RW1   1   /* first-order random walk */
#define INLA_FACTOR_RW2   2   /* second-order random walk */
#define INLA_FACTOR_IID   3   /* identity */

#define INLA_PRIOR_GAUSS    0  /* N(a, b^2) on theta_t */
#define INLA_PRIOR_PC_PREC  1  /* PC prior of the precision exp(theta_t): U = a, alpha = b */

#define INLA_FP64   0   /* every step in IEEE FP64 */
#define INLA_MIXED  1   /* tensor-core (BF16 slices, exact FP32 accumulation) trailing
                           updates, double-float storage, FP64 small diagonal blocks */

#define INLA_OPT_DEVICE_OUT 1  /* x_hat / mean / var outputs are device pointers */
#define INLA_OPT_NO_SHARED_START 2  /* INLA_MIXED: every point runs Newton from x = 0 with its
                                       own factorisations (see inla_eval_batch) */
#define INLA_OPT_VB_MEAN 4  /* the x_hat / mean outputs receive the posterior mean corrected by
                               variational Bayes (Appendix A.2.2, Algorithm 2; see
                               inla_eval_batch) instead of the Laplace mode */
#define INLA_OPT_WOODBURY_VAR 8  /* INLA_MIXED: the var outputs by the Moore-Penrose / Woodbury
                               route of Section 3.1, Eq. (woodeqn) (see inla_eval_batch) */

typedef struct {
  int32_t kind;                 /* INLA_FACTOR_* */
  int32_t size;
  const int64_t *graph_rowptr;  /* ICAR only: symmetric 0/1 adjacency, no diagonal (CSR) */
  const int32_t *graph_col;
} inla_factor;

typedef struct {
  int32_t kind;                 /* INLA_BLOCK_* */
  int32_t size;                 /* number of latent entries in this block */
  double prec;                  /* FIXED */
  int32_t theta_idx;            /* IID, KRON: index of the log precision in theta */
  const double *points;         /* DENSE_EXP: size x 2 coordinates */
  int32_t theta_sigma, theta_range_x, theta_range_y, theta_iid;  /* DENSE_EXP */
  double nugget;                /* DENSE_EXP: added to the covariance diagonal */
  int32_t nfactors;             /* KRON: 1..3 factors, sizes multiply to `size` */
  const inla_factor *factors;
  double eps;                   /* KRON: jitter on the intrinsic structure */
} inla_block;

typedef struct {
  int32_t n, m, k;              /* latent size, observations, constraints (k may be 0) */
  int32_t likelihood;           /* INLA_LIK_* */
  double lik_prec;              /* Gaussian observation precision */
  const int64_t *A_rowptr; const int32_t *A_col; const double *A_val;   /* m x n */
  const double *y;              /* m */
  const double *offset;         /* m, or NULL for zero */
  int32_t nblocks;              /* latent vector = blocks concatenated in order */
  const inla_block *blocks;
  const int64_t *C_rowptr; const int32_t *C_col; const double *C_val;   /* k x n, or NULL */
  int32_t theta_dim;
  const int32_t *theta_prior_kind;            /* theta_dim entries, INLA_PRIOR_* */
  const double *theta_prior_a, *theta_prior_b;
} inla_model_desc;

typedef struct {
  int32_t precision;   /* INLA_FP64 or INLA_MIXED */
  int32_t slices;      /* INLA_MIXED: BF16 slices per operand (2..6) for the prior inversion and
                          the factor at the mode (log-det, variances); 0 = default (5); 6 holds
                          log pi~ to FP64 accuracy (~1e-11 relative measured) */
  int32_t newton_slices; /* INLA_MIXED: slices for the Newton-step factorisations, which only
                          steer convergence (the gradient is exact); 0 = min(4, slices) */
  double newton_tol;   /* infinity-norm step tolerance (default 1e-8) */
  int32_t newton_max;  /* maximum Newton iterations (default 50) */
  int64_t spin_limit;  /* iteration limit of every device-side wait (default 1<<26) */
  void *stream;        /* cudaStream_t to run on, or NULL: the library's own stream of the current
                          device, ordered after the work queued on the legacy default stream
                          before the call and before the work queued there after it */
  int32_t flags;       /* INLA_OPT_* */
  int32_t prior_slices;  /* INLA_MIXED: slices of the prior covariance's factorisation and of the
                          triangular inverse W of its factor; 0 = `slices` */
  double reuse_below;  /* INLA_MIXED modified Newton: a factor may be kept for later iterations
                          once the step (infinity norm) is below this; 0 = default (0.1) */
  double reuse_shrink; /* ... and is kept while every step is at most this fraction of the one
                          before; 0 = default (0.25) */
  int32_t var_slices;  /* INLA_MIXED: slices of the inverse of the factor at the mode, which gives
                          the marginal variances (and their constraint correction): they need
                          ~1e-4 relative where the log-determinant needs ~1e-8; 0 = `slices` */
  int32_t gram_slices; /* INLA_MIXED: slices of the prior precision Q_p = W^T W, which enters log pi~
                          directly (the factorisation and inverse before it only perturb the
                          covariance, whose effect is far smaller); 0 = `prior_slices` */
} inla_opts;

typedef struct inla_model inla_model;   /* opaque; owns device copies of the model */

/* Fill *opts with the defaults above (FP64). */
int inla_opts_default(inla_opts *opts);

/* Validate `desc` and copy the model to the current CUDA device.  The latent field may be
 * re-ordered and padded internally (identity rows); every output uses the caller's order.
 * Constraint rows must each lie in one KRON block and, per block, span exactly the null
 * space of its structure (INLA_E_UNSUPPORTED otherwise).  At most one DENSE_EXP block.
 * Errors: INLA_E_BADARG, INLA_E_UNSUPPORTED, INLA_E_NOMEM, INLA_E_CUDA. */
int inla_model_create(const inla_model_desc *desc, inla_model **out);

/* Release every device and host resource of the model.  NULL is accepted. */
int inla_model_destroy(inla_model *model);

/* One theta (theta_dim doubles): log pi~(theta|y) into *log_post, the mode into x_hat
 * (n doubles, may be NULL) and the Newton iteration count into *newton_iters (may be
 * NULL).  Equivalent to inla_eval_batch with B = 1. */
int inla_eval_theta(inla_model *model, const double *theta, const inla_opts *opts,
                    double *log_post, double *x_hat, int32_t *newton_iters);

/* B theta points, point b on models[model_of_theta[b]] (model_of_theta may be NULL when
 * nmodels == 1).  All points run together on the device.  log_post[b] and status[b]
 * (INLA_OK or a negative code for that point alone) are always written; x_hat[b] and
 * var[b] (n of that model doubles each) are written when the arrays and entries are
 * non-NULL.  The call returns INLA_OK if the batch ran, even when single points failed.
 * INLA_MIXED, Poisson models with several points in the call: the first point of the model
 * runs Newton from x = 0; the others then start from its mode and iterate with its final
 * factor (modified Newton: the gradient is each point's own and exact, so each converges to
 * its own mode to the same step tolerance), taking factorisations of their own only if the
 * steps stop shrinking 4x per iteration.  For the 2t + 1 points of a finite-difference stencil
 * this replaces most Newton-step factorisations.  INLA_OPT_NO_SHARED_START turns it off.
 * INLA_OPT_VB_MEAN: after the Laplace approximation (log_post, var unchanged), the mean is
 * corrected by variational Bayes: with sigma_i^2 = (A Q*^-1 A^T)_ii fixed, each step solves
 * (Q_p + A^T diag(I''(0)) A) lambda = -(A^T I'(0) + Q_p mu), I'(0), I''(0) the means of the
 * negative log-likelihood's first and second derivatives under eta_i ~ N((A mu + offset)_i,
 * sigma_i^2) (15-point Gauss-Hermite), preconditioned by the factor of Q* (same fixed point),
 * until max |lambda| <= 1e-8 (at most 50 steps; INLA_E_NO_CONVERGENCE for the point otherwise).
 * Models with constraints (k > 0) are rejected with INLA_E_UNSUPPORTED.
 * INLA_OPT_WOODBURY_VAR (INLA_MIXED only): the marginal variances are taken from
 * Sigma* = Q+ - Q+ (I + Q_like Q+)^-1 Q_like Q+, Q+ the Moore-Penrose pseudo-inverse of the prior
 * precision without the eps jitter of intrinsic blocks (block by block: 1 / prec, exp(-theta),
 * the dense covariance, and the Kronecker product of the factors' pseudo-inverses over tau), and
 * Q_like = A^T D A at the mode of the kriging route -- evaluated in the symmetric form
 * Q+ - Q+ B^T (I + B Q+ B^T)^-1 B Q+, B = D^1/2 A, whose m x m system needs round_up(m, 256) <=
 * the padded n (INLA_E_UNSUPPORTED otherwise, and with INLA_FP64 or INLA_OPT_VB_MEAN).  As eps -> 0
 * the two routes agree; log_post and x_hat are those of the kriging route. */
int inla_eval_batch(inla_model *const *models, int32_t nmodels, const int32_t *model_of_theta,
                    const double *thetas, int32_t B, const inla_opts *opts,
                    double *log_post, int32_t *status, double *const *x_hat,
                    double *const *var);

/* Gaussian marginals at theta (Appendix A.2.1): mean = x_hat and
 * var = diag(Q*^-1) - diag(Q*^-1 C^T (C Q*^-1 C^T)^-1 C Q*^-1) (n doubles each). */
int inla_marginals(inla_model *model, const double *theta, const inla_opts *opts,
                   double *mean, double *var);

/* Stage 2 (Section 2, Stage 2; Appendix A.2): the latent marginals integrated over K
 * exploration points theta_k of the hyperparameter space (a CCD or grid design).  Inputs per
 * point: log_post[k] = log pi~(theta_k|y) and the Gaussian marginals of that point, rows k of
 * x_hat and var (K x ld, row-major; n <= ld used per row), e.g. from inla_eval_batch;
 * delta[k] >= 0: the design's quadrature weight.  With w_k proportional to
 * delta_k exp(log_post[k]) (normalised; points with a non-finite log_post weigh 0), writes
 * the mixture's moments mean_i = sum_k w_k x_hat_ki and var_i = sum_k w_k (var_ki + x_hat_ki^2)
 * - mean_i^2 (n doubles each).  log_post and delta are host arrays; x_hat, var, mean and
 * var_out are device pointers on the current device with INLA_OPT_DEVICE_OUT in flags, host
 * arrays otherwise.  K <= 4096.  stream: cudaStream_t or NULL; the call synchronizes it.
 * Errors: INLA_E_BADARG (sizes, negative or non-finite delta, no point with weight),
 * INLA_E_NOMEM, INLA_E_CUDA. */
int inla_integrate_marginals(int32_t K, int32_t n, const double *log_post, const double *delta,
                             const double *x_hat, const double *var, int64_t ld, double *mean,
                             double *var_out, int32_t flags, void *stream);

/* Static text for a status code. */
const char *inla_status_string(int status);

/* Allocation-free Ozaki-split tensor-core product C = A B^T (the paper has no counterpart:
 * this is a building block of the mixed path offered on its own).  For callers that cannot
 * call cudaMalloc -- an application that reserves all device memory up front in its own pool
 * and hands out only pointers into it, or code that must not risk the device-wide
 * synchronisation and out-of-memory failure of an allocation mid-work.
 *  A: M x K, B: N x K, C: M x N, row-major FP64 DEVICE pointers on the current device,
 *  caller-owned (inputs read, C overwritten).  M, N, K <= 512, K a multiple of 64,
 *  slices in 2..5; otherwise INLA_E_BADARG.  stream: cudaStream_t or NULL.
 *  Every intermediate lives in one static device array of ~7.4 MB that each GPU loading the
 *  library holds until the process exits; the call allocates nothing (no cudaMalloc, no
 *  library allocator).  The first call on a device looks that array's address up
 *  (cudaGetSymbolAddress); host threads may make their first calls at the same time (the
 *  address is stored atomically).  All calls share the array and it keeps the last call's
 *  contents: calls that overlap on the GPU (other streams, other host threads) race.  The call
 *  reads its error flag back to the host and synchronizes `stream` before returning, so it
 *  cannot be captured into a CUDA graph; INLA_E_TIMEOUT if a bounded device-side wait gave up. */
int inla_ozaki_gemm_noalloc(const double *A, const double *B, double *C, int32_t M, int32_t N, int32_t K,
                            int32_t slices, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* INLA_H */

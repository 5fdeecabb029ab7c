// Internal declarations of libinla (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <vector>
#include <string>
#include "../../include/inla.h"

namespace inla {

constexpr int TB = 64;        // FP64 tile edge
constexpr int PAD = 256;      // latent and dense-block padding unit
constexpr int MAX_THETA = 16;
constexpr int MAX_KRON = 8;
constexpr int HEAVY_LEN = 4096;     // contributions above which a block, not a warp, reduces a sum
constexpr int HEAVY_BLOCKS = 8;     // blocks of a launch given to the heavy sums

#define INLA_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) {                                 \
      return _e == cudaErrorMemoryAllocation ? INLA_E_NOMEM  \
                                             : INLA_E_CUDA;  \
    }                                                        \
  } while (0)

#define INLA_TRY(expr)            \
  do {                            \
    int _s = (expr);              \
    if (_s != INLA_OK) return _s; \
  } while (0)

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Kernel attributes (the dynamic shared-memory limit) and launch geometry belong to the device
// that was current when they were set or queried.  DeviceFlags records a one-time set-up per
// device (indices 0..63; others are never marked, so their set-up runs on every call).
inline int current_device() {
  int d = -1;
  return cudaGetDevice(&d) == cudaSuccess ? d : -1;
}
class DeviceFlags {
 public:
  bool test(int dev) const { return dev >= 0 && dev < 64 && ((bits_.load(std::memory_order_acquire) >> dev) & 1u); }
  void set(int dev) {
    if (dev >= 0 && dev < 64) bits_.fetch_or(uint64_t(1) << dev, std::memory_order_acq_rel);
  }

 private:
  std::atomic<uint64_t> bits_{0};
};

// Structured prior entry of Q_p (lower triangle, internal indices):
// value = a + b * exp(theta[t])  (t < 0: value = a)
struct PriorEntry {
  int32_t row, col, t, pad_;
  double a, b;
};

// Kronecker block: eigenvalues of its structure for log-determinants.
struct KronLogdet {
  int32_t offset;      // into the eigenvalue array
  int32_t size;
  int32_t theta_idx;
  int32_t constrained; // 1: the block's constraints span its null space
  double eps;
};

// A prior block in internal order (the Moore-Penrose route builds the pseudo-inverse of the
// prior precision block by block): INLA_BLOCK_* kind, internal offset and size, its theta index
// (-1 for a fixed block), the fixed precision, and for Kronecker blocks the factors' sizes and
// the offsets of their pseudo-inverses (row-major) in ModelDev::factor_pinv.
constexpr int MAX_BLOCKS = 16;
struct BlockInfo {
  int32_t kind, off, size, theta_idx;
  double prec;
  int32_t nf, fsize[3];
  int64_t pinv_off[3];
};

// Device-resident, theta-independent model data.
struct ModelDev {
  int32_t n, n_pad, m, k, k_pad, nd, nd_pad;   // nd: dense block size (0 if none)
  int32_t nd_off;                              // internal offset of the dense block
  int32_t likelihood;
  double lik_prec;
  int32_t theta_dim;
  // likelihood
  int64_t *A_rowptr; int32_t *A_col; double *A_val;        // m x n_pad, internal columns
  int64_t *At_rowptr; int32_t *At_row; double *At_val;     // n_pad x m (transpose)
  int64_t npairs;
  int32_t *pair_row, *pair_col; int64_t *pair_ptr;         // unique (row >= col) pairs
  // rows of A^T and pairs with more than HEAVY_LEN contributions (e.g. an intercept that every
  // observation loads): reduced by whole blocks instead of one warp each
  int32_t n_heavy_cols, n_heavy_pairs;
  int32_t* heavy_cols;
  int64_t* heavy_pairs;
  // per observation i, the pairs (k, l) of its A row and a_ik a_il (twice for k != l): the
  // variance of eta_i is sum over them of coef * (Q*^-1)_kl
  int64_t* obs_ptr; int32_t* obs_pair; double* obs_coef;
  int32_t nblk;
  BlockInfo blk[MAX_BLOCKS];
  double* factor_pinv;
  int32_t *pc_obs; double *pc_coef;                        // contributions
  double *y, *offset;                                      // offset may be null
  double lgamma_sum;                                       // sum log y! (Poisson)
  // prior
  double *points;                                          // nd x 2
  int32_t theta_sigma, theta_rx, theta_ry, theta_iid;
  double nugget;
  int64_t nentries;
  PriorEntry *entries;
  double prior_const_logdet;                               // fixed blocks
  int32_t nkron;
  KronLogdet kron[MAX_KRON];
  double *kron_eig;
  double logdet_CCt;                                       // constrained blocks
  int32_t n_iid; int32_t iid_theta[MAX_KRON]; int32_t iid_size[MAX_KRON];
  // constraints (k x n_pad), internal columns
  int64_t *C_rowptr; int32_t *C_col; double *C_val;
  int64_t ncct;            // entries of C^T C (lower), value in PriorEntry::a
  PriorEntry *cct;
  double gamma_c;          // weight of C^T C added to Q* in the constrained solves
  // theta prior
  int32_t prior_kind[MAX_THETA];
  double prior_a[MAX_THETA], prior_b[MAX_THETA];
};

}  // namespace inla

struct inla_model {
  inla::ModelDev d;
  std::vector<int32_t> perm;   // perm[original index] = internal index
  std::vector<void*> allocations;
  int device;
};

namespace inla {

// Per-theta working set ("slot"), resident in device memory.
struct Slot {
  // matrices, row-major with leading dimension n_pad (k_pad for S)
  double *Qp;     // prior precision (full symmetric)
  double *L;      // Q, factored in place (lower)
  double *Wk;     // dense-block covariance / inverse factor workspace
  double *Linv;   // n_pad x TB: inverses of the diagonal tiles of L
  double *Z;      // n_pad x k_pad: L^-1 C^T
  double *S;      // k_pad x k_pad: Z^T Z, factored
  double *SLinv;  // k_pad x TB
  double *Wd;     // nd_pad x TB: inverses of the diagonal tiles of the covariance factor
  // vectors
  double *x, *xn, *g, *t1, *t2;    // n_pad
  double *vd;                      // n_pad: double-float copy of a vector (mixed path)
  double *qpart;                   // n_pad / 64 x n_pad: column sums of Q_p's tiles left of the
                                   // diagonal (mixed path, symmetric Q_p v)
  double *vsave;                   // n_pad: the variances while the variational Bayes steps run
  double *eta, *w;                 // m
  double *etav;                    // m: variance of the linear predictor (variational Bayes)
  double *pcov;                    // unique A^T A pairs: (Q*^-1)_kl (variational Bayes)
  double *kv1, *kv2;               // k_pad
  double *red;                     // reduction scratch (256 doubles)
  double *out;                     // scalar outputs (SLOT_NOUT doubles)
  int32_t *info;                   // [0] status flags, [1] failing pivot
  const ModelDev *md;              // device copy of the model struct
  int32_t n_pad, n, m, k, k_pad, nd, nd_pad, nd_off;
  int32_t aux_n;                   // padded size of the Moore-Penrose route's m x m system
  int32_t active;                 // participates in the current Newton step
  double theta[MAX_THETA];
};

// indices into Slot::out
enum {
  OUT_LOGDET_COV = 0,   // log|Sigma| of the dense block
  OUT_LOGDET_Q,         // log|Q*|
  OUT_LOGDET_S,         // log|C Q*^-1 C^T|
  OUT_LOGLIK,           // sum log p(y|eta) (without the constant)
  OUT_QUAD,             // x^T Q_p x
  OUT_STEP,             // max |x_new - x|
  OUT_PRIOR_STRUCT,     // structured prior log-det part (incl. constraint terms)
  OUT_LOG_THETA_PRIOR,  // log pi(theta)
  OUT_LOGDET_TMP,
  OUT_LOGPOST,          // log pi~(theta|y)
  SLOT_NOUT = 16
};

// info flags
enum { INFO_NOT_SPD = 1, INFO_TIMEOUT = 2, INFO_NONFINITE = 4 };

}  // namespace inla

namespace inla {
// Debug mode (environment variable INLA_DEBUG_SYNC=1): every checked site synchronizes the
// stream and records the first site at which a CUDA error became visible.
bool debug_sync_enabled();
int debug_check(cudaStream_t st, const char* site);
// INLA_OK, or INLA_E_CUDA after recording `site` and the pending launch error (which it clears)
int note_launch_error(const char* site);
// number of kernels this library has launched (read and reset by inla_test_launch_count)
extern int64_t g_kernel_launches;
// called before every kernel launch: counts it and, while the profiler is on, records a CUDA
// event on the profiled stream so that per-kernel times can be attributed (prof.cu)
int count_launch(const char* name);
void prof_set_stream(cudaStream_t st);
void prof_phase(const char* name);  // while the profiler is on: a phase boundary of a batch
bool prof_active();          // the per-kernel event profiler is recording
bool oz_stats_active();      // the GEMM launch statistics are recording
}  // namespace inla

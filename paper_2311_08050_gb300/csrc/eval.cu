// One batched theta evaluation: prior build, Newton iterations to the conditional mode
// (Algorithm 1 of Appendix A.2.1, with conditioning by kriging for C x = 0, Section 5.2),
// the final factorisation at the mode, log pi~(theta|y) (Eq. (41)) and the Gaussian
// marginal variances (Appendix A.2.1).  Every point of a batch occupies one "slot"; all
// kernels of a step run over all active slots at once (grid.y / grid.z = slot).
//
// The Newton step is written as x_new = x + Q*(x)^-1 grad f(x), with
// grad f(x) = A^T (y - w) - Q_p x: this equals the solve Q* x_new = grad g + Q_l x of
// Algorithm 1 in exact arithmetic, and its fixed point is the exact mode even when the
// factor is computed in reduced precision.
#include "kernels.h"
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

namespace inla {

void launch_gather(double* dst, const double* src, const int32_t* perm, int n, cudaStream_t st);

// -------------------------------------------------------------------------------------
// device workspace arena (grow-only, process wide)
// -------------------------------------------------------------------------------------
struct Arena {
  void* base = nullptr;
  size_t size = 0;
  int device = -1;
};
static Arena g_arena;
static std::mutex g_mutex;

static int arena_reserve(size_t bytes, int device) {
  if (g_arena.base && g_arena.size >= bytes && g_arena.device == device) return INLA_OK;
  if (g_arena.base) {
    cudaFree(g_arena.base);
    g_arena.base = nullptr;
    g_arena.size = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return INLA_E_NOMEM;
  }
  g_arena.base = p;
  g_arena.size = bytes;
  g_arena.device = device;
  return INLA_OK;
}

struct Carve {
  char* p;
  size_t off = 0;
  explicit Carve(void* base) : p(static_cast<char*>(base)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* r = reinterpret_cast<T*>(p + off);
    off += count * sizeof(T);
    return r;
  }
};

static size_t slot_bytes(const ModelDev& d, bool want_var) {
  (void)want_var;
  const size_t np = d.n_pad, kp = d.k_pad;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) & ~(size_t)255; };
  add(np * np * 8);            // Qp
  add(np * np * 8);            // L
  add(np * np * 8);            // Wk
  add(np * TB * 8);            // Linv
  add(std::max<size_t>(d.nd_pad, 1) * TB * 8);  // Wd
  if (kp) {
    add(np * kp * 8);  // Z
    add(kp * kp * 8);  // S
    add(kp * TB * 8);  // SLinv
    add(kp * 8);
    add(kp * 8);
  }
  for (int v = 0; v < 5; ++v) add(np * 8);
  add(std::max<size_t>(d.m, 1) * 8);
  add(std::max<size_t>(d.m, 1) * 8);
  add(256 * 8);
  add(SLOT_NOUT * 8);
  add(2 * 4);
  add(sizeof(ModelDev));
  return b + 4096;
}

// -------------------------------------------------------------------------------------
// batched blocked routines (host loops over tile steps)
// -------------------------------------------------------------------------------------
struct Batch {
  Slot* d_slots;          // device array
  std::vector<Slot> h;    // host mirror
  int n;                  // number of slots
  int max_t, max_td, max_tk, max_m, max_n, max_k;
  int64_t max_entries, max_pairs;
  cudaStream_t st;
};

static void potrf(Batch& B, int sel) {
  const int T = sel == SEL_L ? B.max_t : sel == SEL_COV ? B.max_td : B.max_tk;
  for (int kt = 0; kt < T; ++kt) {
    launch_potrf_diag(B.d_slots, B.n, sel, kt, T, B.st);
    launch_trsm_panel(B.d_slots, B.n, sel, kt, T, B.st);
    launch_syrk_update(B.d_slots, B.n, sel, kt, T, B.st);
  }
}

static void trtri(Batch& B, int sel, int dst) {
  const int T = sel == SEL_L ? B.max_t : B.max_td;
  for (int jt = T - 1; jt >= 0; --jt)
    launch_trtri_step(B.d_slots, B.n, sel, dst, jt, T, B.st);
}

// dst = M^-1 src for the factor M = L L^T selected by sel (vectors by id)
static void solve_llt(Batch& B, int sel, int src, int tmp, int dst) {
  const int T = sel == SEL_L ? B.max_t : B.max_tk;
  for (int kt = 0; kt < T; ++kt) launch_trsv_fwd_step(B.d_slots, B.n, sel, src, tmp, kt, T, B.st);
  for (int kt = T - 1; kt >= 0; --kt) launch_trsv_bwd_step(B.d_slots, B.n, sel, tmp, dst, kt, T, B.st);
}
static void solve_lt(Batch& B, int sel, int src, int dst) {
  const int T = sel == SEL_L ? B.max_t : B.max_tk;
  for (int kt = T - 1; kt >= 0; --kt) launch_trsv_bwd_step(B.d_slots, B.n, sel, src, dst, kt, T, B.st);
}

enum { V_G = 0, V_T1 = 1, V_T2 = 2, V_KV1 = 3, V_KV2 = 4 };

// Z = L^-1 C^T, S = Z^T Z, factor S
static void constraint_schur(Batch& B) {
  for (int i = 0; i < B.n; ++i)
    if (B.h[i].active && B.h[i].k > 0)
      cudaMemsetAsync(B.h[i].Z, 0, (size_t)B.h[i].n_pad * B.h[i].k_pad * 8, B.st);
  launch_ct_fill(B.d_slots, B.n, B.max_k, B.st);
  for (int kt = 0; kt < B.max_t; ++kt) launch_fwd_rhs_step(B.d_slots, B.n, kt, B.max_t, B.max_tk, B.st);
  launch_schur_syrk(B.d_slots, B.n, B.max_tk, B.max_t, B.st);
  potrf(B, SEL_S);
}

static void sync_active(Batch& B) {
  cudaMemcpyAsync(B.d_slots, B.h.data(), sizeof(Slot) * B.n, cudaMemcpyHostToDevice, B.st);
}

static int read_outputs(Batch& B, std::vector<double>& out, std::vector<int32_t>& info) {
  out.resize((size_t)B.n * SLOT_NOUT);
  info.resize((size_t)B.n * 2);
  for (int i = 0; i < B.n; ++i) {
    cudaMemcpyAsync(&out[(size_t)i * SLOT_NOUT], B.h[i].out, SLOT_NOUT * 8, cudaMemcpyDeviceToHost, B.st);
    cudaMemcpyAsync(&info[(size_t)i * 2], B.h[i].info, 8, cudaMemcpyDeviceToHost, B.st);
  }
  INLA_CUDA_TRY(cudaStreamSynchronize(B.st));
  return INLA_OK;
}

static void fail_slot(Batch& B, std::vector<int>& status, int i, int code) {
  if (status[i] == INLA_OK) status[i] = code;
  B.h[i].active = 0;
}

// objective f(x) = sum log p(y|eta) - 1/2 x^T Q_p x (with the constant of log y!)
static double objective(const ModelDev& md, const double* out) {
  double f = out[OUT_LOGLIK] - 0.5 * out[OUT_QUAD];
  if (md.likelihood == INLA_LIK_POISSON) f -= md.lgamma_sum;
  return f;
}

static int run_batch(Batch& B, const std::vector<const ModelDev*>& models, const inla_opts& o, bool want_var,
                     std::vector<int>& status, std::vector<int>& iters) {
  const int NB = B.n;
  std::vector<double> out;
  std::vector<int32_t> info;
  status.assign(NB, INLA_OK);
  iters.assign(NB, 0);
  for (int i = 0; i < NB; ++i) {
    cudaMemsetAsync(B.h[i].out, 0, SLOT_NOUT * 8, B.st);
    const int32_t init_info[2] = {0, INT_MAX};
    cudaMemcpyAsync(B.h[i].info, init_info, 8, cudaMemcpyHostToDevice, B.st);
    B.h[i].active = 1;
  }
  sync_active(B);
  // ---------------- prior precision ----------------
  launch_theta_prior(B.d_slots, NB, B.st);
  for (int i = 0; i < NB; ++i) cudaMemsetAsync(B.h[i].Qp, 0, (size_t)B.h[i].n_pad * B.h[i].n_pad * 8, B.st);
  if (B.max_td > 0) {
    launch_cov_build(B.d_slots, NB, B.max_td, B.st);
    potrf(B, SEL_COV);
    launch_logdet(B.d_slots, NB, SEL_COV, OUT_LOGDET_COV, B.st);
    trtri(B, SEL_COV, DST_L);
    launch_lauum_cov(B.d_slots, NB, B.max_td, B.st);
  }
  launch_prior_entries(B.d_slots, NB, B.max_entries, B.st);
  launch_mirror_qp(B.d_slots, NB, B.max_t, B.st);
  launch_prior_logdet(B.d_slots, NB, B.st);
  INLA_TRY(read_outputs(B, out, info));
  for (int i = 0; i < NB; ++i)
    if (info[2 * i] & INFO_NOT_SPD) fail_slot(B, status, i, INLA_E_NOT_SPD);
  sync_active(B);
  // ---------------- Newton iterations ----------------
  launch_zero_vec(B.d_slots, NB, 0, B.max_n, B.st);
  launch_eval_lik(B.d_slots, NB, 0, B.max_m, B.st);
  launch_qp_gemv(B.d_slots, NB, 0, B.max_n, B.st);
  INLA_TRY(read_outputs(B, out, info));
  std::vector<double> f_old(NB);
  for (int i = 0; i < NB; ++i) f_old[i] = objective(*models[i], &out[(size_t)i * SLOT_NOUT]);
  std::vector<int> converged(NB, 0);
  int* d_flags = nullptr;
  INLA_CUDA_TRY(cudaMallocAsync((void**)&d_flags, sizeof(int) * NB, B.st));
  std::vector<int> flags(NB, 0);
  for (int it = 1; it <= o.newton_max; ++it) {
    int nact = 0;
    for (int i = 0; i < NB; ++i) nact += B.h[i].active;
    if (nact == 0) break;
    for (int i = 0; i < NB; ++i)
      if (B.h[i].active) iters[i] = it;
    // Q* = Q_p + A^T D A at x ; gradient ; factor ; Newton direction
    launch_copy_qp_to_l(B.d_slots, NB, B.max_t, B.st);
    launch_add_pairs(B.d_slots, NB, B.max_pairs, B.st);
    launch_gradient(B.d_slots, NB, B.max_n, B.st);
    potrf(B, SEL_L);
    solve_llt(B, SEL_L, V_G, V_T2, V_G);
    launch_newton_xu(B.d_slots, NB, B.max_n, B.st);
    if (B.max_k > 0) {
      constraint_schur(B);
      launch_cx(B.d_slots, NB, B.max_k, B.st);
      solve_llt(B, SEL_S, V_KV1, V_KV2, V_KV1);
      launch_z_gemv(B.d_slots, NB, B.max_n, B.st);
      solve_lt(B, SEL_L, V_T2, V_G);
      launch_krige_apply(B.d_slots, NB, B.max_n, B.st);
    }
    launch_eval_lik(B.d_slots, NB, 1, B.max_m, B.st);
    launch_qp_gemv(B.d_slots, NB, 1, B.max_n, B.st);
    launch_step_norm(B.d_slots, NB, B.max_n, B.st);
    INLA_TRY(read_outputs(B, out, info));
    for (int i = 0; i < NB; ++i)
      if (B.h[i].active && (info[2 * i] & INFO_NOT_SPD)) fail_slot(B, status, i, INLA_E_NOT_SPD);
    // step halving while the objective decreases
    for (int h = 0; h < 30; ++h) {
      int any = 0;
      for (int i = 0; i < NB; ++i) {
        flags[i] = 0;
        if (!B.h[i].active || models[i]->likelihood == INLA_LIK_GAUSSIAN) continue;
        const double fn = objective(*models[i], &out[(size_t)i * SLOT_NOUT]);
        if (fn < f_old[i] - 1e-10 * (1.0 + std::fabs(f_old[i]))) flags[i] = any = 1;
      }
      if (!any) break;
      cudaMemcpyAsync(d_flags, flags.data(), sizeof(int) * NB, cudaMemcpyHostToDevice, B.st);
      launch_halve(B.d_slots, NB, d_flags, B.max_n, B.st);
      launch_eval_lik(B.d_slots, NB, 1, B.max_m, B.st);
      launch_qp_gemv(B.d_slots, NB, 1, B.max_n, B.st);
      launch_step_norm(B.d_slots, NB, B.max_n, B.st);
      INLA_TRY(read_outputs(B, out, info));
    }
    launch_accept(B.d_slots, NB, B.max_n, B.st);
    for (int i = 0; i < NB; ++i) {
      if (!B.h[i].active) continue;
      const double* oi = &out[(size_t)i * SLOT_NOUT];
      f_old[i] = objective(*models[i], oi);
      if (!std::isfinite(f_old[i])) {
        fail_slot(B, status, i, INLA_E_NO_CONVERGENCE);
        continue;
      }
      if (models[i]->likelihood == INLA_LIK_GAUSSIAN || oi[OUT_STEP] <= o.newton_tol) {
        converged[i] = 1;
        B.h[i].active = 0;
      }
    }
    sync_active(B);
  }
  cudaFreeAsync(d_flags, B.st);
  for (int i = 0; i < NB; ++i) {
    if (status[i] == INLA_OK && !converged[i]) status[i] = INLA_E_NO_CONVERGENCE;
    B.h[i].active = status[i] == INLA_OK;
  }
  sync_active(B);
  // ---------------- at the mode ----------------
  launch_eval_lik(B.d_slots, NB, 0, B.max_m, B.st);
  launch_qp_gemv(B.d_slots, NB, 0, B.max_n, B.st);
  launch_copy_qp_to_l(B.d_slots, NB, B.max_t, B.st);
  launch_add_pairs(B.d_slots, NB, B.max_pairs, B.st);
  potrf(B, SEL_L);
  launch_logdet(B.d_slots, NB, SEL_L, OUT_LOGDET_Q, B.st);
  if (B.max_k > 0) {
    constraint_schur(B);
    launch_logdet(B.d_slots, NB, SEL_S, OUT_LOGDET_S, B.st);
  }
  if (want_var) {
    trtri(B, SEL_L, DST_WK);
    launch_colsumsq_wk(B.d_slots, NB, B.max_t, B.st);
    if (B.max_k > 0) {
      launch_zt_w(B.d_slots, NB, B.max_tk, B.max_t, B.st);
      for (int kt = 0; kt < B.max_tk; ++kt) launch_fwd_s_rhs_step(B.d_slots, NB, kt, B.max_tk, B.max_t, B.st);
      launch_colsumsq_gt(B.d_slots, NB, B.max_tk, B.max_t, B.st);
      launch_var_finish(B.d_slots, NB, B.max_n, B.st);
    }
  }
  launch_assemble(B.d_slots, NB, B.st);
  INLA_TRY(read_outputs(B, out, info));
  for (int i = 0; i < NB; ++i)
    if (B.h[i].active && (info[2 * i] & INFO_NOT_SPD)) fail_slot(B, status, i, INLA_E_NOT_SPD);
  return INLA_OK;
}

// log-determinant of a host SPD matrix (k_pad x k_pad, k_pad a multiple of TB) on the device
int logdet_spd_device(const std::vector<double>& Mhost, int k, double* result) {
  std::lock_guard<std::mutex> lock(g_mutex);
  Slot s;
  std::memset(&s, 0, sizeof(s));
  void* mem = nullptr;
  const size_t bytes = (size_t)k * k * 8 + (size_t)k * TB * 8 + SLOT_NOUT * 8 + 64 + sizeof(Slot) + 1024;
  INLA_CUDA_TRY(cudaMalloc(&mem, bytes));
  Carve cv(mem);
  s.S = cv.take<double>((size_t)k * k);
  s.SLinv = cv.take<double>((size_t)k * TB);
  s.out = cv.take<double>(SLOT_NOUT);
  s.info = cv.take<int32_t>(2);
  Slot* d_slot = cv.take<Slot>(1);
  s.k = s.k_pad = k;
  s.active = 1;
  int st = INLA_OK;
  const int32_t init_info[2] = {0, INT_MAX};
  if (cudaMemcpy(s.S, Mhost.data(), (size_t)k * k * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s.info, init_info, 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_slot, &s, sizeof(Slot), cudaMemcpyHostToDevice) != cudaSuccess) {
    st = INLA_E_CUDA;
  } else {
    Batch B;
    B.d_slots = d_slot;
    B.n = 1;
    B.max_tk = k / TB;
    B.st = 0;
    potrf(B, SEL_S);
    launch_logdet(d_slot, 1, SEL_S, OUT_LOGDET_S, 0);
    double o[SLOT_NOUT];
    int32_t inf[2];
    if (cudaMemcpy(o, s.out, sizeof(o), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(inf, s.info, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = INLA_E_CUDA;
    else if (inf[0] & INFO_NOT_SPD)
      st = INLA_E_UNSUPPORTED;  // rows of C are linearly dependent
    else
      *result = o[OUT_LOGDET_S];
  }
  cudaFree(mem);
  return st;
}

static int eval_batch_impl(inla_model* const* models, int32_t nmodels, const int32_t* model_of_theta,
                           const double* thetas, int32_t B_, const inla_opts* opts_in, double* log_post,
                           int32_t* status_out, double* const* x_hat, double* const* var,
                           int32_t* iters_out = nullptr) {
  if (!models || nmodels <= 0 || !thetas || B_ <= 0 || !log_post || !status_out) return INLA_E_BADARG;
  if (nmodels > 1 && !model_of_theta) return INLA_E_BADARG;
  inla_opts o;
  inla_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (o.newton_tol <= 0) o.newton_tol = 1e-8;
  if (o.newton_max <= 0) o.newton_max = 50;
  if (o.precision != INLA_FP64) return INLA_E_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(o.stream);
  const bool dev_out = (o.flags & INLA_OPT_DEVICE_OUT) != 0;
  const bool want_var = var != nullptr;
  std::vector<const ModelDev*> mlist(B_);
  int theta_dim = -1;
  for (int b = 0; b < B_; ++b) {
    const int mi = model_of_theta ? model_of_theta[b] : 0;
    if (mi < 0 || mi >= nmodels || !models[mi]) return INLA_E_BADARG;
    mlist[b] = &models[mi]->d;
    if (theta_dim >= 0 && theta_dim != models[mi]->d.theta_dim) return INLA_E_BADARG;
    theta_dim = models[mi]->d.theta_dim;
  }
  for (int64_t i = 0; i < (int64_t)B_ * theta_dim; ++i)
    if (!std::isfinite(thetas[i])) return INLA_E_BADARG;
  int device = 0;
  INLA_CUDA_TRY(cudaGetDevice(&device));
  std::lock_guard<std::mutex> lock(g_mutex);
  // workspace: all slots, the model structs, the slot table, permutations
  size_t bytes = 0;
  for (int b = 0; b < B_; ++b) bytes += slot_bytes(*mlist[b], want_var);
  bytes += sizeof(Slot) * B_ + 4096;
  int max_n_pad = 0;
  for (int mi = 0; mi < nmodels; ++mi) {
    bytes += sizeof(ModelDev) + (size_t)models[mi]->d.n * sizeof(int32_t) + 512;
    max_n_pad = std::max(max_n_pad, models[mi]->d.n_pad);
  }
  bytes += (size_t)max_n_pad * sizeof(double) + 512;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (bytes > (size_t)(0.95 * (double)(free_b + (g_arena.device == device ? g_arena.size : 0))))
    return INLA_E_NOMEM;
  INLA_TRY(arena_reserve(bytes, device));
  Carve cv(g_arena.base);
  Batch Bt;
  Bt.n = B_;
  Bt.st = st;
  Bt.h.resize(B_);
  Bt.max_t = Bt.max_td = Bt.max_tk = Bt.max_m = Bt.max_n = Bt.max_k = 0;
  Bt.max_entries = Bt.max_pairs = 0;
  std::vector<ModelDev*> d_models(nmodels, nullptr);
  for (int mi = 0; mi < nmodels; ++mi) {
    d_models[mi] = cv.take<ModelDev>(1);
    cudaMemcpyAsync(d_models[mi], &models[mi]->d, sizeof(ModelDev), cudaMemcpyHostToDevice, st);
  }
  for (int b = 0; b < B_; ++b) {
    const int mi = model_of_theta ? model_of_theta[b] : 0;
    const ModelDev& d = *mlist[b];
    Slot& s = Bt.h[b];
    std::memset(&s, 0, sizeof(s));
    const size_t np = d.n_pad, kp = d.k_pad;
    s.Qp = cv.take<double>(np * np);
    s.L = cv.take<double>(np * np);
    s.Wk = cv.take<double>(np * np);
    s.Linv = cv.take<double>(np * TB);
    s.Wd = cv.take<double>(std::max<size_t>(d.nd_pad, 1) * TB);
    if (kp) {
      s.Z = cv.take<double>(np * kp);
      s.S = cv.take<double>(kp * kp);
      s.SLinv = cv.take<double>(kp * TB);
      s.kv1 = cv.take<double>(kp);
      s.kv2 = cv.take<double>(kp);
    }
    s.x = cv.take<double>(np);
    s.xn = cv.take<double>(np);
    s.g = cv.take<double>(np);
    s.t1 = cv.take<double>(np);
    s.t2 = cv.take<double>(np);
    s.eta = cv.take<double>(std::max<size_t>(d.m, 1));
    s.w = cv.take<double>(std::max<size_t>(d.m, 1));
    s.red = cv.take<double>(256);
    s.out = cv.take<double>(SLOT_NOUT);
    s.info = cv.take<int32_t>(2);
    s.md = d_models[mi];
    s.n_pad = d.n_pad;
    s.n = d.n;
    s.m = d.m;
    s.k = d.k;
    s.k_pad = d.k_pad;
    s.nd = d.nd;
    s.nd_pad = d.nd_pad;
    s.active = 1;
    for (int t = 0; t < theta_dim; ++t) s.theta[t] = thetas[(size_t)b * theta_dim + t];
    Bt.max_t = std::max(Bt.max_t, d.n_pad / TB);
    Bt.max_td = std::max(Bt.max_td, d.nd_pad / TB);
    Bt.max_tk = std::max(Bt.max_tk, d.k_pad / TB);
    Bt.max_m = std::max(Bt.max_m, d.m);
    Bt.max_n = std::max(Bt.max_n, d.n_pad);
    Bt.max_k = std::max(Bt.max_k, d.k_pad);
    Bt.max_entries = std::max(Bt.max_entries, d.nentries);
    Bt.max_pairs = std::max(Bt.max_pairs, d.npairs);
  }
  Bt.d_slots = cv.take<Slot>(B_);
  // permutations (internal -> original gather), one per model
  std::vector<int32_t*> d_perm(nmodels, nullptr);
  for (int mi = 0; mi < nmodels; ++mi) {
    d_perm[mi] = cv.take<int32_t>(models[mi]->d.n);
    cudaMemcpyAsync(d_perm[mi], models[mi]->perm.data(), sizeof(int32_t) * models[mi]->d.n, cudaMemcpyHostToDevice, st);
  }
  double* d_gather = cv.take<double>(Bt.max_n);
  if (cv.off > g_arena.size) return INLA_E_NOMEM;
  std::vector<int> status, iters;
  int rc = run_batch(Bt, mlist, o, want_var, status, iters);
  if (rc != INLA_OK) return rc;
  std::vector<double> out;
  std::vector<int32_t> info;
  // outputs
  for (int b = 0; b < B_; ++b) Bt.h[b].active = 1;
  INLA_TRY(read_outputs(Bt, out, info));
  for (int b = 0; b < B_; ++b) {
    const int mi = model_of_theta ? model_of_theta[b] : 0;
    const int n = models[mi]->d.n;
    status_out[b] = status[b];
    if (iters_out) iters_out[b] = iters[b];
    log_post[b] =status[b] == INLA_OK ? out[(size_t)b * SLOT_NOUT + OUT_LOGPOST] : NAN;
    const double* srcs[2] = {Bt.h[b].x, Bt.h[b].t1};
    double* const* dsts[2] = {x_hat, var};
    for (int q = 0; q < 2; ++q) {
      if (!dsts[q] || !dsts[q][b]) continue;
      if (dev_out) {
        launch_gather(dsts[q][b], srcs[q], d_perm[mi], n, st);
      } else {
        launch_gather(d_gather, srcs[q], d_perm[mi], n, st);
        cudaMemcpyAsync(dsts[q][b], d_gather, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
      }
    }
  }
  INLA_CUDA_TRY(cudaStreamSynchronize(st));
  INLA_CUDA_TRY(cudaGetLastError());
  return INLA_OK;
}

__global__ void k_gather(double* dst, const double* src, const int32_t* perm, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[perm[i]];
}
void launch_gather(double* dst, const double* src, const int32_t* perm, int n, cudaStream_t st) {
  k_gather<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(dst, src, perm, n);
}

}  // namespace inla

using namespace inla;

extern "C" int inla_opts_default(inla_opts* o) {
  if (!o) return INLA_E_BADARG;
  std::memset(o, 0, sizeof(*o));
  o->precision = INLA_FP64;
  o->slices = 0;
  o->newton_tol = 1e-8;
  o->newton_max = 50;
  o->spin_limit = (int64_t)1 << 26;
  o->stream = nullptr;
  o->flags = 0;
  return INLA_OK;
}

extern "C" int inla_eval_batch(inla_model* const* models, int32_t nmodels, const int32_t* model_of_theta,
                               const double* thetas, int32_t B, const inla_opts* opts, double* log_post,
                               int32_t* status, double* const* x_hat, double* const* var) {
  int rc = eval_batch_impl(models, nmodels, model_of_theta, thetas, B, opts, log_post, status, x_hat, var);
  if (rc == INLA_E_CUDA) cudaGetLastError();
  return rc;
}

extern "C" int inla_eval_theta(inla_model* model, const double* theta, const inla_opts* opts, double* log_post,
                               double* x_hat, int32_t* newton_iters) {
  if (!model || !theta || !log_post) return INLA_E_BADARG;
  int32_t st = 0;
  double* xs[1] = {x_hat};
  inla_model* ms[1] = {model};
  int32_t it = 0;
  int rc = eval_batch_impl(ms, 1, nullptr, theta, 1, opts, log_post, &st, x_hat ? xs : nullptr, nullptr, &it);
  if (rc == INLA_E_CUDA) cudaGetLastError();
  if (newton_iters) *newton_iters = it;
  if (rc != INLA_OK) return rc;
  return st;
}

extern "C" int inla_marginals(inla_model* model, const double* theta, const inla_opts* opts, double* mean,
                              double* var) {
  if (!model || !theta || !mean || !var) return INLA_E_BADARG;
  int32_t st = 0;
  double lp = 0;
  double* xs[1] = {mean};
  double* vs[1] = {var};
  inla_model* ms[1] = {model};
  int rc = inla_eval_batch(ms, 1, nullptr, theta, 1, opts, &lp, &st, xs, vs);
  if (rc != INLA_OK) return rc;
  return st;
}

extern "C" const char* inla_status_string(int s) {
  switch (s) {
    case INLA_OK: return "ok";
    case INLA_E_BADARG: return "invalid argument";
    case INLA_E_CUDA: return "CUDA runtime error";
    case INLA_E_NOT_SPD: return "matrix not positive definite";
    case INLA_E_NO_CONVERGENCE: return "Newton iteration did not converge";
    case INLA_E_TIMEOUT: return "device-side wait timed out";
    case INLA_E_UNSUPPORTED: return "unsupported model or option";
    case INLA_E_NOMEM: return "out of device memory";
    default: return "unknown status";
  }
}

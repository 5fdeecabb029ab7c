// One batched theta evaluation: prior build, Newton iterations to the conditional mode
// (Algorithm 1 of Appendix A.2.1, with conditioning by kriging for C x = 0, Section 5.2),
// the final factorisation at the mode, log pi~(theta|y) (Eq. (41)) and the Gaussian
// marginal variances (Appendix A.2.1).  Every point of a batch occupies one "slot"; all
// kernels of a step run over all active slots at once (grid.y / grid.z = slot).  Points
// are grouped by model shape so that a group's matrices have uniform per-slot strides.
//
// The Newton step is written as x_new = x + Q*(x)^-1 grad f(x), with
// grad f(x) = A^T (y - w) - Q_p x: this equals the solve Q* x_new = grad g + Q_l x of
// Algorithm 1 in exact arithmetic, and its fixed point is the exact mode even when the
// factor is computed in reduced precision (mixed path).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include "mixed.h"

namespace inla {

void launch_gather(double* dst, const double* src, const int32_t* perm, int n, cudaStream_t st);

int64_t g_kernel_launches = 0;
static char g_debug_site[256] = "";
// last batch's Newton iterations: largest step over the active points, fresh factor or reused
struct NewtonTraceEntry {
  double step;
  int refactored;
};
static std::vector<NewtonTraceEntry> g_newton_trace;
bool debug_sync_enabled() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("INLA_DEBUG_SYNC");
    on = (e && e[0] == '1') ? 1 : 0;
  }
  return on == 1;
}
int note_launch_error(const char* site) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return INLA_OK;
  if (!g_debug_site[0]) snprintf(g_debug_site, sizeof(g_debug_site), "%s: %s", site, cudaGetErrorString(e));
  return INLA_E_CUDA;
}
int debug_check(cudaStream_t st, const char* site) {
  if (!debug_sync_enabled()) return INLA_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (!g_debug_site[0]) snprintf(g_debug_site, sizeof(g_debug_site), "%s: %s", site, cudaGetErrorString(e));
    return INLA_E_CUDA;
  }
  return INLA_OK;
}

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
  mixed_graphs_clear();  // captured graphs hold pointers into the old workspace
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

// bump allocator over a base pointer; with base == nullptr it only measures
struct Carve {
  char* p;
  size_t off = 0;
  explicit Carve(void* base) : p(static_cast<char*>(base)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* r = p ? reinterpret_cast<T*>(p + off) : nullptr;
    off += count * sizeof(T);
    return r;
  }
};

// -------------------------------------------------------------------------------------
// FP64 blocked routines (host loops over tile steps)
// -------------------------------------------------------------------------------------
static void potrf64(Batch& B, int sel) {
  const int T = sel == SEL_L ? B.max_t : sel == SEL_COV ? B.max_td : B.max_tk;
  for (int kt = 0; kt < T; ++kt) {
    launch_potrf_diag(B.d_slots, B.n, sel, kt, T, B.st);
    launch_trsm_panel(B.d_slots, B.n, sel, kt, T, B.st);
    launch_syrk_update(B.d_slots, B.n, sel, kt, T, B.st);
  }
}
static void trtri64(Batch& B, int sel, int dst) {
  const int T = sel == SEL_L ? B.max_t : B.max_td;
  for (int jt = T - 1; jt >= 0; --jt) launch_trtri_step(B.d_slots, B.n, sel, dst, jt, T, B.st);
}

enum { V_G = 0, V_T1 = 1, V_T2 = 2, V_KV1 = 3, V_KV2 = 4 };

static int trsv_df(Batch& B, int sel, int src, int dst, int backward) {
  TrsvArgs a;
  a.slots = B.d_slots;
  a.sel = sel;
  a.src = src;
  a.dst = dst;
  a.nslots = B.n;
  a.T = sel == SEL_L ? B.max_t : B.max_tk;
  a.backward = backward;
  a.flags = B.flags;
  a.err = B.err;
  a.spin_limit = B.spin_limit;
  return launch_trsv_df(a, B.st);
}

// dst = M^-1 src for M = L L^T selected by sel; tmp receives L^-1 src
static int solve_llt(Batch& B, int sel, int src, int tmp, int dst) {
  const int T = sel == SEL_L ? B.max_t : B.max_tk;
  if (B.mixed) {
    INLA_TRY(trsv_df(B, sel, src, tmp, 0));
    return trsv_df(B, sel, tmp, dst, 1);
  }
  for (int kt = 0; kt < T; ++kt) launch_trsv_fwd_step(B.d_slots, B.n, sel, src, tmp, kt, T, B.st);
  for (int kt = T - 1; kt >= 0; --kt) launch_trsv_bwd_step(B.d_slots, B.n, sel, tmp, dst, kt, T, B.st);
  return INLA_OK;
}
static int solve_lt(Batch& B, int sel, int src, int dst) {
  const int T = sel == SEL_L ? B.max_t : B.max_tk;
  if (B.mixed) return trsv_df(B, sel, src, dst, 1);
  for (int kt = T - 1; kt >= 0; --kt) launch_trsv_bwd_step(B.d_slots, B.n, sel, src, dst, kt, T, B.st);
  return INLA_OK;
}

// ---- precision-dispatched steps ----
static int op_potrf(Batch& B, int sel) {
  if (B.mixed) return mixed_potrf(B, sel);
  potrf64(B, sel);
  return INLA_OK;
}
static void op_logdet(Batch& B, int sel, int out) {
  if (B.mixed) launch_logdet_df(B.d_slots, B.n, sel, out, B.st);
  else launch_logdet(B.d_slots, B.n, sel, out, B.st);
}
static void op_qp_gemv(Batch& B, int which) {
  if (B.mixed) {
    launch_qp_gemv_df(B.d_slots, B.n, which, B.max_n, B.st);
    launch_quad(B.d_slots, B.n, which, B.st);
  } else {
    launch_qp_gemv(B.d_slots, B.n, which, B.max_n, B.st);
  }
}
static void op_assemble_q(Batch& B) {
  launch_copy_qp_to_l(B.d_slots, B.n, B.max_t, B.st);  // bit copy (FP64 or df64 elements)
  if (B.mixed) launch_add_pairs_df(B.d_slots, B.n, B.max_pairs, B.st);
  else launch_add_pairs(B.d_slots, B.n, B.max_pairs, B.st);
  if (B.max_k > 0) {  // Q* + gamma C^T C: same kriged results, conditioned null directions
    if (B.mixed) launch_add_cct_df(B.d_slots, B.n, B.st);
    else launch_add_cct(B.d_slots, B.n, B.st);
  }
}
// Z = L^-1 C^T, S = Z^T Z, factor S
static int op_schur(Batch& B) {
  if (B.mixed) return mixed_schur(B);
  for (int i = 0; i < B.n; ++i)
    if (B.h[i].active && B.h[i].k > 0) cudaMemsetAsync(B.h[i].Z, 0, (size_t)B.h[i].n_pad * B.h[i].k_pad * 8, B.st);
  launch_ct_fill(B.d_slots, B.n, B.max_k, B.st);
  for (int kt = 0; kt < B.max_t; ++kt) launch_fwd_rhs_step(B.d_slots, B.n, kt, B.max_t, B.max_tk, B.st);
  launch_schur_syrk(B.d_slots, B.n, B.max_tk, B.max_t, B.st);
  potrf64(B, SEL_S);
  return INLA_OK;
}
static int op_prior_dense(Batch& B) {
  if (B.mixed) {
    launch_cov_build_df(B.d_slots, B.n, B.max_td, B.st);
    INLA_TRY(mixed_potrf(B, SEL_COV));
    launch_logdet_df(B.d_slots, B.n, SEL_COV, OUT_LOGDET_COV, B.st);
    INLA_TRY(mixed_inverse_factor(B, SEL_COV, false));
    const int S_keep = B.S;
    B.S = B.S_gram;  // Q_p itself: its own slice count
    const int rc = mixed_lauum_cov(B);
    B.S = S_keep;
    return rc;
  }
  launch_cov_build(B.d_slots, B.n, B.max_td, B.st);
  potrf64(B, SEL_COV);
  launch_logdet(B.d_slots, B.n, SEL_COV, OUT_LOGDET_COV, B.st);
  trtri64(B, SEL_COV, DST_L);
  launch_lauum_cov(B.d_slots, B.n, B.max_td, B.st);
  return INLA_OK;
}
static int op_variances(Batch& B) {
  if (B.mixed) {
    // the inverse of the factor at the mode only feeds the variances (and, with the variational
    // Bayes correction, the linear predictor's variances): its own slice count
    const int S_keep = B.S;
    B.S = B.S_var;
    int rc = mixed_inverse_factor(B, SEL_L, true);
    if (rc == INLA_OK) {
      launch_rowsumsq_wk_df(B.d_slots, B.n, B.max_n, B.st);
      if (B.max_k > 0 && (rc = mixed_var_constraint(B)) == INLA_OK)
        launch_var_finish(B.d_slots, B.n, B.max_n, B.st);
    }
    B.S = S_keep;
    return rc;
  }
  trtri64(B, SEL_L, DST_WK);
  launch_colsumsq_wk(B.d_slots, B.n, B.max_t, B.st);
  if (B.max_k > 0) {
    launch_zt_w(B.d_slots, B.n, B.max_tk, B.max_t, B.st);
    for (int kt = 0; kt < B.max_tk; ++kt) launch_fwd_s_rhs_step(B.d_slots, B.n, kt, B.max_tk, B.max_t, B.st);
    launch_colsumsq_gt(B.d_slots, B.n, B.max_tk, B.max_t, B.st);
    launch_var_finish(B.d_slots, B.n, B.max_n, B.st);
  }
  return INLA_OK;
}

static void sync_active(Batch& B) {
  cudaMemcpyAsync(B.d_slots, B.h.data(), sizeof(Slot) * B.n, cudaMemcpyHostToDevice, B.st);
}

static int read_outputs(Batch& B, std::vector<double>& out, std::vector<int32_t>& info, int* err_flag = nullptr) {
  out.resize((size_t)B.n * SLOT_NOUT);
  info.resize((size_t)B.n * 2);
  for (int i = 0; i < B.n; ++i) {
    cudaMemcpyAsync(&out[(size_t)i * SLOT_NOUT], B.h[i].out, SLOT_NOUT * 8, cudaMemcpyDeviceToHost, B.st);
    cudaMemcpyAsync(&info[(size_t)i * 2], B.h[i].info, 8, cudaMemcpyDeviceToHost, B.st);
  }
  int e = 0;
  if (B.err) cudaMemcpyAsync(&e, B.err, 4, cudaMemcpyDeviceToHost, B.st);
  INLA_CUDA_TRY(cudaStreamSynchronize(B.st));
  INLA_CUDA_TRY(cudaGetLastError());
  if (err_flag) *err_flag = e;
  return e ? INLA_E_TIMEOUT : INLA_OK;
}

static void fail_slot(Batch& B, int* status, int i, int code) {
  if (status[i] == INLA_OK) status[i] = code;
  B.h[i].active = 0;
}

// objective f(x) = sum log p(y|eta) - 1/2 x^T Q_p x (with the constant of log y!)
static double objective(const ModelDev& md, const double* out) {
  double f = out[OUT_LOGLIK] - 0.5 * out[OUT_QUAD];
  if (md.likelihood == INLA_LIK_POISSON) f -= md.lgamma_sum;
  return f;
}

// Slots [lo, hi) of a batch as a batch of their own: the strided routines see them as slots
// 0 .. hi - lo - 1 (slot lo's matrices are the view's base; the slice workspaces are shared and
// their slot numbering restarts).  Host-side changes to the view's slots are copied back by
// copy_back.
static Batch view_of(const Batch& B, int lo, int hi) {
  Batch V = B;
  V.d_slots = B.d_slots + lo;
  V.h.assign(B.h.begin() + lo, B.h.begin() + hi);
  V.n = hi - lo;
  return V;
}
static void copy_back(Batch& B, const Batch& V, int lo) {
  for (int i = 0; i < V.n; ++i) B.h[lo + i] = V.h[i];
}
// the factor of Q* and the constraint Schur matrices a slot's solves read
static void set_factor_ptrs(Slot& dst, const Slot& src) {
  dst.L = src.L;
  dst.Linv = src.Linv;
  dst.Z = src.Z;
  dst.S = src.S;
  dst.SLinv = src.SLinv;
}

// Newton iterations of Algorithm 1 over the slots of V (all active on entry), each step
// x_new = x + Q*(x)^-1 grad f(x), kriged when constrained, halved while the objective falls.
// start_shared: the slots start from the x the caller set, with the factor (and Schur matrices)
// their pointers name -- another point's final factor, read only -- and keep it while the steps
// shrink at least 4x per iteration (modified Newton: the gradient is exact, so the fixed point
// is still the mode); `own` then holds their own matrix pointers, restored before the first
// factorisation of their own.
// wls_start: the slots start instead from the solution of a weighted least-squares system
// Q_p + A^T W A (Poisson: W = diag(y + 1/2) with the working response log(y + 1/2) - offset;
// Gaussian: its exact Newton system) -- one factorisation, kept as the first iterations'
// factor while it serves (start_shared), which near the mode approximates the Hessian
// A^T diag(exp(eta)) A + Q_p well: fewer Newton factorisations than from x = 0.
static int newton_phase(Batch& V, const ModelDev* const* models, const inla_opts& o, int* status, int* iters,
                        int* converged, int* d_flags, bool start_shared, const std::vector<Slot>& own,
                        bool wls_start = false, bool* handed_over = nullptr) {
  const int NB = V.n;
  std::vector<double> out;
  std::vector<int32_t> info;
  V.S = V.S_newton;
  if (!start_shared) launch_zero_vec(V.d_slots, NB, 0, V.max_n, V.st);
  if (wls_start) {
    launch_wls_start(V.d_slots, NB, V.max_m, V.max_n, V.st);
    op_assemble_q(V);
    launch_gradient(V.d_slots, NB, V.max_n, V.st);
    INLA_TRY(op_potrf(V, SEL_L));
    INLA_TRY(solve_llt(V, SEL_L, V_G, V_T2, V_G));
    launch_newton_xu(V.d_slots, NB, V.max_n, V.st);  // xn = 0 + g
    if (V.max_k > 0) {
      INLA_TRY(op_schur(V));
      launch_cx(V.d_slots, NB, V.max_k, V.st);
      INLA_TRY(solve_llt(V, SEL_S, V_KV1, V_KV2, V_KV1));
      if (V.mixed) launch_z_gemv_df(V.d_slots, NB, V.max_n, V.st);
      else launch_z_gemv(V.d_slots, NB, V.max_n, V.st);
      INLA_TRY(solve_lt(V, SEL_L, V_T2, V_G));
      launch_krige_apply(V.d_slots, NB, V.max_n, V.st);
    }
    launch_step_norm(V.d_slots, NB, V.max_n, V.st);
    launch_accept(V.d_slots, NB, V.max_n, V.st);
    INLA_TRY(read_outputs(V, out, info));
    double mx = 0.0;
    for (int i = 0; i < NB; ++i) {
      if (V.h[i].active && (info[2 * i] & INFO_NOT_SPD)) fail_slot(V, status, i, INLA_E_NOT_SPD);
      if (V.h[i].active) mx = std::max(mx, out[(size_t)i * SLOT_NOUT + OUT_STEP]);
    }
    g_newton_trace.push_back({mx, 1});
    sync_active(V);
    start_shared = true;  // the start system's factor serves the first iterations
  }
  launch_eval_lik(V.d_slots, NB, 0, V.max_m, V.st);
  op_qp_gemv(V, 0);
  INLA_TRY(read_outputs(V, out, info));
  std::vector<double> f_old(NB);
  for (int i = 0; i < NB; ++i) f_old[i] = objective(*models[i], &out[(size_t)i * SLOT_NOUT]);
  std::vector<int> flags(NB, 0);
  int rc = INLA_OK;
  double last_step = 1e300;
  bool reuse_ok = true;
  bool shared = start_shared;
  int it_own = start_shared ? -1 : 1;  // iteration of the first factorisation of the slots' own
  for (int it = 1; it <= o.newton_max && rc == INLA_OK; ++it) {
    int nact = 0;
    for (int i = 0; i < NB; ++i) nact += V.h[i].active;
    if (nact == 0) break;
    // Q* = Q_p + A^T D A at x ; gradient ; factor ; Newton direction.  The mixed path reuses the
    // last factor once the steps are small and shrinking fast (modified Newton): the gradient
    // stays exact, so the fixed point is unchanged; a reused step that does not shrink the step
    // by 4x forces a fresh factor at the next iteration.
    bool refactor;
    if (shared) {
      refactor = !reuse_ok;
      if (refactor) {  // convergence slowed: the slots factor their own Q* from here on
        for (int i = 0; i < NB; ++i) set_factor_ptrs(V.h[i], own[i]);
        sync_active(V);
        shared = false;
        it_own = it;
      }
    } else {
      refactor = !V.mixed || it - it_own < 2 || last_step > o.reuse_below || !reuse_ok;
      // hand-over: the slots' own factor will now be kept (modified Newton near the mode), so the
      // caller can run the remaining iterations together with other points that share it
      if (handed_over && !refactor && it_own > 0) {
        *handed_over = true;
        break;
      }
    }
    for (int i = 0; i < NB; ++i)
      if (V.h[i].active) iters[i] = it;
    if (refactor) op_assemble_q(V);
    launch_gradient(V.d_slots, NB, V.max_n, V.st);
    if ((rc = debug_check(V.st, "newton assemble")) != INLA_OK) break;
    if (refactor && (rc = op_potrf(V, SEL_L)) != INLA_OK) break;
    if ((rc = debug_check(V.st, "newton potrf")) != INLA_OK) break;
    if ((rc = solve_llt(V, SEL_L, V_G, V_T2, V_G)) != INLA_OK) break;
    if ((rc = debug_check(V.st, "newton solve")) != INLA_OK) break;
    launch_newton_xu(V.d_slots, NB, V.max_n, V.st);
    if (V.max_k > 0) {
      if (refactor && (rc = op_schur(V)) != INLA_OK) break;
      launch_cx(V.d_slots, NB, V.max_k, V.st);
      if ((rc = solve_llt(V, SEL_S, V_KV1, V_KV2, V_KV1)) != INLA_OK) break;
      if (V.mixed) launch_z_gemv_df(V.d_slots, NB, V.max_n, V.st);
      else launch_z_gemv(V.d_slots, NB, V.max_n, V.st);
      if ((rc = solve_lt(V, SEL_L, V_T2, V_G)) != INLA_OK) break;
      launch_krige_apply(V.d_slots, NB, V.max_n, V.st);
      if ((rc = debug_check(V.st, "newton kriging")) != INLA_OK) break;
    }
    launch_eval_lik(V.d_slots, NB, 1, V.max_m, V.st);
    op_qp_gemv(V, 1);
    launch_step_norm(V.d_slots, NB, V.max_n, V.st);
    if ((rc = read_outputs(V, out, info)) != INLA_OK) break;
    for (int i = 0; i < NB; ++i)
      if (V.h[i].active && (info[2 * i] & INFO_NOT_SPD)) fail_slot(V, status, i, INLA_E_NOT_SPD);
    // step halving while the objective decreases
    for (int h = 0; h < 30; ++h) {
      int any = 0;
      for (int i = 0; i < NB; ++i) {
        flags[i] = 0;
        if (!V.h[i].active || models[i]->likelihood == INLA_LIK_GAUSSIAN) continue;
        const double fn = objective(*models[i], &out[(size_t)i * SLOT_NOUT]);
        if (fn < f_old[i] - 1e-10 * (1.0 + std::fabs(f_old[i]))) flags[i] = any = 1;
      }
      if (!any) break;
      cudaMemcpyAsync(d_flags, flags.data(), sizeof(int) * NB, cudaMemcpyHostToDevice, V.st);
      launch_halve(V.d_slots, NB, d_flags, V.max_n, V.st);
      launch_eval_lik(V.d_slots, NB, 1, V.max_m, V.st);
      op_qp_gemv(V, 1);
      launch_step_norm(V.d_slots, NB, V.max_n, V.st);
      if ((rc = read_outputs(V, out, info)) != INLA_OK) break;
    }
    if (rc != INLA_OK) break;
    launch_accept(V.d_slots, NB, V.max_n, V.st);
    {
      double mx = 0.0;
      for (int i = 0; i < NB; ++i)
        if (V.h[i].active) mx = std::max(mx, out[(size_t)i * SLOT_NOUT + OUT_STEP]);
      reuse_ok = (refactor && !shared) || mx < o.reuse_shrink * last_step;
      last_step = mx;
      g_newton_trace.push_back({mx, refactor ? 1 : 0});
    }
    for (int i = 0; i < NB; ++i) {
      if (!V.h[i].active) continue;
      const double* oi = &out[(size_t)i * SLOT_NOUT];
      f_old[i] = objective(*models[i], oi);
      if (!std::isfinite(f_old[i])) {
        fail_slot(V, status, i, INLA_E_NO_CONVERGENCE);
        continue;
      }
      if (models[i]->likelihood == INLA_LIK_GAUSSIAN || oi[OUT_STEP] <= o.newton_tol) {
        converged[i] = 1;
        V.h[i].active = 0;
      }
    }
    sync_active(V);
  }
  if (shared) {  // the slots name their own matrices again
    for (int i = 0; i < NB; ++i) set_factor_ptrs(V.h[i], own[i]);
    sync_active(V);
  }
  return rc;
}

// Q* at the mode and its factor (and, with constraints, Z = L^-1 C^T and the factor of
// S = Z^T Z) for the slots of V that are still healthy; the likelihood and x^T Q_p x at x.
static int final_factor(Batch& V) {
  V.S = V.S_exact;
  sync_active(V);
  launch_eval_lik(V.d_slots, V.n, 0, V.max_m, V.st);
  op_qp_gemv(V, 0);
  op_assemble_q(V);
  INLA_TRY(op_potrf(V, SEL_L));
  INLA_TRY(debug_check(V.st, "final potrf"));
  if (V.max_k > 0) INLA_TRY(op_schur(V));
  return debug_check(V.st, "final schur");
}

// One batch: prior precision of every point; Newton to the mode; the factor at the mode;
// log-determinants, variances and log pi~.  Slots [0, nlead) run Newton from x = 0.  Slots
// [nlead, NB) ("followers", mixed path only) each name an earlier slot anchor_of[i] of the same
// model: they start from that slot's mode with its final factor (see newton_phase), which for the
// points of one finite-difference stencil -- theta apart by the FD step -- converges in a few
// cheap iterations instead of a Newton factorisation per step.
// Variational Bayes correction of the mean (Appendix A.2.2, Algorithm 2; see vb.cu) for the
// healthy slots, in place on x: sigma_i^2 of the linear predictor from the inverse factor held
// in Wk, then steps mu += Q*^-1 (-c) with c = A^T I'(0) + Q_p mu until max |step| <= 1e-8.
// The variances (t1) are set aside while t1 serves the steps.
static int vb_correction(Batch& B, const inla_opts& o, int* status) {
  (void)o;
  const int NB = B.n;
  std::vector<double> out;
  std::vector<int32_t> info;
  for (int i = 0; i < NB; ++i)
    if (B.h[i].active) cudaMemcpyAsync(B.h[i].vsave, B.h[i].t1, sizeof(double) * B.h[i].n_pad, cudaMemcpyDeviceToDevice, B.st);
  launch_vb_prepare(B.d_slots, NB, B.mixed ? 1 : 0, B.max_pairs, B.max_m, B.st);
  std::vector<int> done(NB, 0);
  constexpr int kVbMax = 50;
  constexpr double kVbTol = 1e-8;
  int rc = INLA_OK;
  for (int it = 0; it < kVbMax; ++it) {
    int nact = 0;
    for (int i = 0; i < NB; ++i) nact += B.h[i].active;
    if (nact == 0) break;
    if ((rc = launch_vb_terms(B.d_slots, NB, B.max_m, B.st)) != INLA_OK) break;
    op_qp_gemv(B, 0);                                   // t1 = Q_p mu
    launch_gradient(B.d_slots, NB, B.max_n, B.st);      // g = A^T (-I') - Q_p mu = -c
    if ((rc = solve_llt(B, SEL_L, V_G, V_T2, V_G)) != INLA_OK) break;
    launch_newton_xu(B.d_slots, NB, B.max_n, B.st);     // xn = mu + step
    launch_step_norm(B.d_slots, NB, B.max_n, B.st);
    launch_accept(B.d_slots, NB, B.max_n, B.st);
    if ((rc = read_outputs(B, out, info)) != INLA_OK) break;
    for (int i = 0; i < NB; ++i)
      if (B.h[i].active && out[(size_t)i * SLOT_NOUT + OUT_STEP] <= kVbTol) {
        done[i] = 1;
        B.h[i].active = 0;
      }
    sync_active(B);
  }
  for (int i = 0; i < NB; ++i) {
    if (B.h[i].active && !done[i] && status[i] == INLA_OK) status[i] = INLA_E_NO_CONVERGENCE;
    B.h[i].active = status[i] == INLA_OK;
  }
  sync_active(B);
  for (int i = 0; i < NB; ++i)
    if (B.h[i].active) cudaMemcpyAsync(B.h[i].t1, B.h[i].vsave, sizeof(double) * B.h[i].n_pad, cudaMemcpyDeviceToDevice, B.st);
  return rc;
}

static int run_batch(Batch& B, const std::vector<const ModelDev*>& models, const inla_opts& o, bool want_var,
                     std::vector<int>& status, std::vector<int>& iters, int nlead, const std::vector<int>& anchor_of) {
  const bool vb = (o.flags & INLA_OPT_VB_MEAN) != 0;
  const int NB = B.n;
  std::vector<double> out;
  std::vector<int32_t> info;
  status.assign(NB, INLA_OK);
  iters.assign(NB, 0);
  if (B.err) cudaMemsetAsync(B.err, 0, 4, B.st);
  for (int i = 0; i < NB; ++i) {
    cudaMemsetAsync(B.h[i].out, 0, SLOT_NOUT * 8, B.st);
    const int32_t init_info[2] = {0, INT_MAX};
    cudaMemcpyAsync(B.h[i].info, init_info, 8, cudaMemcpyHostToDevice, B.st);
    B.h[i].active = 1;
  }
  sync_active(B);
  // ---------------- prior precision ----------------
  prof_phase("prior");
  B.S = B.S_prior;
  launch_theta_prior(B.d_slots, NB, B.st);
  for (int i = 0; i < NB; ++i) cudaMemsetAsync(B.h[i].Qp, 0, (size_t)B.h[i].n_pad * B.h[i].n_pad * 8, B.st);
  INLA_TRY(debug_check(B.st, "prior start"));
  if (B.max_td > 0) INLA_TRY(op_prior_dense(B));
  INLA_TRY(debug_check(B.st, "prior dense"));
  if (B.mixed) launch_prior_entries_df(B.d_slots, NB, B.max_entries, B.st);
  else launch_prior_entries(B.d_slots, NB, B.max_entries, B.st);
  launch_mirror_qp(B.d_slots, NB, B.max_t, B.st);
  launch_prior_logdet(B.d_slots, NB, B.st);
  INLA_TRY(read_outputs(B, out, info));
  for (int i = 0; i < NB; ++i)
    if (info[2 * i] & INFO_NOT_SPD) fail_slot(B, status.data(), i, INLA_E_NOT_SPD);
  sync_active(B);
  int* d_flags = nullptr;
  INLA_CUDA_TRY(cudaMallocAsync((void**)&d_flags, sizeof(int) * NB, B.st));
  std::vector<int> converged(NB, 0);
  g_newton_trace.clear();
  int rc = INLA_OK;
  // ---------------- Newton, leaders ----------------
  // With followers, the leaders stop as soon as they would keep their factor for the remaining
  // (modified Newton) iterations: those then run in one batch with the followers, which start from
  // their anchor's iterate with its factor, and every mode is factored in one batched call.
  prof_phase("newton_lead");
  const bool followers = nlead < NB;
  bool handed = false;
  {
    Batch V = view_of(B, 0, nlead);
    std::vector<Slot> own(V.h);
    rc = newton_phase(V, models.data(), o, status.data(), iters.data(), converged.data(), d_flags, false, own,
                      V.mixed && !(o.flags & INLA_OPT_NO_SHARED_START), followers && V.mixed ? &handed : nullptr);
    copy_back(B, V, 0);
  }
  // a point that failed or did not converge leaves the rest of the evaluation
  auto settle = [&](int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      if (status[i] == INLA_OK && !converged[i]) status[i] = INLA_E_NO_CONVERGENCE;
      B.h[i].active = status[i] == INLA_OK;
    }
  };
  if (rc == INLA_OK && followers && handed) {
    // the leaders stopped with a factor of their own near their modes: they finish their
    // (modified Newton) iterations in one batch with the followers, which start from their
    // anchor's iterate with that factor; then every mode is factored in one batched call
    for (int i = 0; i < nlead; ++i) B.h[i].active = status[i] == INLA_OK && !converged[i];
    sync_active(B);
    bool anchors_ok = true;
    for (int i = nlead; i < NB; ++i) anchors_ok = anchors_ok && status[anchor_of[i]] == INLA_OK;
    // the leaders' iterations before the hand-over, added to those after it
    std::vector<int> iters_lead(iters.begin(), iters.begin() + nlead), cont(nlead);
    for (int i = 0; i < nlead; ++i) cont[i] = B.h[i].active;
    if (anchors_ok) {
      std::vector<Slot> own(B.h);
      for (int i = nlead; i < NB; ++i) {
        if (!B.h[i].active) continue;
        Slot& f = B.h[i];
        const Slot& a = B.h[anchor_of[i]];
        cudaMemcpyAsync(f.x, a.x, sizeof(double) * f.n_pad, cudaMemcpyDeviceToDevice, B.st);
        set_factor_ptrs(f, a);
      }
      sync_active(B);
      prof_phase("newton_follow");
      rc = newton_phase(B, models.data(), o, status.data(), iters.data(), converged.data(), d_flags, true, own);
    } else {
      // an anchor failed: the leaders finish on their own, the followers start from zero
      {
        Batch V = view_of(B, 0, nlead);
        std::vector<Slot> own(V.h);
        rc = newton_phase(V, models.data(), o, status.data(), iters.data(), converged.data(), d_flags, true, own);
        copy_back(B, V, 0);
      }
      if (rc == INLA_OK) {
        Batch F = view_of(B, nlead, NB);
        std::vector<Slot> own(F.h);
        prof_phase("newton_follow");
        rc = newton_phase(F, models.data() + nlead, o, status.data() + nlead, iters.data() + nlead,
                          converged.data() + nlead, d_flags, false, own);
        copy_back(B, F, nlead);
      }
    }
    for (int i = 0; i < nlead; ++i)
      if (cont[i]) iters[i] += iters_lead[i];
    if (rc == INLA_OK) {
      settle(0, NB);
      prof_phase("factor_modes");
      rc = final_factor(B);
    }
  } else if (rc == INLA_OK && followers) {
    // the leaders converged on their start-system factor: their factor at the mode first, then
    // the followers from their anchor's mode with that factor
    settle(0, nlead);
    prof_phase("factor_lead");
    Batch V = view_of(B, 0, nlead);
    rc = final_factor(V);
    copy_back(B, V, 0);
    if (rc == INLA_OK) {
      bool anchors_ok = true;
      for (int i = nlead; i < NB; ++i) anchors_ok = anchors_ok && B.h[anchor_of[i]].active;
      Batch F = view_of(B, nlead, NB);
      std::vector<Slot> own(F.h);
      for (int i = nlead; i < NB; ++i) {
        if (!B.h[i].active) continue;
        Slot& f = F.h[i - nlead];
        if (anchors_ok) {
          const Slot& a = B.h[anchor_of[i]];
          cudaMemcpyAsync(f.x, a.x, sizeof(double) * f.n_pad, cudaMemcpyDeviceToDevice, B.st);
          set_factor_ptrs(f, a);
        }
      }
      sync_active(F);
      prof_phase("newton_follow");
      rc = newton_phase(F, models.data() + nlead, o, status.data() + nlead, iters.data() + nlead,
                        converged.data() + nlead, d_flags, anchors_ok, own);
      copy_back(B, F, nlead);
      if (rc == INLA_OK) {
        settle(nlead, NB);
        prof_phase("factor_follow");
        Batch G = view_of(B, nlead, NB);
        rc = final_factor(G);
        copy_back(B, G, nlead);
      }
    }
  } else if (rc == INLA_OK) {
    settle(0, nlead);
    prof_phase("factor_lead");
    rc = final_factor(B);
  }
  cudaFreeAsync(d_flags, B.st);
  if (rc != INLA_OK) return rc;
  sync_active(B);
  // ---------------- at the modes: log-determinants, variances, log pi~ ----------------
  prof_phase("logdet_variances");
  B.S = B.S_exact;
  op_logdet(B, SEL_L, OUT_LOGDET_Q);
  if (B.max_k > 0) op_logdet(B, SEL_S, OUT_LOGDET_S);
  if (o.flags & INLA_OPT_WOODBURY_VAR) {
    if (want_var) INLA_TRY(mixed_woodbury_variances(B));
  } else if (want_var || vb) {
    INLA_TRY(op_variances(B));
  }
  INLA_TRY(debug_check(B.st, "final variances"));
  launch_assemble(B.d_slots, NB, B.st);
  INLA_TRY(read_outputs(B, out, info));
  for (int i = 0; i < NB; ++i)
    if (B.h[i].active && (info[2 * i] & INFO_NOT_SPD)) fail_slot(B, status.data(), i, INLA_E_NOT_SPD);
  if (vb) {
    sync_active(B);
    prof_phase("vb_mean");
    INLA_TRY(vb_correction(B, o, status.data()));
  }
  return INLA_OK;
}

// log-determinant of a host SPD matrix (k x k, k a multiple of TB) on the device, FP64
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
    B.mixed = false;
    potrf64(B, SEL_S);
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

// -------------------------------------------------------------------------------------
// one group of points with identical model shapes
// -------------------------------------------------------------------------------------
struct Layout {
  int np, ndp, kp, m, S;
  bool mixed, want_var;
  int64_t npairs = 0;   // variational Bayes: the largest A^T A pair count of the group
  bool vb = false;
};

// carve the group's workspace (uniform strides); returns the bytes used
static size_t carve_group(Carve& cv, const Layout& L, int G, Batch& B, std::vector<Slot>& h) {
  const size_t np = L.np, kp = L.kp, ndp = std::max(L.ndp, 1), m = std::max(L.m, 1);
  B.np = L.np;
  B.ndp = L.ndp;
  B.kp = L.kp;
  B.mat_stride = (int64_t)np * np;
  B.z_stride = (int64_t)np * kp;
  B.s_stride = (int64_t)kp * kp;
  B.linv_stride = (int64_t)np * TB;
  B.wd_stride = (int64_t)ndp * TB;
  B.slinv_stride = (int64_t)kp * TB;
  double* Qp = cv.take<double>(G * np * np);
  double* Lm = cv.take<double>(G * np * np);
  double* Wk = cv.take<double>(G * np * np);
  double* Linv = cv.take<double>(G * np * TB);
  double* Wd = cv.take<double>(G * ndp * TB);
  double *Z = nullptr, *S = nullptr, *SLinv = nullptr, *kv1 = nullptr, *kv2 = nullptr;
  if (kp) {
    Z = cv.take<double>(G * np * kp);
    S = cv.take<double>(G * kp * kp);
    SLinv = cv.take<double>(G * kp * TB);
    kv1 = cv.take<double>(G * kp);
    kv2 = cv.take<double>(G * kp);
  }
  double* vecs = cv.take<double>(G * np * 7);
  double* mvecs = cv.take<double>(G * m * (L.vb ? 3 : 2));
  double* pcov = L.vb ? cv.take<double>(G * std::max<int64_t>(L.npairs, 1)) : nullptr;
  double* red = cv.take<double>(G * 256);
  double* qpart = L.mixed ? cv.take<double>(G * (np / TB) * np) : nullptr;
  double* outs = cv.take<double>(G * SLOT_NOUT);
  int32_t* infos = cv.take<int32_t>(G * 2);
  B.mixed = L.mixed;
  B.S = L.S;
  B.PA = B.PB = B.PBIG = nullptr;
  B.EA = B.EB = B.EBIG = nullptr;
  B.err = cv.take<int32_t>(1);
  B.flags = cv.take<int32_t>(G * (np / TB + 1));
  if (L.mixed) {
    const int64_t nch = (int64_t)(np + OZ_CHUNK - 1) / OZ_CHUNK;
    B.pa_cap = (int64_t)L.S * np * std::max<size_t>(MIXED_NB_MAX, kp);
    B.pb_cap = (int64_t)L.S * np * MIXED_NB_MAX;
    B.pbig_cap = (int64_t)L.S * np * np;
    B.ea_cap = nch * (int64_t)std::max<size_t>(np, kp) + np;
    B.eb_cap = nch * (int64_t)np + np;
    B.ebig_cap = nch * (int64_t)np;
    B.PA = cv.take<uint16_t>(G * B.pa_cap);
    B.PB = cv.take<uint16_t>(G * B.pb_cap);
    B.PBIG = cv.take<uint16_t>(G * B.pbig_cap);
    B.EA = cv.take<int32_t>(G * B.ea_cap);
    B.EB = cv.take<int32_t>(G * B.eb_cap);
    B.EBIG = cv.take<int32_t>(G * B.ebig_cap);
  }
  h.resize(G);
  for (int i = 0; i < G; ++i) {
    Slot& s = h[i];
    std::memset(&s, 0, sizeof(s));
    s.Qp = Qp ? Qp + i * np * np : nullptr;
    s.L = Lm ? Lm + i * np * np : nullptr;
    s.Wk = Wk ? Wk + i * np * np : nullptr;
    s.Linv = Linv ? Linv + i * np * TB : nullptr;
    s.Wd = Wd ? Wd + i * ndp * TB : nullptr;
    if (kp && Z) {
      s.Z = Z + i * np * kp;
      s.S = S + i * kp * kp;
      s.SLinv = SLinv + i * kp * TB;
      s.kv1 = kv1 + i * kp;
      s.kv2 = kv2 + i * kp;
    }
    if (vecs) {
      double* v = vecs + i * np * 7;
      s.x = v;
      s.xn = v + np;
      s.g = v + 2 * np;
      s.t1 = v + 3 * np;
      s.t2 = v + 4 * np;
      s.vd = v + 5 * np;
      s.vsave = v + 6 * np;
      s.eta = mvecs + i * m * (L.vb ? 3 : 2);
      s.w = s.eta + m;
      if (L.vb) {
        s.etav = s.eta + 2 * m;
        s.pcov = pcov + i * std::max<int64_t>(L.npairs, 1);
      }
      s.red = red + i * 256;
      s.qpart = qpart ? qpart + (size_t)i * (np / TB) * np : nullptr;
      s.out = outs + i * SLOT_NOUT;
      s.info = infos + i * 2;
    }
  }
  return cv.off;
}

// A call without a stream runs on the library's own non-blocking stream of the device (CUDA graphs
// and side streams need a capturable stream; the legacy default stream is not one), ordered after
// the work queued on the legacy default stream before the call and before the work queued there
// after it (events both ways, on every return path).
namespace {
struct OwnStream {
  cudaStream_t st = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
};
OwnStream g_own_stream[64];
std::mutex g_own_mu;
class LegacyBridge {
 public:
  // the stream to run on: `requested`, or the device's own stream when it is NULL
  cudaStream_t begin(cudaStream_t requested) {
    if (requested) return requested;
    const int dev = current_device();
    if (dev < 0 || dev >= 64) return requested;
    std::lock_guard<std::mutex> lk(g_own_mu);
    OwnStream& r = g_own_stream[dev];
    if (!r.st) {
      OwnStream n;
      if (cudaStreamCreateWithFlags(&n.st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&n.in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&n.out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return requested;  // stays on the legacy stream
      }
      r = n;
    }
    if (cudaEventRecord(r.in, 0) != cudaSuccess || cudaStreamWaitEvent(r.st, r.in, 0) != cudaSuccess) {
      cudaGetLastError();
      return requested;
    }
    res_ = &r;
    return r.st;
  }
  ~LegacyBridge() {
    if (!res_) return;
    cudaEventRecord(res_->out, res_->st);
    cudaStreamWaitEvent(0, res_->out, 0);
  }

 private:
  OwnStream* res_ = nullptr;
};
}  // namespace

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
  if (o.spin_limit <= 0) o.spin_limit = (int64_t)1 << 26;
  if (!(o.reuse_below > 0)) o.reuse_below = 0.1;
  if (!(o.reuse_shrink > 0)) o.reuse_shrink = 0.25;
  if (o.reuse_shrink >= 1.0) return INLA_E_BADARG;
  if (o.precision != INLA_FP64 && o.precision != INLA_MIXED) return INLA_E_BADARG;
  const bool mixed = o.precision == INLA_MIXED;
  const int S_exact = mixed ? (o.slices == 0 ? 5 : o.slices) : 0;
  const int S_newton = mixed ? (o.newton_slices == 0 ? std::min(4, S_exact) : o.newton_slices) : 0;
  const int S_prior = mixed ? (o.prior_slices == 0 ? S_exact : o.prior_slices) : 0;
  const int S_var = mixed ? (o.var_slices == 0 ? S_exact : o.var_slices) : 0;
  const int S_gram = mixed ? (o.gram_slices == 0 ? S_prior : o.gram_slices) : 0;
  if (mixed && (S_exact < 2 || S_exact > OZ_MAX_S || S_newton < 2 || S_newton > OZ_MAX_S || S_prior < 2 ||
                S_prior > OZ_MAX_S || S_var < 2 || S_var > OZ_MAX_S || S_gram < 2 || S_gram > OZ_MAX_S))
    return INLA_E_BADARG;
  const int S = std::max(std::max(std::max(S_exact, S_newton), std::max(S_prior, S_var)), S_gram);  // workspace
  LegacyBridge bridge;
  cudaStream_t st = bridge.begin(static_cast<cudaStream_t>(o.stream));
  prof_set_stream(st);
  const bool dev_out = (o.flags & INLA_OPT_DEVICE_OUT) != 0;
  const bool want_var = var != nullptr;
  const bool vb = (o.flags & INLA_OPT_VB_MEAN) != 0;
  int theta_dim = -1;
  std::vector<int> mi_of(B_);
  for (int b = 0; b < B_; ++b) {
    const int mi = model_of_theta ? model_of_theta[b] : 0;
    if (mi < 0 || mi >= nmodels || !models[mi]) return INLA_E_BADARG;
    mi_of[b] = mi;
    if (theta_dim >= 0 && theta_dim != models[mi]->d.theta_dim) return INLA_E_BADARG;
    theta_dim = models[mi]->d.theta_dim;
  }
  for (int64_t i = 0; i < (int64_t)B_ * theta_dim; ++i)
    if (!std::isfinite(thetas[i])) return INLA_E_BADARG;
  if (vb)
    for (int b = 0; b < B_; ++b)
      if (models[mi_of[b]]->d.k > 0) return INLA_E_UNSUPPORTED;  // variational Bayes: no constraints
  if (o.flags & INLA_OPT_WOODBURY_VAR) {
    // the Moore-Penrose route: mixed path, its m x m system inside the slot's n_pad x n_pad
    // buffers, and not with the variational Bayes correction (which needs the inverse factor)
    if (!mixed || vb) return INLA_E_UNSUPPORTED;
    for (int b = 0; b < B_; ++b) {
      const ModelDev& d = models[mi_of[b]]->d;
      if (round_up(std::max(d.m, 1), PAD) > d.n_pad) return INLA_E_UNSUPPORTED;
    }
  }
  int device = 0;
  INLA_CUDA_TRY(cudaGetDevice(&device));
  std::lock_guard<std::mutex> lock(g_mutex);
  // group the points by model shape
  std::map<std::tuple<int, int, int, int, int, int>, std::vector<int>> groups;
  for (int b = 0; b < B_; ++b) {
    const ModelDev& d = models[mi_of[b]]->d;
    groups[std::make_tuple(d.n_pad, d.nd_pad, d.k_pad, d.m, d.nd, d.nd_off)].push_back(b);
  }
  // workspace: the largest group, plus model structs, permutations, gather buffer
  size_t need = 0;
  for (auto& kv : groups) {
    const ModelDev& d = models[mi_of[kv.second[0]]]->d;
    Layout L{d.n_pad, d.nd_pad, d.k_pad, d.m, S, mixed, want_var};
    L.vb = vb;
    for (int b : kv.second) L.npairs = std::max(L.npairs, models[mi_of[b]]->d.npairs);
    Carve cv(nullptr);
    Batch Bt;
    std::vector<Slot> h;
    size_t b = carve_group(cv, L, (int)kv.second.size(), Bt, h);
    b += sizeof(Slot) * kv.second.size() + 4096;
    need = std::max(need, b);
  }
  int max_np = 0;
  size_t extra = 0;
  for (int mi = 0; mi < nmodels; ++mi) {
    extra += sizeof(ModelDev) + (size_t)models[mi]->d.n * sizeof(int32_t) + 1024;
    max_np = std::max(max_np, models[mi]->d.n_pad);
  }
  extra += (size_t)max_np * sizeof(double) + 1024;
  need = (size_t)round_up((int64_t)need, 256);  // the fixed part starts on a 256-byte boundary
  const size_t bytes = need + extra;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (bytes > (size_t)(0.95 * (double)(free_b + (g_arena.device == device ? g_arena.size : 0)))) return INLA_E_NOMEM;
  INLA_TRY(arena_reserve(bytes, device));
  // fixed part at the end of the arena: model structs, permutations, gather buffer
  Carve cfix(static_cast<char*>(g_arena.base) + need);
  std::vector<ModelDev*> d_models(nmodels, nullptr);
  std::vector<int32_t*> d_perm(nmodels, nullptr);
  for (int mi = 0; mi < nmodels; ++mi) {
    d_models[mi] = cfix.take<ModelDev>(1);
    cudaMemcpyAsync(d_models[mi], &models[mi]->d, sizeof(ModelDev), cudaMemcpyHostToDevice, st);
    d_perm[mi] = cfix.take<int32_t>(models[mi]->d.n);
    cudaMemcpyAsync(d_perm[mi], models[mi]->perm.data(), sizeof(int32_t) * models[mi]->d.n, cudaMemcpyHostToDevice, st);
  }
  double* d_gather = cfix.take<double>(max_np);
  const bool share = mixed && !(o.flags & INLA_OPT_NO_SHARED_START);
  for (auto& kv : groups) {
    // Order the group's points: leaders (Newton from x = 0) first, then followers (the later
    // points of a Poisson model with several points in the group: they start from the first
    // point's mode and final factor).  anchor_of: the leader slot of each follower slot.
    std::vector<int> idx;
    std::vector<int> anchor_of;
    int nlead = 0;
    {
      std::map<int, int> first_of_model;  // model index -> its first point's position in idx
      std::vector<int> followers;
      for (int b : kv.second) {
        const int mi = mi_of[b];
        const bool poisson = models[mi]->d.likelihood == INLA_LIK_POISSON;
        if (share && poisson && first_of_model.count(mi)) {
          followers.push_back(b);
        } else {
          if (!first_of_model.count(mi)) first_of_model[mi] = (int)idx.size();
          idx.push_back(b);
        }
      }
      nlead = (int)idx.size();
      anchor_of.assign(nlead, -1);
      for (int b : followers) {
        idx.push_back(b);
        anchor_of.push_back(first_of_model[mi_of[b]]);
      }
    }
    const int G = (int)idx.size();
    const ModelDev& d0 = models[mi_of[idx[0]]]->d;
    Layout L{d0.n_pad, d0.nd_pad, d0.k_pad, d0.m, S, mixed, want_var};
    L.vb = vb;
    for (int b : idx) L.npairs = std::max(L.npairs, models[mi_of[b]]->d.npairs);
    Carve cv(g_arena.base);
    Batch Bt;
    carve_group(cv, L, G, Bt, Bt.h);
    Bt.d_slots = cv.take<Slot>(G);
    Bt.n = G;
    Bt.st = st;
    Bt.spin_limit = o.spin_limit;
    Bt.S_exact = S_exact;
    Bt.S_newton = S_newton;
    Bt.S_prior = S_prior;
    Bt.S_var = S_var;
    Bt.S_gram = S_gram;
    Bt.max_t = d0.n_pad / TB;
    Bt.max_td = d0.nd_pad / TB;
    Bt.max_tk = d0.k_pad / TB;
    Bt.max_m = d0.m;
    Bt.max_n = d0.n_pad;
    Bt.max_k = d0.k_pad;
    Bt.max_entries = 0;
    Bt.max_pairs = 0;
    std::vector<const ModelDev*> mlist(G);
    for (int g = 0; g < G; ++g) {
      const int b = idx[g];
      const ModelDev& d = models[mi_of[b]]->d;
      mlist[g] = &d;
      Slot& s = Bt.h[g];
      s.md = d_models[mi_of[b]];
      s.n_pad = d.n_pad;
      s.n = d.n;
      s.m = d.m;
      s.k = d.k;
      s.k_pad = d.k_pad;
      s.nd = d.nd;
      s.nd_pad = d.nd_pad;
      s.nd_off = d.nd_off;
      s.aux_n = (int32_t)round_up(std::max(d.m, 1), PAD);
      s.active = 1;
      for (int t = 0; t < theta_dim; ++t) s.theta[t] = thetas[(size_t)b * theta_dim + t];
      Bt.max_entries = std::max(Bt.max_entries, d.nentries);
      Bt.max_pairs = std::max(Bt.max_pairs, d.npairs);
    }
    if (mixed) {
      for (int g = 1; g < G; ++g)
        if (Bt.h[g].nd != Bt.h[0].nd) return INLA_E_UNSUPPORTED;
    }
    std::vector<int> status, iters;
    int rc = run_batch(Bt, mlist, o, want_var, status, iters, nlead, anchor_of);
    if (rc != INLA_OK) return rc;
    std::vector<double> out;
    std::vector<int32_t> info;
    for (int g = 0; g < G; ++g) Bt.h[g].active = 1;
    INLA_TRY(read_outputs(Bt, out, info));
    for (int g = 0; g < G; ++g) {
      const int b = idx[g];
      const int mi = mi_of[b];
      const int n = models[mi]->d.n;
      status_out[b] = status[g];
      if (iters_out) iters_out[b] = iters[g];
      log_post[b] = status[g] == INLA_OK ? out[(size_t)g * SLOT_NOUT + OUT_LOGPOST] : NAN;
      const double* srcs[2] = {Bt.h[g].x, Bt.h[g].t1};
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
  }
  INLA_CUDA_TRY(cudaGetLastError());
  return INLA_OK;
}

__global__ void k_gather(double* dst, const double* src, const int32_t* perm, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[perm[i]];
}
void launch_gather(double* dst, const double* src, const int32_t* perm, int n, cudaStream_t st) {
  count_launch("k_gather"), k_gather<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(dst, src, perm, n);
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
  o->reuse_below = 0.1;
  o->reuse_shrink = 0.25;
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

extern "C" const char* inla_test_debug_site(void) { return g_debug_site; }

extern "C" int64_t inla_test_launch_count(void) {
  const int64_t n = g_kernel_launches;
  g_kernel_launches = 0;
  return n;
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

extern "C" int inla_test_newton_trace(double* steps, int32_t* refactored, int32_t cap) {
  const int n = (int)g_newton_trace.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (steps) steps[i] = g_newton_trace[i].step;
    if (refactored) refactored[i] = g_newton_trace[i].refactored;
  }
  return n;
}

extern "C" int inla_test_outer_block(int32_t n_pad, int32_t slices) { return mixed_nb_choice(n_pad, slices); }
extern "C" int inla_test_inverse_block(int32_t n_pad, int32_t slices) { return mixed_inverse_nb_choice(n_pad, slices); }


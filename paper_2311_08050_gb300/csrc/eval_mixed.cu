// Blocked dense routines of the mixed path.  Matrices are double-float; every product with a
// non-trivial K runs on the Ozaki-split tensor-core GEMM; the 64 x 64 diagonal tiles are
// factored and inverted in double-float.  Two-level blocking: outer panels of NB columns (the
// trailing updates' K; C traffic n^3 / (3 NB) element updates per factorisation; NB tuned per
// matrix size for the Cholesky); inside a Cholesky panel, recursive halving down to 64-wide
// tile columns; 64-wide inner steps in the triangular solves.
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include "df64.cuh"
#include "mixed.h"

namespace inla {

namespace {

constexpr int IB = TB;    // inner block (64)

struct MRef {
  float2* base;       // slot-0 matrix
  int64_t stride;     // elements between slots
  int n, ld;
  double* linv;       // slot-0 diagonal-tile inverses (n x 64, double-float in FP64-sized cells)
  int64_t linv_stride;
  int sel;
};

MRef mref(const Batch& B, int sel) {
  const Slot& s = B.h[0];
  if (sel == SEL_L) return MRef{reinterpret_cast<float2*>(s.L), B.mat_stride, B.np, B.np, s.Linv, B.linv_stride, sel};
  if (sel == SEL_COV) return MRef{reinterpret_cast<float2*>(s.Wk), B.mat_stride, B.ndp, B.np, s.Wd, B.wd_stride, sel};
  if (sel == SEL_AUX) return MRef{reinterpret_cast<float2*>(s.Qp), B.mat_stride, s.aux_n, B.np, s.Linv, B.linv_stride, sel};
  return MRef{reinterpret_cast<float2*>(s.S), B.s_stride, B.kp, B.kp, s.SLinv, B.slinv_stride, sel};
}

OzOperand operand(uint16_t* planes, int32_t* exps, int rows, int K) {
  OzOperand o;
  o.planes = planes;
  o.exps = exps;
  o.rows = rows;
  o.K = K;
  o.ld_k = (int)round_up(K, OZ_BK);
  o.plane_stride = (int64_t)rows * o.ld_k;
  o.exp_chunk_stride = rows;
  o.exp_slot_stride = (int64_t)((K + OZ_CHUNK - 1) / OZ_CHUNK) * rows;
  return o;
}

OzArgs gemm_args(const Batch& B, float2* C, int64_t c_stride, int ldc, int M, int N, int K, float alpha, float beta) {
  OzArgs a;
  memset(&a, 0, sizeof(a));
  a.C = C;
  a.C_slot_stride = c_stride;
  a.ldc = ldc;
  a.M = M;
  a.N = N;
  a.K = K;
  a.alpha = alpha;
  a.beta = beta;
  a.S = B.S;
  a.spin_limit = B.spin_limit;
  a.err = B.err;
  return a;
}

// Side stream: of two independent slicing launches (the operands of one GEMM), the first runs on
// a per-device side stream forked from the batch's stream and joined back before the GEMM (events;
// inside a graph capture they become graph edges), so that the two overlap.  Off (everything on
// the batch's stream) for the legacy default stream and while the per-kernel profiler, the GEMM
// statistics or debug synchronisation is on.
struct SideRes {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
SideRes g_side[64];
std::mutex g_side_mu;

class Side {
 public:
  explicit Side(const Batch& B) : main_(B.st) {
    if (!main_ || prof_active() || oz_stats_active() || debug_sync_enabled()) return;
    const int dev = current_device();
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(g_side_mu);
    SideRes& r = g_side[dev];
    if (!r.st) {
      SideRes n;
      if (cudaStreamCreateWithFlags(&n.st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&n.fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&n.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return;  // stays off (a partial set-up is leaked rather than half used)
      }
      r = n;
    }
    res_ = &r;
  }
  ~Side() { join(); }
  bool on() const { return res_ != nullptr; }
  // a side launch that a later Side (the next tile's) joins: the side stream keeps its order
  cudaStream_t fork_detached() {
    if (!res_) return main_;
    cudaEventRecord(res_->fork, main_);
    cudaStreamWaitEvent(res_->st, res_->fork, 0);
    return res_->st;
  }
  // the stream for the side launch (ordered after everything issued so far on the batch's stream)
  cudaStream_t fork() {
    if (!res_) return main_;
    cudaEventRecord(res_->fork, main_);
    cudaStreamWaitEvent(res_->st, res_->fork, 0);
    forked_ = true;
    return res_->st;
  }
  // the batch's stream waits for the side launch (also on every early return, by the destructor)
  void join() {
    if (!forked_) return;
    cudaEventRecord(res_->join, res_->st);
    cudaStreamWaitEvent(main_, res_->join, 0);
    forked_ = false;
  }

 private:
  cudaStream_t main_;
  SideRes* res_ = nullptr;
  bool forked_ = false;
};

}  // namespace

// Columns [c0, c1) of an outer panel, every slot: rows >= c0 hold A minus the updates of the
// columns left of c0.  64 wide: factor the diagonal tile in double-float and form the tile
// column below it as X = A_panel Linv^T.  Wider: factor the left half recursively, update the
// right half with one product of K = the left half's width, factor the right half.  The
// within-panel updates are then a few long-K products (K = 256, 128, 64 for a 512-wide panel)
// rather than one K = 64 update per tile column.
static int mixed_panel(Batch& B, const MRef& M, int c0, int c1) {
  const int n = M.n, S = B.S;
  if (c1 - c0 <= IB) {
    const int R = n - c0 - IB;
    // the panel below the tile is sliced (side stream) while the tile is factored
    Side side(B);
    OzOperand pa = operand(B.PA, B.EA, R > 0 ? R : 1, IB);
    if (R > 0) oz_slice_df(M.base, M.stride, M.ld, c0 + IB, c0, R, IB, false, pa, S, B.n, side.fork());
    // the tile kernel also slices its inverse tile: the B operand of the panel product
    OzOperand pb = operand(B.PB, B.EB, IB, IB);
    launch_potrf_diag_df(B.d_slots, B.n, M.sel, c0 / IB, R > 0 ? &pb : nullptr, S, B.st);
    if (R <= 0) return INLA_OK;
    float2* panel = M.base + (int64_t)(c0 + IB) * M.ld + c0;
    side.join();
    OzArgs a = gemm_args(B, panel, M.stride, M.ld, R, IB, IB, 0.f, 1.f);
    return oz_gemm(pa, pb, a, B.n, B.st);
  }
  const int mid = c0 + (c1 - c0) / (2 * IB) * IB;
  INLA_TRY(mixed_panel(B, M, c0, mid));
  // A[mid:, mid:c1] -= L[mid:, c0:mid] L[mid:c1, c0:mid]^T  (B operand: the first w rows of A's)
  const int R = n - mid, K = mid - c0, w = c1 - mid;
  OzOperand px = operand(B.PA, B.EA, R, K);
  oz_slice_df(M.base, M.stride, M.ld, mid, c0, R, K, false, px, S, B.n, B.st);
  OzOperand pxt = px;
  pxt.rows = w;
  float2* C0 = M.base + (int64_t)mid * M.ld + mid;
  Side side(B);
  if (side.on() && R > IB) {
    // Look-ahead: the next diagonal tile's 64 rows first (its factorisation needs only them); the
    // other rows on the side stream, with one SM per slot left to the tile's factorisation, which
    // runs meanwhile.  The next tile's panel is sliced on the side stream after them, and the tile
    // joins the side stream before its triangular-solve product.
    OzOperand pxa = px;
    pxa.rows = IB;
    OzArgs ua = gemm_args(B, C0, M.stride, M.ld, IB, w, K, 1.f, -1.f);
    INLA_TRY(oz_gemm(pxa, pxt, ua, B.n, B.st));
    OzOperand pxb = px;
    pxb.planes += (int64_t)IB * px.ld_k;
    pxb.exps += IB;
    pxb.rows = R - IB;
    OzArgs ub = gemm_args(B, C0 + (int64_t)IB * M.ld, M.stride, M.ld, R - IB, w, K, 1.f, -1.f);
    ub.max_ctas = std::max(1, oz_num_sms() - B.n);
    INLA_TRY(oz_gemm(pxb, pxt, ub, B.n, side.fork_detached()));
  } else {
    OzArgs u = gemm_args(B, C0, M.stride, M.ld, R, w, K, 1.f, -1.f);
    INLA_TRY(oz_gemm(px, pxt, u, B.n, B.st));
  }
  return mixed_panel(B, M, mid, c1);
}

// In-place Cholesky of the matrix selected by `sel` (lower triangle), every slot: the launches.
static int mixed_potrf_launches(Batch& B, int sel, int nb) {
  const MRef M = mref(B, sel);
  const int n = M.n, S = B.S;
  for (int K0 = 0; K0 < n; K0 += nb) {
    const int kend = std::min(K0 + nb, n);
    INLA_TRY(mixed_panel(B, M, K0, kend));
    const int R2 = n - kend;
    if (R2 > 0) {
      OzOperand pp = operand(B.PA, B.EA, R2, kend - K0);
      oz_slice_df(M.base, M.stride, M.ld, kend, K0, R2, kend - K0, false, pp, S, B.n, B.st);
      OzArgs a = gemm_args(B, M.base + (int64_t)kend * M.ld + kend, M.stride, M.ld, R2, R2, kend - K0, 1.f, -1.f);
      a.lower = 1;
      INLA_TRY(oz_gemm(pp, pp, a, B.n, B.st));
    }
  }
  return INLA_OK;
}

// The blocked Cholesky issues ~1300 launches at n = 16384 whose sequence depends only on the
// batch layout (buffers, strides, slot count), the matrix selected and the slice count.  The
// first call with a layout runs the launches; the second captures them into a CUDA graph
// (stream capture, this thread only) and every later call replays it.  Off when the per-kernel
// profiler, the GEMM statistics or debug synchronisation is on, or on the legacy default stream
// (which cannot be captured).
namespace {
struct PotrfGraphKey {
  int sel, S, n_slots, nb;
  const void* ptrs[7];
  int64_t spin;
  bool operator<(const PotrfGraphKey& o) const {
    if (sel != o.sel) return sel < o.sel;
    if (S != o.S) return S < o.S;
    if (n_slots != o.n_slots) return n_slots < o.n_slots;
    if (nb != o.nb) return nb < o.nb;
    if (spin != o.spin) return spin < o.spin;
    for (int i = 0; i < 7; ++i)
      if (ptrs[i] != o.ptrs[i]) return ptrs[i] < o.ptrs[i];
    return false;
  }
};
struct PotrfGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  bool failed = false;
};
std::map<PotrfGraphKey, PotrfGraph> g_potrf_graphs;
}  // namespace

void mixed_graphs_clear() {
  for (auto& kv : g_potrf_graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  g_potrf_graphs.clear();
}

// Outer-block tuner: for each blocked routine (the Cholesky, the transposed inverse, the forward
// substitution with many right-hand sides) and shape (matrix size, slices, slots, right-hand
// sides), the first two real calls run with the candidates 256 and 512 in turn, timed with CUDA
// events on the stream (no extra work); once both timings are complete, the faster candidate is
// used from then on.
namespace {
constexpr int kNbCandidates[2] = {256, 512};
struct NbTune {
  cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int runs = 0;
  int best = 0;  // 0: undecided
};
enum { NB_POTRF = 0, NB_INVERSE = 1, NB_TRSM = 2 };
std::map<std::tuple<int, int, int, int, int>, NbTune> g_nb_tune;  // (routine, size, slices, slots, rhs)

// INLA_OUTER_BLOCK=256 or 512 pins the outer block of every tuned mixed routine (no tuning
// runs): under a profiler the tuner's timings would not reflect the unprofiled program.
int pinned_nb() {
  static const int v = [] {
    const char* e = getenv("INLA_OUTER_BLOCK");
    const int x = e ? atoi(e) : 0;
    return (x == kNbCandidates[0] || x == kNbCandidates[1]) ? x : 0;
  }();
  return v;
}

int pick_nb(int routine, int n, int S, int nslots, int rhs, NbTune*& tune, int& cand) {
  tune = nullptr;
  cand = -1;
  if (pinned_nb()) return pinned_nb();
  if (n < 2 * kNbCandidates[1]) return kNbCandidates[0];  // too small for the wider block to matter
  NbTune& t = g_nb_tune[std::make_tuple(routine, n, S, nslots, rhs)];
  if (t.best) return t.best;
  if (t.runs == 2) {
    float ms[2] = {0.f, 0.f};
    bool done = true;
    for (int c = 0; c < 2; ++c)
      done = done && cudaEventQuery(t.ev[c][1]) == cudaSuccess &&
             cudaEventElapsedTime(&ms[c], t.ev[c][0], t.ev[c][1]) == cudaSuccess;
    cudaGetLastError();
    if (done) {
      t.best = ms[1] < ms[0] ? kNbCandidates[1] : kNbCandidates[0];
      for (auto& e2 : t.ev)
        for (auto& e : e2) cudaEventDestroy(e);
      return t.best;
    }
    return kNbCandidates[0];  // timings not complete yet
  }
  cand = t.runs;
  tune = &t;
  return kNbCandidates[cand];
}

// A tuning run brackets the routine's launches with the candidate's events.
struct TuneTimer {
  NbTune* t;
  int cand;
  cudaStream_t st;
  int begin() {
    if (!t) return INLA_OK;
    for (auto& e : t->ev[cand])
      if (!e && cudaEventCreate(&e) != cudaSuccess) return INLA_E_CUDA;
    cudaEventRecord(t->ev[cand][0], st);
    return INLA_OK;
  }
  void end() {
    if (!t) return;
    cudaEventRecord(t->ev[cand][1], st);
    ++t->runs;
  }
};

int nb_choice(int routine, int n, int S) {
  if (pinned_nb()) return pinned_nb();
  int best = 0, most_slots = -1;  // the decided choice for the largest batch of this size
  for (const auto& kv : g_nb_tune)
    if (std::get<0>(kv.first) == routine && std::get<1>(kv.first) == n && std::get<2>(kv.first) == S &&
        kv.second.best && std::get<3>(kv.first) > most_slots) {
      most_slots = std::get<3>(kv.first);
      best = kv.second.best;
    }
  return best;
}
}  // namespace

int mixed_nb_choice(int n, int S) { return nb_choice(NB_POTRF, n, S); }
int mixed_inverse_nb_choice(int n, int S) { return nb_choice(NB_INVERSE, n, S); }

int mixed_potrf(Batch& B, int sel) {
  const MRef M = mref(B, sel);
  NbTune* tune = nullptr;
  int cand = -1;
  const int nb = pick_nb(NB_POTRF, M.n, B.S, B.n, 0, tune, cand);
  if (tune) {
    // a tuning run: timed, never captured
    TuneTimer tt{tune, cand, B.st};
    INLA_TRY(tt.begin());
    const int rc = mixed_potrf_launches(B, sel, nb);
    tt.end();
    return rc;
  }
  if (B.st == nullptr || prof_active() || oz_stats_active() || debug_sync_enabled())
    return mixed_potrf_launches(B, sel, nb);
  PotrfGraphKey key{sel, B.S, B.n, nb, {B.d_slots, M.base, M.linv, B.PA, B.PB, B.EA, B.err}, B.spin_limit};
  auto it = g_potrf_graphs.find(key);
  if (it == g_potrf_graphs.end()) {
    if (g_potrf_graphs.size() >= 32) mixed_graphs_clear();
    g_potrf_graphs[key] = PotrfGraph{};
    return mixed_potrf_launches(B, sel, nb);  // first use of this layout: plain launches
  }
  PotrfGraph& g = it->second;
  if (g.failed) return mixed_potrf_launches(B, sel, nb);
  if (!g.exec) {
    cudaGraph_t graph = nullptr;
    const int64_t c0 = g_kernel_launches;
    int rc = INLA_OK;
    if (cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g.failed = true;
      return mixed_potrf_launches(B, sel, nb);
    }
    rc = mixed_potrf_launches(B, sel, nb);
    const cudaError_t e = cudaStreamEndCapture(B.st, &graph);
    if (rc != INLA_OK || e != cudaSuccess || !graph ||
        cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      g.exec = nullptr;
      g.failed = true;
      g_kernel_launches = c0;
      return mixed_potrf_launches(B, sel, nb);  // nothing ran during the capture
    }
    cudaGraphDestroy(graph);
    g.launches = g_kernel_launches - c0;
    g_kernel_launches = c0;
  }
  if (cudaGraphLaunch(g.exec, B.st) != cudaSuccess) return note_launch_error("mixed potrf graph launch");
  g_kernel_launches += g.launches;
  return INLA_OK;
}

// X <- F^-1 X (forward substitution, F lower-triangular factor selected by `fsel`), X with
// `nrows` = F.n rows and `ncols` columns (leading dimension ldx).  identity: X = I on entry,
// so block row K only has nonzero columns [0, end of block K).
static int trsm_left_nb(Batch& B, const MRef& F, float2* X, int64_t x_stride, int ldx, int ncols, bool identity,
                        int NB) {
  const int n = F.n, S = B.S;
  for (int K0 = 0; K0 < n; K0 += NB) {
    const int kend = std::min(K0 + NB, n);
    const int nc = identity ? std::min(kend, ncols) : ncols;
    for (int j0 = K0; j0 < kend; j0 += IB) {
      // X[j0 tile, 0:nc] = Linv_j X[j0 tile, 0:nc]
      OzOperand pl = operand(B.PA, B.EA, IB, IB);
      OzOperand px = operand(B.PB, B.EB, nc, IB);
      {
        Side side(B);
        oz_slice_df(reinterpret_cast<float2*>(F.linv) + (int64_t)(j0 / IB) * IB * IB, F.linv_stride, IB, 0, 0, IB,
                    IB, false, pl, S, B.n, side.fork());
        oz_slice_df(X, x_stride, ldx, j0, 0, nc, IB, true, px, S, B.n, B.st);
      }
      OzArgs a = gemm_args(B, X + (int64_t)j0 * ldx, x_stride, ldx, IB, nc, IB, 0.f, 1.f);
      INLA_TRY(oz_gemm(pl, px, a, B.n, B.st));
      const int r_hi = kend;
      if (j0 + IB < r_hi) {
        const int R = r_hi - j0 - IB;
        OzOperand pf = operand(B.PA, B.EA, R, IB);
        OzOperand px2 = operand(B.PB, B.EB, nc, IB);
        {
          Side side(B);
          oz_slice_df(F.base, F.stride, F.ld, j0 + IB, j0, R, IB, false, pf, S, B.n, side.fork());
          oz_slice_df(X, x_stride, ldx, j0, 0, nc, IB, true, px2, S, B.n, B.st);
        }
        OzArgs u = gemm_args(B, X + (int64_t)(j0 + IB) * ldx, x_stride, ldx, R, nc, IB, 1.f, -1.f);
        INLA_TRY(oz_gemm(pf, px2, u, B.n, B.st));
      }
    }
    const int R = n - kend;
    if (R > 0) {
      OzOperand pf = operand(B.PA, B.EA, R, kend - K0);
      OzOperand px = operand(B.PB, B.EB, nc, kend - K0);
      {
        Side side(B);
        oz_slice_df(F.base, F.stride, F.ld, kend, K0, R, kend - K0, false, pf, S, B.n, side.fork());
        oz_slice_df(X, x_stride, ldx, K0, 0, nc, kend - K0, true, px, S, B.n, B.st);
      }
      OzArgs u = gemm_args(B, X + (int64_t)kend * ldx, x_stride, ldx, R, nc, kend - K0, 1.f, -1.f);
      INLA_TRY(oz_gemm(pf, px, u, B.n, B.st));
    }
  }
  return INLA_OK;
}
static int trsm_left(Batch& B, int fsel, float2* X, int64_t x_stride, int ldx, int ncols, bool identity) {
  const MRef F = mref(B, fsel);
  NbTune* tune = nullptr;
  int cand = -1;
  const int nb = pick_nb(NB_TRSM, F.n, B.S, B.n, ncols, tune, cand);
  TuneTimer tt{tune, cand, B.st};
  INLA_TRY(tt.begin());
  const int rc = trsm_left_nb(B, F, X, x_stride, ldx, ncols, identity, nb);
  if (rc == INLA_OK) tt.end();
  return rc;
}

// Y = F^-T (upper triangular: the transpose of the inverse of the lower factor F), written into
// Wk (into_wk) or into L.  Column blocks of Y in increasing order: Y[:, K] = Y[:, K] Linv_K^T, then
// Y[:, J] -= Y[:, K] F[J, K]^T for the blocks J > K -- the transpose of forward substitution on
// the rows of F^-1, so that every operand is sliced by rows (Y's column block and F's row block
// are both K-contiguous) and only the first kend rows of Y (its nonzero part) enter.
static int inverse_factor_nb(Batch& B, const MRef& F, bool into_wk, int NB) {
  const Slot& s0 = B.h[0];
  const int n = F.n, S = B.S;
  float2* Y = reinterpret_cast<float2*>(into_wk ? s0.Wk : s0.L);
  const int64_t ys = B.mat_stride;
  const int ld = B.np;
  for (int i = 0; i < B.n; ++i)
    cudaMemsetAsync(into_wk ? B.h[i].Wk : B.h[i].L, 0, (size_t)B.mat_stride * 8, B.st);
  launch_diag_ones_df(Y, ys, ld, n, B.n, B.st);
  for (int K0 = 0; K0 < n; K0 += NB) {
    const int kend = std::min(K0 + NB, n);
    const int nc = kend;  // rows of Y that can be nonzero in columns [K0, kend)
    for (int j0 = K0; j0 < kend; j0 += IB) {
      // Y[0:nc, j0 tile] = Y[0:nc, j0 tile] Linv_j^T
      OzOperand py = operand(B.PA, B.EA, nc, IB);
      OzOperand pl = operand(B.PB, B.EB, IB, IB);
      {
        Side side(B);
        oz_slice_df(reinterpret_cast<float2*>(F.linv) + (int64_t)(j0 / IB) * IB * IB, F.linv_stride, IB, 0, 0, IB,
                    IB, false, pl, S, B.n, side.fork());
        oz_slice_df(Y, ys, ld, 0, j0, nc, IB, false, py, S, B.n, B.st);
      }
      OzArgs a = gemm_args(B, Y + j0, ys, ld, nc, IB, IB, 0.f, 1.f);
      INLA_TRY(oz_gemm(py, pl, a, B.n, B.st));
      if (j0 + IB < kend) {
        // Y[0:nc, j0+64 .. kend] -= Y[0:nc, j0 tile] F[j0+64 .. kend, j0 tile]^T
        const int R = kend - j0 - IB;
        OzOperand py2 = operand(B.PA, B.EA, nc, IB);
        OzOperand pf = operand(B.PB, B.EB, R, IB);
        {
          Side side(B);
          oz_slice_df(F.base, F.stride, F.ld, j0 + IB, j0, R, IB, false, pf, S, B.n, side.fork());
          oz_slice_df(Y, ys, ld, 0, j0, nc, IB, false, py2, S, B.n, B.st);
        }
        OzArgs u = gemm_args(B, Y + j0 + IB, ys, ld, nc, R, IB, 1.f, -1.f);
        INLA_TRY(oz_gemm(py2, pf, u, B.n, B.st));
      }
    }
    const int R = n - kend;
    if (R > 0) {
      // Y[0:nc, kend .. n] -= Y[0:nc, K0:kend] F[kend .. n, K0:kend]^T
      OzOperand py = operand(B.PA, B.EA, nc, kend - K0);
      OzOperand pf = operand(B.PB, B.EB, R, kend - K0);
      {
        Side side(B);
        oz_slice_df(F.base, F.stride, F.ld, kend, K0, R, kend - K0, false, pf, S, B.n, side.fork());
        oz_slice_df(Y, ys, ld, 0, K0, nc, kend - K0, false, py, S, B.n, B.st);
      }
      OzArgs u = gemm_args(B, Y + kend, ys, ld, nc, R, kend - K0, 1.f, -1.f);
      INLA_TRY(oz_gemm(py, pf, u, B.n, B.st));
    }
  }
  return INLA_OK;
}
int mixed_inverse_factor(Batch& B, int sel, bool into_wk) {
  const MRef F = mref(B, sel);
  NbTune* tune = nullptr;
  int cand = -1;
  const int nb = pick_nb(NB_INVERSE, F.n, B.S, B.n, 0, tune, cand);
  TuneTimer tt{tune, cand, B.st};
  INLA_TRY(tt.begin());
  const int rc = inverse_factor_nb(B, F, into_wk, nb);
  if (rc == INLA_OK) tt.end();
  return rc;
}

// Q_p[0:nd, 0:nd] = W^T W = Y Y^T with Y = L_Sigma^-T held in L (upper): row k of Y is nonzero
// from column k on, so the lower tiles (m0 >= n0) need k >= m0 only
int mixed_lauum_cov(Batch& B) {
  const Slot& s0 = B.h[0];
  const int ndp = B.ndp, nd = s0.nd, S = B.S;
  OzOperand pw = operand(B.PBIG, B.EBIG, ndp, ndp);
  oz_slice_df(reinterpret_cast<float2*>(s0.L), B.mat_stride, B.np, 0, 0, ndp, ndp, false, pw, S, B.n, B.st);
  float2* C = reinterpret_cast<float2*>(s0.Qp) + (int64_t)s0.nd_off * B.np + s0.nd_off;
  OzArgs a = gemm_args(B, C, B.mat_stride, B.np, nd, nd, ndp, 0.f, 1.f);
  a.lower = 1;
  a.k_mode = 1;
  return oz_gemm(pw, pw, a, B.n, B.st);
}

// Z = L^-1 C^T ; S = Z^T Z (identity on the padding) ; factor S
int mixed_schur(Batch& B) {
  const Slot& s0 = B.h[0];
  const int S = B.S;
  for (int i = 0; i < B.n; ++i) cudaMemsetAsync(B.h[i].Z, 0, (size_t)B.z_stride * 8, B.st);
  launch_ct_fill_df(B.d_slots, B.n, B.kp, B.st);
  float2* Z = reinterpret_cast<float2*>(s0.Z);
  INLA_TRY(trsm_left(B, SEL_L, Z, B.z_stride, B.kp, B.kp, false));
  OzOperand pz = operand(B.PA, B.EA, B.kp, B.np);
  oz_slice_df(Z, B.z_stride, B.kp, 0, 0, B.kp, B.np, true, pz, S, B.n, B.st);
  OzArgs a = gemm_args(B, reinterpret_cast<float2*>(s0.S), B.s_stride, B.kp, B.kp, B.kp, B.np, 0.f, 1.f);
  a.lower = 1;
  INLA_TRY(oz_gemm(pz, pz, a, B.n, B.st));
  launch_s_pad_identity(B.d_slots, B.n, B.kp, B.st);
  return mixed_potrf(B, SEL_S);
}

// t2 = colsumsq(L_S^-1 Z^T W), W = Q*^-1's factor inverse, held transposed (Y = W^T) in Wk; uses
// L as scratch.  G = Z^T W = Z^T Y^T: B operand = the rows of Y
int mixed_var_constraint(Batch& B) {
  const Slot& s0 = B.h[0];
  const int S = B.S;
  float2* Z = reinterpret_cast<float2*>(s0.Z);
  float2* W = reinterpret_cast<float2*>(s0.Wk);
  float2* G = reinterpret_cast<float2*>(s0.L);
  OzOperand pz = operand(B.PA, B.EA, B.kp, B.np);
  oz_slice_df(Z, B.z_stride, B.kp, 0, 0, B.kp, B.np, true, pz, S, B.n, B.st);
  OzOperand pw = operand(B.PBIG, B.EBIG, B.np, B.np);
  oz_slice_df(W, B.mat_stride, B.np, 0, 0, B.np, B.np, false, pw, S, B.n, B.st);
  OzArgs a = gemm_args(B, G, B.mat_stride, B.np, B.kp, B.np, B.np, 0.f, 1.f);
  a.k_mode = 2;
  INLA_TRY(oz_gemm(pz, pw, a, B.n, B.st));
  INLA_TRY(trsm_left(B, SEL_S, G, B.mat_stride, B.np, B.np, false));
  launch_colsumsq_gt_df(B.d_slots, B.n, B.np / TB, B.st);
  return INLA_OK;
}

// Marginal variances by the Moore-Penrose / Woodbury route (Section 3.1, Eq. (woodeqn)) in its
// symmetric m x m form: with B = D^1/2 A (D the likelihood weights at the mode),
//   Sigma* = Q+ - Q+ B^T (I + B Q+ B^T)^-1 B Q+,
// so diag(Sigma*)_j = Q+_jj - |L_M^-1 (B Q+)_{:,j}|^2 with L_M the factor of M = I + B Q+ B^T.
// Q+ (block pseudo-inverse of the prior precision) in Wk, G = B Q+ in L (rows [0, m)), M in Qp
// (aux_n x aux_n), its factor by the mixed Cholesky, Z = L_M^-1 G by forward substitution, the
// variances into t1.  Needs aux_n <= n_pad.
int mixed_woodbury_variances(Batch& B) {
  launch_woodbury_terms_df(B.d_slots, B.n, B.np, B.st);
  INLA_TRY(mixed_potrf(B, SEL_AUX));
  INLA_TRY(trsm_left(B, SEL_AUX, reinterpret_cast<float2*>(B.h[0].L), B.mat_stride, B.np, B.np, false));
  launch_woodbury_var_df(B.d_slots, B.n, B.np, B.st);
  return INLA_OK;
}

__global__ void k_diag_ones_df(float2* base, int64_t slot_stride, int ld, int n) {
  float2* W = base + blockIdx.y * slot_stride;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    W[(int64_t)i * ld + i] = make_float2(1.f, 0.f);
}
void launch_diag_ones_df(float2* base, int64_t slot_stride, int ld, int n, int nslots, cudaStream_t st) {
  count_launch("k_diag_ones_df"), k_diag_ones_df<<<dim3(std::min(1024, (n + 255) / 256), nslots), 256, 0, st>>>(base, slot_stride, ld, n);
}

}  // namespace inla

// Surrogate network kernels: forward, backpropagation, Adam, input gradients (FP32).
//
// The layer products are N x 128 x 128 with N ~ 2000 (tens of MFLOP): launch latency and
// memory traffic bound them, not arithmetic, so they run on the FP32 pipes with every weight
// gradient reduced by one thread over the samples (deterministic, no atomics), and a training
// epoch -- four kernels -- is captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include <vector>
#include "../../include/inla.h"
#include "../../include/inla_surrogate.h"
#include "internal.h"

namespace inla {
namespace {

constexpr int H = INLA_MLP_HIDDEN;
constexpr int TS = 16;  // samples per block in the per-sample kernels

struct Off {
  int W1, b1, W2, b2, w3, b3, P;
};
__host__ __device__ inline Off offsets(int D) {
  Off o;
  o.W1 = 0;
  o.b1 = H * D;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + H * H;
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + H;
  o.P = o.b3 + 1;
  return o;
}

// a1 = tanh(W1 x + b1), a2 = tanh(W2 a1 + b2), f = w3 . a2 + b3 for TS samples per block;
// thread i = hidden unit i.  W2 is staged transposed in shared memory (conflict-free reads).
__global__ void __launch_bounds__(H) k_mlp_fwd(const float* __restrict__ P, const float* __restrict__ X, int N, int D,
                                               float* __restrict__ A1, float* __restrict__ A2, float* __restrict__ F) {
  extern __shared__ float sm[];
  float* W2T = sm;                 // [j][i]
  float* a1s = sm + H * H;         // [s][j]
  float* xs = a1s + TS * H;        // [s][d]
  float* red = xs + TS * INLA_MLP_MAX_DIN;  // [s][warp]
  const Off o = offsets(D);
  const int i = threadIdx.x, s0 = blockIdx.x * TS;
  for (int e = i; e < H * H; e += H) {
    const int r = e / H, c = e % H;  // W2[r][c]
    W2T[c * H + r] = P[o.W2 + e];
  }
  // every slot of the input tile is written (zeros beyond D and N): the unrolled layer-1 loop
  // reads all INLA_MLP_MAX_DIN of them
  for (int e = i; e < TS * INLA_MLP_MAX_DIN; e += H) {
    const int s = e / INLA_MLP_MAX_DIN, d = e % INLA_MLP_MAX_DIN;
    xs[e] = (s0 + s < N && d < D) ? X[(size_t)(s0 + s) * D + d] : 0.f;
  }
  __syncthreads();
  float w1[INLA_MLP_MAX_DIN];
#pragma unroll
  for (int d = 0; d < INLA_MLP_MAX_DIN; ++d) w1[d] = d < D ? P[o.W1 + i * D + d] : 0.f;
  const float b1 = P[o.b1 + i];
  for (int s = 0; s < TS; ++s) {
    float z = b1;
#pragma unroll
    for (int d = 0; d < INLA_MLP_MAX_DIN; ++d) z = fmaf(w1[d], xs[s * INLA_MLP_MAX_DIN + d], z);
    const float a = tanhf(z);
    a1s[s * H + i] = a;
    if (s0 + s < N) A1[(size_t)(s0 + s) * H + i] = a;
  }
  __syncthreads();
  float acc[TS];
  const float b2 = P[o.b2 + i];
#pragma unroll
  for (int s = 0; s < TS; ++s) acc[s] = b2;
  for (int j = 0; j < H; ++j) {
    const float w = W2T[j * H + i];
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = fmaf(w, a1s[s * H + j], acc[s]);
  }
  const float w3 = P[o.w3 + i];
  const int lane = i & 31, warp = i >> 5;
#pragma unroll
  for (int s = 0; s < TS; ++s) {
    const float a = tanhf(acc[s]);
    if (s0 + s < N) A2[(size_t)(s0 + s) * H + i] = a;
    float c = w3 * a;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0) red[s * 4 + warp] = c;
  }
  __syncthreads();
  if (i < TS && s0 + i < N) F[s0 + i] = ((red[i * 4] + red[i * 4 + 1]) + (red[i * 4 + 2] + red[i * 4 + 3])) + P[o.b3];
}

// Per-sample backpropagation: d3 = df-loss weight (2 (f - y) / N, or 1 for input gradients),
// d2 = d3 w3 (1 - a2^2), d1 = (W2^T d2) (1 - a1^2).  Thread = hidden unit; W2 staged in shared
// memory in its own layout (thread j reads column j: conflict-free).  With dX set, also
// dX = W1^T d1 per sample (input gradients).
__global__ void __launch_bounds__(H) k_mlp_bwd_delta(const float* __restrict__ P, const float* __restrict__ F,
                                                     const float* __restrict__ Y, int N, int D,
                                                     const float* __restrict__ A1, const float* __restrict__ A2,
                                                     float* __restrict__ D1, float* __restrict__ D2,
                                                     float* __restrict__ D3, float* __restrict__ dX) {
  extern __shared__ float sm[];
  float* W2s = sm;                 // [i][j]
  float* d2s = sm + H * H;         // [s][i]
  float* red = d2s + TS * H;       // [s][d][warp]
  const Off o = offsets(D);
  const int t = threadIdx.x, s0 = blockIdx.x * TS;
  for (int e = t; e < H * H; e += H) W2s[e] = P[o.W2 + e];
  const float w3 = P[o.w3 + t];
  for (int s = 0; s < TS; ++s) {
    const int n = s0 + s;
    float d3 = 0.f, a2 = 0.f;
    if (n < N) {
      d3 = Y ? 2.f * (F[n] - Y[n]) / (float)N : 1.f;
      a2 = A2[(size_t)n * H + t];
      if (t == 0 && D3) D3[n] = d3;
    }
    const float d2 = d3 * w3 * (1.f - a2 * a2);
    d2s[s * H + t] = d2;
    if (n < N && D2) D2[(size_t)n * H + t] = d2;
  }
  __syncthreads();
  float acc[TS];
#pragma unroll
  for (int s = 0; s < TS; ++s) acc[s] = 0.f;
  for (int i = 0; i < H; ++i) {
    const float w = W2s[i * H + t];  // W2[i][t]
#pragma unroll
    for (int s = 0; s < TS; ++s) acc[s] = fmaf(w, d2s[s * H + i], acc[s]);
  }
  const int lane = t & 31, warp = t >> 5;
  for (int s = 0; s < TS; ++s) {
    const int n = s0 + s;
    const float a1 = n < N ? A1[(size_t)n * H + t] : 0.f;
    const float d1 = acc[s] * (1.f - a1 * a1);
    if (n < N && D1) D1[(size_t)n * H + t] = d1;
    if (dX) {
      for (int d = 0; d < D; ++d) {
        float c = d1 * P[o.W1 + t * D + d];
        for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
        if (lane == 0) red[(s * INLA_MLP_MAX_DIN + d) * 4 + warp] = c;
      }
    }
  }
  if (dX) {
    __syncthreads();
    for (int e = t; e < TS * D; e += H) {
      const int s = e / D, d = e % D;
      const float* r = red + (s * INLA_MLP_MAX_DIN + d) * 4;
      if (s0 + s < N) dX[(size_t)(s0 + s) * D + d] = (r[0] + r[1]) + (r[2] + r[3]);
    }
  }
}

// Parameter gradients, one thread per parameter, each a sum over the N samples; thread 0 also
// writes the loss (before the update) into loss_hist[step] and advances the step counter.
__global__ void __launch_bounds__(256) k_mlp_bwd_grad(const float* __restrict__ X, const float* __restrict__ Y,
                                                      const float* __restrict__ F, int N, int D,
                                                      const float* __restrict__ A1, const float* __restrict__ A2,
                                                      const float* __restrict__ D1, const float* __restrict__ D2,
                                                      const float* __restrict__ D3, float* __restrict__ G,
                                                      int* step, float* loss_hist, int loss_base, int loss_cap) {
  const Off o = offsets(D);
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0) {
    __shared__ float part[256];
    float l = 0.f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
      const float r = F[n] - Y[n];
      l = fmaf(r, r, l);
    }
    part[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int st = *step, k = st - loss_base;
      if (loss_hist && k >= 0 && k < loss_cap) loss_hist[k] = part[0] / (float)N;
      *step = st + 1;
    }
  }
  if (p >= o.P) return;
  float g0 = 0.f, g1 = 0.f;  // two partial sums for more independent adds
  if (p < o.b1) {
    const int i = p / D, d = p % D;
    for (int n = 0; n + 1 < N; n += 2) {
      g0 = fmaf(D1[(size_t)n * H + i], X[(size_t)n * D + d], g0);
      g1 = fmaf(D1[(size_t)(n + 1) * H + i], X[(size_t)(n + 1) * D + d], g1);
    }
    if (N & 1) g0 = fmaf(D1[(size_t)(N - 1) * H + i], X[(size_t)(N - 1) * D + d], g0);
  } else if (p < o.W2) {
    const int i = p - o.b1;
    for (int n = 0; n < N; ++n) g0 += D1[(size_t)n * H + i];
  } else if (p < o.b2) {
    const int i = (p - o.W2) / H, j = (p - o.W2) % H;
    for (int n = 0; n + 1 < N; n += 2) {
      g0 = fmaf(D2[(size_t)n * H + i], A1[(size_t)n * H + j], g0);
      g1 = fmaf(D2[(size_t)(n + 1) * H + i], A1[(size_t)(n + 1) * H + j], g1);
    }
    if (N & 1) g0 = fmaf(D2[(size_t)(N - 1) * H + i], A1[(size_t)(N - 1) * H + j], g0);
  } else if (p < o.w3) {
    const int i = p - o.b2;
    for (int n = 0; n < N; ++n) g0 += D2[(size_t)n * H + i];
  } else if (p < o.b3) {
    const int i = p - o.w3;
    for (int n = 0; n < N; ++n) g0 = fmaf(D3[n], A2[(size_t)n * H + i], g0);
  } else {
    for (int n = 0; n < N; ++n) g0 += D3[n];
  }
  G[p] = g0 + g1;
}

// Adam with bias correction; the step counter was advanced by k_mlp_bwd_grad (t >= 1).
__global__ void __launch_bounds__(256) k_mlp_adam(float* __restrict__ Pm, const float* __restrict__ G,
                                                  float* __restrict__ Mm, float* __restrict__ Vm, int np,
                                                  const int* step, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float t = (float)(*step);
  const float g = G[p];
  const float m = b1 * Mm[p] + (1.f - b1) * g;
  const float v = b2 * Vm[p] + (1.f - b2) * g * g;
  Mm[p] = m;
  Vm[p] = v;
  const float mh = m / (1.f - powf(b1, t)), vh = v / (1.f - powf(b2, t));
  Pm[p] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace
}  // namespace inla

using namespace inla;

struct inla_mlp {
  int D, maxN, np;
  float *P, *G, *M, *V, *X, *Y, *F, *A1, *A2, *D1, *D2, *D3, *dX;
  int* step;
  void* mem;
};

namespace {
size_t fwd_smem() { return (size_t)(H * H + TS * H + TS * INLA_MLP_MAX_DIN + TS * 4) * sizeof(float); }
size_t bwd_smem() { return (size_t)(H * H + TS * H + TS * INLA_MLP_MAX_DIN * 4) * sizeof(float); }

int set_smem_attrs() {
  static DeviceFlags done;  // the shared-memory limits are per-device attributes
  const int dev = current_device();
  if (done.test(dev)) return INLA_OK;
  if (cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem()) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_bwd_delta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem()) !=
          cudaSuccess)
    return INLA_E_CUDA;
  done.set(dev);
  return INLA_OK;
}

void launch_forward(inla_mlp* n, int N, cudaStream_t st) {
  count_launch("k_mlp_fwd"), k_mlp_fwd<<<(N + TS - 1) / TS, H, fwd_smem(), st>>>(n->P, n->X, N, n->D, n->A1, n->A2, n->F);
}
void launch_backward(inla_mlp* n, int N, float* loss_hist, int loss_base, int loss_cap, cudaStream_t st) {
  count_launch("k_mlp_bwd_delta"), k_mlp_bwd_delta<<<(N + TS - 1) / TS, H, bwd_smem(), st>>>(n->P, n->F, n->Y, N, n->D, n->A1, n->A2, n->D1, n->D2, n->D3, nullptr);
  count_launch("k_mlp_bwd_grad"), k_mlp_bwd_grad<<<(n->np + 255) / 256, 256, 0, st>>>(n->X, n->Y, n->F, N, n->D, n->A1, n->A2, n->D1, n->D2, n->D3, n->G, n->step, loss_hist, loss_base, loss_cap);
}
int upload(inla_mlp* n, const float* X, const float* y, int N) {
  if (cudaMemcpy(n->X, X, sizeof(float) * (size_t)N * n->D, cudaMemcpyHostToDevice) != cudaSuccess) return INLA_E_CUDA;
  if (y && cudaMemcpy(n->Y, y, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess) return INLA_E_CUDA;
  return INLA_OK;
}
int finish(int rc) {
  if (rc == INLA_OK && cudaDeviceSynchronize() != cudaSuccess) rc = INLA_E_CUDA;
  if (rc != INLA_OK) cudaGetLastError();
  return rc;
}
}  // namespace

extern "C" int64_t inla_mlp_num_params(int32_t din) { return offsets(din).P; }

extern "C" int inla_mlp_create(int32_t din, int32_t max_samples, inla_mlp** out) {
  if (!out || din < 1 || din > INLA_MLP_MAX_DIN || max_samples < 1) return INLA_E_BADARG;
  *out = nullptr;
  if (set_smem_attrs() != INLA_OK) return INLA_E_CUDA;
  inla_mlp* n = new inla_mlp();
  n->D = din;
  n->maxN = max_samples;
  n->np = offsets(din).P;
  const size_t N = (size_t)max_samples, np = (size_t)n->np;
  const size_t floats = 4 * np + N * din * 2 + N * 3 + N * H * 4 + 64;
  if (cudaMalloc(&n->mem, floats * sizeof(float) + 256) != cudaSuccess) {
    cudaGetLastError();
    delete n;
    return INLA_E_NOMEM;
  }
  float* f = static_cast<float*>(n->mem);
  n->P = f; f += np;
  n->G = f; f += np;
  n->M = f; f += np;
  n->V = f; f += np;
  n->X = f; f += N * din;
  n->dX = f; f += N * din;
  n->Y = f; f += N;
  n->F = f; f += N;
  n->D3 = f; f += N;
  n->A1 = f; f += N * H;
  n->A2 = f; f += N * H;
  n->D1 = f; f += N * H;
  n->D2 = f; f += N * H;
  n->step = reinterpret_cast<int*>(f);
  if (cudaMemset(n->mem, 0, floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(n->mem);
    delete n;
    return INLA_E_CUDA;
  }
  *out = n;
  return INLA_OK;
}

extern "C" int inla_mlp_destroy(inla_mlp* n) {
  if (!n) return INLA_OK;
  cudaFree(n->mem);
  delete n;
  return INLA_OK;
}

extern "C" int inla_mlp_set_params(inla_mlp* n, const float* params) {
  if (!n || !params) return INLA_E_BADARG;
  int rc = INLA_OK;
  if (cudaMemcpy(n->P, params, sizeof(float) * n->np, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->M, 0, sizeof(float) * n->np) != cudaSuccess ||
      cudaMemset(n->V, 0, sizeof(float) * n->np) != cudaSuccess || cudaMemset(n->step, 0, sizeof(int)) != cudaSuccess)
    rc = INLA_E_CUDA;
  return finish(rc);
}

extern "C" int inla_mlp_get_params(const inla_mlp* n, float* params) {
  if (!n || !params) return INLA_E_BADARG;
  return finish(cudaMemcpy(params, n->P, sizeof(float) * n->np, cudaMemcpyDeviceToHost) == cudaSuccess ? INLA_OK
                                                                                                      : INLA_E_CUDA);
}

extern "C" int inla_mlp_loss_grad(inla_mlp* n, const float* X, const float* y, int32_t N, float* loss, float* grad) {
  if (!n || !X || !y || N < 1 || N > n->maxN) return INLA_E_BADARG;
  int rc = upload(n, X, y, N);
  if (rc != INLA_OK) return finish(rc);
  float* lh = nullptr;
  int step0 = 0;
  if (cudaMalloc(&lh, sizeof(float)) != cudaSuccess) return finish(INLA_E_NOMEM);
  if (cudaMemcpy(&step0, n->step, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = INLA_E_CUDA;
  if (rc == INLA_OK) {
    launch_forward(n, N, 0);
    launch_backward(n, N, lh, step0, 1, 0);
    if (cudaPeekAtLastError() != cudaSuccess) rc = note_launch_error("mlp loss/grad");
  }
  // no update was made: put the step counter back
  if (rc == INLA_OK &&
      (cudaMemcpy(n->step, &step0, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
       (loss && cudaMemcpy(loss, lh, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) ||
       (grad && cudaMemcpy(grad, n->G, sizeof(float) * n->np, cudaMemcpyDeviceToHost) != cudaSuccess)))
    rc = INLA_E_CUDA;
  cudaFree(lh);
  return finish(rc);
}

extern "C" int inla_mlp_train(inla_mlp* n, const float* X, const float* y, int32_t N, int32_t epochs, float lr,
                              float* loss_out) {
  if (!n || !X || !y || N < 1 || N > n->maxN || epochs < 0 || !(lr > 0.f)) return INLA_E_BADARG;
  if (epochs == 0) return INLA_OK;
  int rc = upload(n, X, y, N);
  if (rc != INLA_OK) return finish(rc);
  float* lh = nullptr;
  int step0 = 0;
  if (cudaMalloc(&lh, sizeof(float) * (size_t)epochs) != cudaSuccess) return finish(INLA_E_NOMEM);
  if (cudaMemcpy(&step0, n->step, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = INLA_E_CUDA;
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (rc == INLA_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = INLA_E_CUDA;
  // the loss history is indexed by the step counter relative to this call's first step
  if (rc == INLA_OK && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = INLA_E_CUDA;
  if (rc == INLA_OK) {
    launch_forward(n, N, st);
    launch_backward(n, N, lh, step0, epochs, st);
    count_launch("k_mlp_adam"), k_mlp_adam<<<(n->np + 255) / 256, 256, 0, st>>>(n->P, n->G, n->M, n->V, n->np, n->step, lr);
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess || !graph) rc = note_launch_error("mlp epoch capture");
  }
  if (rc == INLA_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = note_launch_error("mlp graph");
  for (int ep = 0; rc == INLA_OK && ep < epochs; ++ep)
    if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = note_launch_error("mlp graph launch");
  if (rc == INLA_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = INLA_E_CUDA;
  if (rc == INLA_OK && loss_out &&
      cudaMemcpy(loss_out, lh, sizeof(float) * (size_t)epochs, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = INLA_E_CUDA;
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (st) cudaStreamDestroy(st);
  cudaFree(lh);
  return finish(rc);
}

extern "C" int inla_mlp_predict(inla_mlp* n, const float* X, int32_t N, float* f, float* dfdx) {
  if (!n || !X || !f || N < 1 || N > n->maxN) return INLA_E_BADARG;
  int rc = upload(n, X, nullptr, N);
  if (rc != INLA_OK) return finish(rc);
  launch_forward(n, N, 0);
  if (dfdx)
    count_launch("k_mlp_bwd_delta"), k_mlp_bwd_delta<<<(N + TS - 1) / TS, H, bwd_smem(), 0>>>(n->P, n->F, nullptr, N, n->D, n->A1, n->A2, nullptr, nullptr, nullptr, n->dX);
  if (cudaPeekAtLastError() != cudaSuccess) return finish(note_launch_error("mlp predict"));
  if (cudaMemcpy(f, n->F, sizeof(float) * (size_t)N, cudaMemcpyDeviceToHost) != cudaSuccess ||
      (dfdx && cudaMemcpy(dfdx, n->dX, sizeof(float) * (size_t)N * n->D, cudaMemcpyDeviceToHost) != cudaSuccess))
    rc = INLA_E_CUDA;
  return finish(rc);
}

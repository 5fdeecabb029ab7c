// Allocation-free variant of the Ozaki-split tensor-core GEMM.
//
// Some callers cannot call cudaMalloc: a host application that reserves all device memory
// up front in its own pool and hands out only pointers into it, or code that must not risk
// the implicit device synchronisation and out-of-memory failure of an allocation in the
// middle of its work.  This entry point takes the caller's device buffers for the inputs and
// the output and keeps every intermediate (BF16 slice planes, exponents, the double-float
// product, an error flag) in one file-scope static __device__ array of fixed size, which
// every GPU that loads the library holds until the process exits.
#include <atomic>
#include <cstdint>
#include <cstring>
#include "../../include/inla.h"
#include "df64.cuh"
#include "ozaki.h"

namespace inla {

namespace {

constexpr int NOALLOC_MAX_DIM = 512;   // M, N, K <= 512
constexpr int NOALLOC_MAX_S = 5;
constexpr size_t kPlaneElems = (size_t)NOALLOC_MAX_S * NOALLOC_MAX_DIM * NOALLOC_MAX_DIM;  // per operand
constexpr size_t kExpElems = (size_t)(NOALLOC_MAX_DIM / OZ_CHUNK + 1) * NOALLOC_MAX_DIM;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffPlaneA = 0;
constexpr size_t kOffPlaneB = align256(kOffPlaneA + kPlaneElems * sizeof(uint16_t));
constexpr size_t kOffExpA = align256(kOffPlaneB + kPlaneElems * sizeof(uint16_t));
constexpr size_t kOffExpB = align256(kOffExpA + kExpElems * sizeof(int32_t));
constexpr size_t kOffC = align256(kOffExpB + kExpElems * sizeof(int32_t));
constexpr size_t kOffErr = align256(kOffC + (size_t)NOALLOC_MAX_DIM * NOALLOC_MAX_DIM * sizeof(float2));
constexpr size_t kScratchBytes = align256(kOffErr + sizeof(int32_t));  // ~7.4 MB

// The shared workspace.  In host code its name is only a stand-in for the device object:
// kernels receive the address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The array's device address, looked up once per device (with that device current).  Atomic: two
// host threads making their first call at once may both look it up; both store the same value.
constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_addr[kMaxDevices];

__global__ void k_noalloc_df_to_f64(const float2* src, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i].x + (double)src[i].y;
}

}  // namespace
}  // namespace inla

using namespace inla;

extern "C" int inla_ozaki_gemm_noalloc(const double* A, const double* B, double* C, int32_t M, int32_t N,
                                       int32_t K, int32_t slices, void* stream) {
  if (!A || !B || !C) return INLA_E_BADARG;
  if (M <= 0 || N <= 0 || K <= 0 || M > NOALLOC_MAX_DIM || N > NOALLOC_MAX_DIM || K > NOALLOC_MAX_DIM ||
      (K % OZ_BK) != 0 || slices < 2 || slices > NOALLOC_MAX_S)
    return INLA_E_BADARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return INLA_E_CUDA;
  // set-up, once per device, with that device current
  void* addr = g_scratch_addr[dev].load();
  if (!addr) {
    if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) {
      cudaGetLastError();
      return INLA_E_CUDA;
    }
    g_scratch_addr[dev].store(addr);
  }
  char* base = static_cast<char*>(addr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int S = slices;
  const int ldk = K;  // K is a multiple of 64
  const int nch = (K + OZ_CHUNK - 1) / OZ_CHUNK;
  OzOperand oa{reinterpret_cast<uint16_t*>(base + kOffPlaneA), reinterpret_cast<int32_t*>(base + kOffExpA), M, K, ldk,
               (int64_t)M * ldk, M, (int64_t)nch * M};
  OzOperand ob{reinterpret_cast<uint16_t*>(base + kOffPlaneB), reinterpret_cast<int32_t*>(base + kOffExpB), N, K, ldk,
               (int64_t)N * ldk, N, (int64_t)nch * N};
  float2* cdf = reinterpret_cast<float2*>(base + kOffC);
  int32_t* err = reinterpret_cast<int32_t*>(base + kOffErr);
  // the error flag must start at zero; the planes, exponents and product are fully rewritten
  if (cudaMemsetAsync(err, 0, sizeof(int32_t), st) != cudaSuccess) return INLA_E_CUDA;
  oz_slice_f64(A, 0, K, 0, 0, M, K, false, oa, S, 1, st);
  oz_slice_f64(B, 0, K, 0, 0, N, K, false, ob, S, 1, st);
  // a launch-configuration error does not stick to the stream: check each launch
  if (cudaPeekAtLastError() != cudaSuccess) return note_launch_error("noalloc slicing");
  OzArgs a;
  std::memset(&a, 0, sizeof(a));
  a.C = cdf;
  a.ldc = N;
  a.M = M;
  a.N = N;
  a.K = K;
  a.alpha = 0.f;
  a.beta = 1.f;
  a.S = S;
  a.spin_limit = (int64_t)1 << 26;
  a.err = err;
  int rc = oz_gemm(oa, ob, a, 1, st);
  if (rc != INLA_OK) return rc;
  count_launch("k_noalloc_df_to_f64");
  k_noalloc_df_to_f64<<<128, 256, 0, st>>>(cdf, C, (int64_t)M * N);
  if (cudaPeekAtLastError() != cudaSuccess) return note_launch_error("noalloc conversion");
  int32_t herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return INLA_E_CUDA;
  }
  return herr ? INLA_E_TIMEOUT : INLA_OK;
}

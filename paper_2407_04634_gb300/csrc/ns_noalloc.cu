// ns_project_noalloc: the CGS2 projection of ns_project for callers that cannot
// allocate device memory while they run, e.g. code inside a CUDA graph being
// captured, a custom allocator's own callback, or an embedded host that hands
// the library only pre-allocated buffers.  Its scratch (the per-row-chunk partial
// dot products and the second-pass coefficients) lives in one file-scope device
// array instead of coming from cudaMalloc.
#include <mutex>

#include "../../include/nullspace.h"
#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace {

// Fixed scratch: 4 MiB on every GPU that loads this library, held until the
// process exits.  Partials need ceil(n / 32768) * K * w doubles, the second-pass
// coefficients K * w more.
constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 19;
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once per
// device; the host-side symbol is only a stand-in and must not be passed to kernels).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_add_coeffs(double* C, const double* C2, int cnt) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) C[t] += C2[t];
}

template <int W>
void run(int64_t n, int K, const double* V, double* Wm, double* C, double* scratch, cudaStream_t s) {
  ns::VParts<double> P;
  P.X = V;
  P.kx = K;
  P.Z = nullptr;
  P.kz = 0;
  P.p = 1;
  double* C2 = scratch;
  double* part = scratch + (size_t)K * W;
  ns::Red red;  // unused: no Gram is requested
  ns::proj_dots<double, W>(P, Wm, nullptr, W, n, C, part, s);
  ns::proj_update<double, W>(P, C, Wm, nullptr, W, n, 0, nullptr, nullptr, nullptr, red, s);
  ns::proj_dots<double, W>(P, Wm, nullptr, W, n, C2, part, s);
  ns::proj_update<double, W>(P, C2, Wm, nullptr, W, n, 0, nullptr, nullptr, nullptr, red, s);
  k_add_coeffs<<<ns::ceil_div((int64_t)K * W, 256), 256, 0, s>>>(C, C2, K * W);
}

}  // namespace

extern "C" ns_status ns_project_noalloc(int64_t n, int K, int w, const double* V, double* W, double* C,
                                        void* stream) {
  if (n < 1 || K < 1 || !(w == 1 || w == 2 || w == 4 || w == 8) || !V || !W || !C) return NS_ERR_INVALID_ARG;
  const int64_t rpc = n < (int64_t)ns::kThreads * 128 ? n : (int64_t)ns::kThreads * 128;
  const int64_t nchunks = (n + rpc - 1) / rpc;
  const size_t need = (size_t)K * w * (size_t)(nchunks + 1);
  if (need > kNoAllocScratchDoubles) return NS_ERR_INVALID_ARG;  // beyond the fixed scratch
  if ((size_t)K * w * sizeof(double) > 190 * 1024) return NS_ERR_INVALID_ARG;  // coefficient tile limit
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (w) {
    case 1: run<1>(n, K, V, W, C, scratch, s); break;
    case 2: run<2>(n, K, V, W, C, scratch, s); break;
    case 4: run<4>(n, K, V, W, C, scratch, s); break;
    default: run<8>(n, K, V, W, C, scratch, s); break;
  }
  return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

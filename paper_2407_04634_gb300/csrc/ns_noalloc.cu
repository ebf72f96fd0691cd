// ns_project_noalloc: the CGS2 projection of ns_project for callers that cannot
// allocate device memory while they run, e.g. code inside a CUDA graph being
// captured, a custom allocator's own callback, or an embedded host that hands
// the library only pre-allocated buffers.  Its scratch (the per-row-chunk partial
// dot products and the second-pass coefficients) lives in one file-scope device
// array instead of coming from cudaMalloc.
#include <cuda.h>  // driver types for the context-id query (resolved at run time, not linked)

#include <mutex>

#include "../../include/nullspace.h"
#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace {

// Fixed scratch: 4 MiB on every GPU that loads this library, held until the
// process exits.  Partials need ceil(n / 32768) * K * w doubles, the second-pass
// coefficients K * w more.
constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 19;
constexpr size_t kMaxCoeffBytes = 190 * 1024;  // the update kernel stages K x w coefficients in shared memory
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// The scratch address is a property of the module loaded into a context, so it is
// cached per device together with the id of the context it was looked up in: after
// a context reset (cudaDeviceReset, a new primary context) the id changes and the
// address is looked up again instead of reusing a dead one.
constexpr int kMaxDevices = 64;
struct Slot {
  unsigned long long ctx_id = 0;
  double* ptr = nullptr;
};
std::mutex g_mutex;
Slot g_slot[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
std::once_flag g_entry_once;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// id of the current context, 0 when the driver cannot tell (then every call
// outside a capture repeats the lookup, and calls inside one reuse the last address)
unsigned long long current_context_id() {
  std::call_once(g_entry_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();  // a failed query is ours to clear (no error was pending on entry)
  });
  if (!g_ctx_current || !g_ctx_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&c) != CUDA_SUCCESS || !c || g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context.  The host-side symbol
// is only a stand-in and is never passed to a kernel.  A lookup may load the
// library's device code into the context, which must not happen while `s` is being
// captured into a graph: such a call is refused with NS_ERR_STATE before any lookup.
ns_status scratch_address(cudaStream_t s, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return NS_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lock(g_mutex);
  Slot& sl = g_slot[dev];
  if (capturing && !sl.ptr) return NS_ERR_STATE;  // first call on this device: make it outside a capture
  const unsigned long long id = current_context_id();
  if (sl.ptr && (id != 0 ? sl.ctx_id == id : capturing)) {
    *out = sl.ptr;
    return NS_OK;
  }
  if (capturing) return NS_ERR_STATE;  // first call in this context: make it outside a capture
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  // raise the update kernels' shared-memory limit for every size this entry accepts,
  // so no later call (a captured one included) changes a function attribute
  cudaError_t e = ns::proj_update_reserve_smem<double, 1>(kMaxCoeffBytes);
  if (e == cudaSuccess) e = ns::proj_update_reserve_smem<double, 2>(kMaxCoeffBytes);
  if (e == cudaSuccess) e = ns::proj_update_reserve_smem<double, 4>(kMaxCoeffBytes);
  if (e == cudaSuccess) e = ns::proj_update_reserve_smem<double, 8>(kMaxCoeffBytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  sl.ctx_id = id;
  sl.ptr = static_cast<double*>(p);
  *out = sl.ptr;
  return NS_OK;
}

__global__ void k_add_coeffs(double* C, const double* C2, int cnt) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) C[t] += C2[t];
}

// Error raised by the launches just enqueued (none was pending on entry, so any
// error seen here is this call's own and is cleared before returning).
bool launch_failed() {
  if (cudaPeekAtLastError() == cudaSuccess) return false;
  cudaGetLastError();
  return true;
}

template <int W>
ns_status run(int64_t n, int K, const double* V, double* Wm, double* C, double* scratch, cudaStream_t s) {
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
  if (launch_failed()) return NS_ERR_CUDA;
  if (ns::proj_update<double, W>(P, C, Wm, nullptr, W, n, 0, nullptr, nullptr, nullptr, red, s) != cudaSuccess ||
      launch_failed())
    return NS_ERR_CUDA;
  ns::proj_dots<double, W>(P, Wm, nullptr, W, n, C2, part, s);
  if (launch_failed()) return NS_ERR_CUDA;
  if (ns::proj_update<double, W>(P, C2, Wm, nullptr, W, n, 0, nullptr, nullptr, nullptr, red, s) != cudaSuccess ||
      launch_failed())
    return NS_ERR_CUDA;
  k_add_coeffs<<<ns::ceil_div((int64_t)K * W, 256), 256, 0, s>>>(C, C2, K * W);
  return launch_failed() ? NS_ERR_CUDA : NS_OK;
}

}  // namespace

extern "C" ns_status ns_project_noalloc(int64_t n, int K, int w, const double* V, double* W, double* C,
                                        void* stream) {
  if (n < 1 || K < 1 || !(w == 1 || w == 2 || w == 4 || w == 8) || !V || !W || !C) return NS_ERR_INVALID_ARG;
  const int64_t rpc = n < (int64_t)ns::kThreads * 128 ? n : (int64_t)ns::kThreads * 128;
  const int64_t nchunks = (n + rpc - 1) / rpc;
  const size_t need = (size_t)K * w * (size_t)(nchunks + 1);
  if (need > kNoAllocScratchDoubles) return NS_ERR_INVALID_ARG;          // beyond the fixed scratch
  if ((size_t)K * w * sizeof(double) > kMaxCoeffBytes) return NS_ERR_INVALID_ARG;  // coefficient tile limit
  // an error left pending by the caller's earlier work is reported, not cleared or
  // blamed on this call's launches: nothing is enqueued
  if (cudaPeekAtLastError() != cudaSuccess) return NS_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  const ns_status st = scratch_address(s, &scratch);
  if (st != NS_OK) return st;
  switch (w) {
    case 1: return run<1>(n, K, V, W, C, scratch, s);
    case 2: return run<2>(n, K, V, W, C, scratch, s);
    case 4: return run<4>(n, K, V, W, C, scratch, s);
    default: return run<8>(n, K, V, W, C, scratch, s);
  }
}

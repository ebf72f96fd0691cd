// Batched persistent form: shared definitions of the device kernel (k_batched.cu)
// and its host driver (ns_batch.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ns {

constexpr int kBMaxR = 64;     // restart length limit of the batched kernel
constexpr int kBMaxLock = 32;  // nullity limit per instance
constexpr int kBThreads = 256;    // largest CTA size (128 and 256 are built)
constexpr int kBStats = 13;    // per-instance counters in BatchArgs::istats

struct BatchArgs {
  // concatenated CSR: instance i has n[i] rows, local row pointers at rowptr + rp_off[i],
  // entries at col/val + nz_off[i] (column indices local to the instance)
  const int64_t* rowptr;
  const int* col;
  const float* val;
  const double* val64;
  const int64_t* rp_off;
  const int64_t* nz_off;
  const int* nrows;
  const int64_t* out_off;  // basis of instance i at basis + out_off[i] (n[i] x kBMaxLock, column-major)
  const int* order;        // processing order (decreasing nnz)
  int count;
  uint64_t seed;
  double eps, tol;
  int R;
  int64_t max_matvec;
  double stop_factor;
  double refine_tol;
  int refine_maxit;
  // per-slot workspace
  float* ws32;
  double* ws64;
  int64_t ws32_stride, ws64_stride;
  int nmax;
  // outputs
  double* basis;
  int* nullity;
  int* status;
  long long* istats;  // per instance: matvecs, restarts, reorths, refine iterations, SM clock cycles,
                      // then the cycles of six phases (steps, reorth, eig, locking, restart, refine),
                      // then the FP32 and FP64 Jacobi sweeps of the projected problems
  unsigned* queue;
};

// Kernel attributes for the (LANES, block) variant and the CTAs one SM holds.
cudaError_t batched_prepare(int lanes, int block, int R, int* blocks_per_sm);
// One persistent launch of grid CTAs of `block` threads (128 or 256) over the
// queue a.queue (which must read 0).
void batched_launch(const BatchArgs& a, int lanes, int block, int grid, cudaStream_t s);
// Entry checks of a freshly copied batch (column inside the instance, finite value):
// ORs 2 (column) / 4 (value) into *err.
void batch_validate(const BatchArgs& a, unsigned* err, cudaStream_t s);
// Gather every instance's n_i x N_i basis block (plen[i] = n_i N_i doubles) to packed + poff[i].
void batch_pack(const double* basis, const int64_t* out_off, const int64_t* poff, const int64_t* plen, int count,
                double* packed, cudaStream_t s);
// Workspace per CTA slot, in elements.
size_t batched_ws32_per_slot(int nmax, int R);
size_t batched_ws64_per_slot(int nmax);

}  // namespace ns

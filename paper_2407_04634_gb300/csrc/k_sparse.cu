// Sparse kernels: CSR validation, transpose, norms and the SpMM products of the
// operator B = A^T A + eps D (or A + eps D), Eq. (defB) and Alg. 1 (its perturbed operator).
#include <algorithm>

#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace ns {

int choose_lanes(int64_t nrows, int64_t nnz) {
  const double avg = nrows > 0 ? (double)nnz / (double)nrows : 1.0;
  int V = 1;
  while (V < 32 && 2.0 * V <= avg) V *= 2;
  return V;
}

// ---------------------------------------------------------------------------
// row segment of a CSR product, V lanes per row, D columns of the dense operand
// ---------------------------------------------------------------------------
// The row's nonzeros are taken four per lane at a time: the four column indices and
// values are loaded together, then the four gathered rows of v, so each lane keeps
// four dependent gathers in flight instead of one (the rows of a Laplacian or an
// incidence matrix hold 2-12 entries, so most rows finish in one or two rounds).
template <typename T, int D, int V>
__device__ __forceinline__ void row_product(const Csr<T>& M, const T* __restrict__ v, int64_t row, int lane,
                                            T (&acc)[D]) {
#pragma unroll
  for (int q = 0; q < D; ++q) acc[q] = T(0);
  if (row < M.nrows) {
    const int64_t s = __ldg(M.rowptr + row), e = __ldg(M.rowptr + row + 1);
    int64_t k = s + lane;
    for (; k + 3 * V < e; k += 4 * V) {
      int c[4];
      T a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = __ldg(M.col + k + u * V);
        a[u] = __ldg(M.val + k + u * V);
      }
      T xv[4][D];
#pragma unroll
      for (int u = 0; u < 4; ++u) load_row<T, D>(v + (int64_t)c[u] * D, xv[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] = fma(a[u], xv[u][q], acc[q]);
    }
    if (k < e) {  // the last one to three entries of this lane, predicated
      int c[3];
      T a[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const bool ok = k + u * V < e;
        c[u] = ok ? __ldg(M.col + k + u * V) : 0;
        a[u] = ok ? __ldg(M.val + k + u * V) : T(0);
      }
      T xv[3][D];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if (k + u * V < e) {
          load_row<T, D>(v + (int64_t)c[u] * D, xv[u]);
        } else {
#pragma unroll
          for (int q = 0; q < D; ++q) xv[u][q] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] = fma(a[u], xv[u][q], acc[q]);
    }
  }
  if constexpr (V > 1) {
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  }
}

template <typename T, int D, int V>
__global__ void __launch_bounds__(kThreads) k_spmm_plain(Csr<T> M, const T* __restrict__ v, T* __restrict__ y) {
  const int lane = threadIdx.x % V;
  const int64_t row = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / V;
  T acc[D];
  row_product<T, D, V>(M, v, row, lane, acc);
  if (lane == 0 && row < M.nrows) store_row<T, D>(y + row * D, acc);
}

// Lanczos step product (Alg. 2 (the block recurrence)):  Q' = M v + eps D x - Q_{j-1} Gamma_{j-1}^T
// and Xi_j = sym(Q_j^T Q'); the block that finishes last reduces Xi_j.
template <typename T, int D, int V>
__global__ void __launch_bounds__(kThreads) k_spmm_lanczos(Csr<T> M, const T* __restrict__ v, StepOps<T> op,
                                                           Red red) {
  constexpr int RPB = kThreads / V;
  constexpr int NP = D * D;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  __shared__ T g_s[D * D];
  if (threadIdx.x < D * D) g_s[threadIdx.x] = op.gprev ? (T)op.gprev[threadIdx.x] : T(0);
  __syncthreads();
  const int lane = threadIdx.x % V, grp = threadIdx.x / V;
  const bool has_prev = op.qprev != nullptr;
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  for (int64_t tile = blockIdx.x; tile * RPB < M.nrows; tile += gridDim.x) {
    const int64_t row = tile * RPB + grp;
    // epilogue operands do not depend on the gather: issue their loads first
    T xi[D], qp[D];
    T de = T(0);
    const bool lead = (lane == 0 && row < M.nrows);
    if (lead) {
      load_row<T, D>(op.x + row * D, xi);
      de = (T)op.eps * __ldg(op.Dv + row);
      if (has_prev) load_row<T, D>(op.qprev + row * D, qp);
    }
    T acc[D];
    row_product<T, D, V>(M, v, row, lane, acc);
    if (lead) {
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = fma(de, xi[q], acc[q]);
      if (has_prev) {
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) acc[r] = fma(-qp[c], g_s[r * D + c], acc[r]);
      }
      store_row<T, D>(op.out + row * D, acc);
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) part[a * D + b] = fma(xi[a], acc[b], part[a * D + b]);
    }
  }
  double pd[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
  block_sum<NP>(pd, red_s, tot);
  if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, NP, red.ticket, tot, red_s)) {
    if (threadIdx.x == 0) {
      double X[D * D];
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) X[a * D + b] = 0.5 * (tot[a * D + b] + tot[b * D + a]);
      for (int k = 0; k < D * D; ++k) op.xi[k] = X[k];
      *op.xi_norm = sym_norm2(X, D);
    }
  }
}

// ---------------------------------------------------------------------------
// Sliced ELLPACK schedule (code kSchedSell): a warp takes a slice of kSellC
// consecutive rows, lane l its row kSellC s + l.  Entry j of all the slice's rows
// is one contiguous kSellC-wide run of col / val, so every warp load of the
// structure is a single coalesced access; only the gathers of v are scattered.
// Four entries per lane are in flight at a time.
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void sell_row(const Csr<T>& M, const T* __restrict__ v, int64_t slice, int lane,
                                         T (&acc)[D]) {
#pragma unroll
  for (int q = 0; q < D; ++q) acc[q] = T(0);
  const int64_t p0 = __ldg(M.sptr + slice);
  const int64_t len = (__ldg(M.sptr + slice + 1) - p0) / kSellC;
  const int* cp = M.scol + p0 + lane;
  const T* vp = M.sval + p0 + lane;
  int64_t j = 0;
  for (; j + 4 <= len; j += 4) {
    int c[4];
    T a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c[u] = __ldg(cp + (j + u) * kSellC);
      a[u] = __ldg(vp + (j + u) * kSellC);
    }
    T xv[4][D];
#pragma unroll
    for (int u = 0; u < 4; ++u) load_row<T, D>(v + (int64_t)c[u] * D, xv[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = fma(a[u], xv[u][q], acc[q]);
  }
  for (; j < len; ++j) {
    const int c = __ldg(cp + j * kSellC);
    const T a = __ldg(vp + j * kSellC);
    T xv[D];
    load_row<T, D>(v + (int64_t)c * D, xv);
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = fma(a, xv[q], acc[q]);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_spmm_plain_sell(Csr<T> M, const T* __restrict__ v, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t nslices = (M.nrows + kSellC - 1) / kSellC;
  const int64_t wid = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t sl = wid; sl < nslices; sl += nw) {
    T acc[D];
    sell_row<T, D>(M, v, sl, lane, acc);
    const int64_t row = sl * kSellC + lane;
    if (row < M.nrows) store_row<T, D>(y + row * D, acc);
  }
}

// the Lanczos step product of k_spmm_lanczos on the sliced layout (same epilogue)
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_spmm_lanczos_sell(Csr<T> M, const T* __restrict__ v, StepOps<T> op,
                                                                Red red) {
  constexpr int NP = D * D;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  __shared__ T g_s[D * D];
  if (threadIdx.x < D * D) g_s[threadIdx.x] = op.gprev ? (T)op.gprev[threadIdx.x] : T(0);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const bool has_prev = op.qprev != nullptr;
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  const int64_t nslices = (M.nrows + kSellC - 1) / kSellC;
  const int64_t wid = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t sl = wid; sl < nslices; sl += nw) {
    const int64_t row = sl * kSellC + lane;
    const bool lead = row < M.nrows;
    T xi[D], qp[D];
    T de = T(0);
    if (lead) {  // epilogue operands first: they do not depend on the gathers
      load_row<T, D>(op.x + row * D, xi);
      de = (T)op.eps * __ldg(op.Dv + row);
      if (has_prev) load_row<T, D>(op.qprev + row * D, qp);
    }
    T acc[D];
    sell_row<T, D>(M, v, sl, lane, acc);
    if (lead) {
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = fma(de, xi[q], acc[q]);
      if (has_prev) {
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int c = 0; c < D; ++c) acc[r] = fma(-qp[c], g_s[r * D + c], acc[r]);
      }
      store_row<T, D>(op.out + row * D, acc);
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) part[a * D + b] = fma(xi[a], acc[b], part[a * D + b]);
    }
  }
  double pd[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
  block_sum<NP>(pd, red_s, tot);
  if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, NP, red.ticket, tot, red_s)) {
    if (threadIdx.x == 0) {
      double X[D * D];
      for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) X[a * D + b] = 0.5 * (tot[a * D + b] + tot[b * D + a]);
      for (int k = 0; k < D * D; ++k) op.xi[k] = X[k];
      *op.xi_norm = sym_norm2(X, D);
    }
  }
}

// slice lengths: the longest row of each slice
__global__ void k_sell_len(const int64_t* __restrict__ rowptr, int64_t nrows, int* __restrict__ len) {
  const int64_t nslices = (nrows + kSellC - 1) / kSellC;
  for (int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; sl < nslices;
       sl += (int64_t)gridDim.x * blockDim.x) {
    int64_t mx = 0;
    for (int l = 0; l < kSellC; ++l) {
      const int64_t r = sl * kSellC + l;
      if (r < nrows) mx = max(mx, rowptr[r + 1] - rowptr[r]);
    }
    len[sl] = (int)mx;
  }
}

// padded column-major copy: lane l of slice s writes entry j of row kSellC s + l
__global__ void k_sell_fill(const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, int64_t nrows, const int64_t* __restrict__ sptr,
                            int* __restrict__ scol, double* __restrict__ sval) {
  const int64_t nslices = (nrows + kSellC - 1) / kSellC;
  const int64_t total = nslices * kSellC;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sl = t / kSellC, r = t;
    const int l = (int)(t % kSellC);
    const int64_t p0 = sptr[sl], len = (sptr[sl + 1] - p0) / kSellC;
    const int64_t s = r < nrows ? rowptr[r] : 0, e = r < nrows ? rowptr[r + 1] : 0;
    for (int64_t j = 0; j < len; ++j) {
      const bool real = s + j < e;
      scol[p0 + j * kSellC + l] = real ? col[s + j] : 0;
      sval[p0 + j * kSellC + l] = real ? val[s + j] : 0.0;
    }
  }
}

void sell_lengths(const int64_t* rowptr, int64_t nrows, int* slice_len, cudaStream_t s) {
  const int64_t nslices = (nrows + kSellC - 1) / kSellC;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((nslices + 255) / 256, 152 * 16));
  k_sell_len<<<g, 256, 0, s>>>(rowptr, nrows, slice_len);
}

void sell_fill(const int64_t* rowptr, const int* col, const double* val, int64_t nrows, const int64_t* sptr,
               int* scol, double* sval, cudaStream_t s) {
  const int64_t total = (nrows + kSellC - 1) / kSellC * kSellC;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_sell_fill<<<g, 256, 0, s>>>(rowptr, col, val, nrows, sptr, scol, sval);
}

static int sell_grid(int64_t nrows) {
  const int64_t nslices = (nrows + kSellC - 1) / kSellC;
  const int64_t blocks = (nslices + (kThreads / 32) - 1) / (kThreads / 32);
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, kMaxBlocks));
}

// y = M v and per-column dots sum_i w_i[c] y_i[c] (w defaults to the rows of v) or
// squared norms sum_i y_i[c]^2 (sq = 1); used by the CG / CGLS refinement.
template <typename T, int D, int V>
__global__ void __launch_bounds__(kThreads) k_spmm_coldot(Csr<T> M, const T* __restrict__ v, T* __restrict__ y,
                                                          const T* __restrict__ w, int sq, Red red, double* dots) {
  constexpr int RPB = kThreads / V;
  __shared__ double red_s[(kThreads / 32) * D];
  __shared__ double tot[D];
  const int lane = threadIdx.x % V, grp = threadIdx.x / V;
  double part[D];
#pragma unroll
  for (int k = 0; k < D; ++k) part[k] = 0.0;
  const T* wv = w ? w : v;
  for (int64_t tile = blockIdx.x; tile * RPB < M.nrows; tile += gridDim.x) {
    const int64_t row = tile * RPB + grp;
    T acc[D];
    row_product<T, D, V>(M, v, row, lane, acc);
    if (lane == 0 && row < M.nrows) {
      store_row<T, D>(y + row * D, acc);
      if (sq) {
#pragma unroll
        for (int q = 0; q < D; ++q) part[q] += (double)acc[q] * (double)acc[q];
      } else {
        T wr[D];
        load_row<T, D>(wv + row * D, wr);
#pragma unroll
        for (int q = 0; q < D; ++q) part[q] += (double)wr[q] * (double)acc[q];
      }
    }
  }
  block_sum<D>(part, red_s, tot);
  if (threadIdx.x < D) red.part[(size_t)blockIdx.x * D + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, D, red.ticket, tot, red_s)) {
    if (threadIdx.x < D) dots[threadIdx.x] = tot[threadIdx.x];
  }
}

// The same product for wide panels (the refinement's 16 columns): D lanes per row,
// lane c owning column c, so a gathered row of the panel is one coalesced D-wide
// access and no cross-lane reduction is needed.  The nonzeros of a row are walked
// four at a time (their column indices, then the four gathers, are in flight
// together).  Each thread keeps its column's dot product (FP32 partials for FP32
// data, FP64 for FP64), reduced per column in shared memory and across blocks.
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_spmm_panel(Csr<T> M, const T* __restrict__ v, T* __restrict__ y,
                                                         const T* __restrict__ w, int sq, Red red, double* dots) {
  static_assert(kThreads % D == 0 && 32 % D == 0, "D lanes per row within a warp");
  constexpr int RPB = kThreads / D;
  __shared__ double red_s[kThreads];
  __shared__ double tot[D];
  const int c = threadIdx.x % D, grp = threadIdx.x / D;
  const T* wv = w ? w : v;
  T part = T(0);
  for (int64_t tile = blockIdx.x; tile * RPB < M.nrows; tile += gridDim.x) {
    const int64_t row = tile * RPB + grp;
    if (row < M.nrows) {
      const int64_t s = __ldg(M.rowptr + row), e = __ldg(M.rowptr + row + 1);
      T acc = T(0);
      int64_t k = s;
      for (; k + 4 <= e; k += 4) {
        int col[4];
        T a[4], x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          col[u] = __ldg(M.col + k + u);
          a[u] = __ldg(M.val + k + u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __ldg(v + (int64_t)col[u] * D + c);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = fma(a[u], x[u], acc);
      }
      for (; k < e; ++k) acc = fma(__ldg(M.val + k), __ldg(v + (int64_t)__ldg(M.col + k) * D + c), acc);
      y[row * D + c] = acc;
      part = sq ? fma(acc, acc, part) : fma(__ldg(wv + row * D + c), acc, part);
    }
  }
  red_s[threadIdx.x] = (double)part;
  __syncthreads();
  if (threadIdx.x < D) {
    double sum = 0.0;
    for (int j = threadIdx.x; j < kThreads; j += D) sum += red_s[j];
    tot[threadIdx.x] = sum;
  }
  __syncthreads();
  if (threadIdx.x < D) red.part[(size_t)blockIdx.x * D + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, D, red.ticket, tot, red_s))
    if (threadIdx.x < D) dots[threadIdx.x] = tot[threadIdx.x];
}

// ---------------------------------------------------------------------------
// TMA-staged schedule (lanes code kSchedTma): a CTA takes kTmaRows consecutive
// rows per tile.  One thread copies the tile's col/val segment (the 16-byte
// aligned span around it; the CSR arrays carry kCsrPad entries of padding) into
// shared memory with cp.async.bulk, completing on an mbarrier, one tile ahead of
// the CTA (double buffer).  Every thread then owns one row: its col/val come
// from shared memory, so the only global loads left in the loop are the x
// gathers, up to eight of them in flight per thread.  A tile whose segment exceeds
// kTmaCap entries is read from global memory directly.  The mbarrier wait is
// bounded: on expiry the kernel counts it in g_wait_timeouts and the CTA stops.
// ---------------------------------------------------------------------------
constexpr int kTmaRows = kThreads;
constexpr int kTmaCap = 3072;
constexpr int kTmaSlot = kTmaCap + 8;  // aligned span of kTmaCap entries + slack
constexpr unsigned kWaitLimit = 1u << 22;  // tries of a bounded mbarrier wait

__device__ unsigned g_wait_timeouts;

struct TmaTile {
  int64_t s, e;    // segment of the tile
  int64_t cs, vs;  // first staged entry of col / val
  int staged;
  int pad;
};

template <typename T>
constexpr size_t tma_smem_bytes() {
  return 256 + 2 * (size_t)kTmaSlot * (sizeof(int) + sizeof(T));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// non-blocking test with a short sleep between tries: at most kWaitLimit tries
// (well under a second), then false
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// thread 0: describe tile `tile` in info and, if it fits, start its bulk copies
template <typename T>
__device__ __forceinline__ void tma_issue(const Csr<T>& M, int64_t tile, TmaTile& info, int* col_s, T* val_s,
                                          uint32_t bar) {
  const int64_t r0 = tile * kTmaRows;
  const int64_t r1 = (r0 + kTmaRows < M.nrows) ? r0 + kTmaRows : M.nrows;
  const int64_t s = __ldg(M.rowptr + r0), e = __ldg(M.rowptr + r1);
  constexpr int64_t va = 16 / (int64_t)sizeof(T);  // entries per 16 bytes
  const int64_t cs = s & ~(int64_t)3, ce = (e + 3) & ~(int64_t)3;
  const int64_t vs = s & ~(va - 1), ve = (e + va - 1) & ~(va - 1);
  info.s = s;
  info.e = e;
  info.cs = cs;
  info.vs = vs;
  info.staged = (e > s && e - s <= kTmaCap) ? 1 : 0;
  if (!info.staged) return;
  const uint32_t bc = (uint32_t)(4 * (ce - cs)), bv = (uint32_t)(sizeof(T) * (ve - vs));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bc + bv) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(col_s)),
               "l"(M.col + cs), "r"(bc), "r"(bar)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(val_s)),
               "l"(M.val + vs), "r"(bv), "r"(bar)
               : "memory");
}

// LANCZOS = true: the fused Lanczos step (eps D x, -Q_{j-1} Gamma^T, Xi partials);
// false: y = M v.
template <typename T, int D, bool LANCZOS>
__global__ void __launch_bounds__(kThreads) k_spmm_tma(Csr<T> M, const T* __restrict__ v, StepOps<T> op, T* y,
                                                       Red red) {
  constexpr int NP = D * D;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);     // 2 mbarriers
  TmaTile* info = reinterpret_cast<TmaTile*>(smem_raw + 64);  // 2 tiles
  int* col_s = reinterpret_cast<int*>(smem_raw + 256);        // 2 x kTmaSlot
  T* val_s = reinterpret_cast<T*>(smem_raw + 256 + 2 * (size_t)kTmaSlot * sizeof(int));
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  __shared__ T g_s[D * D];
  __shared__ int abort_s;
  const int tid = threadIdx.x;
  const int64_t ntiles = (M.nrows + kTmaRows - 1) / kTmaRows;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_s = 0;
  }
  if constexpr (LANCZOS) {
    if (tid < D * D) g_s[tid] = op.gprev ? (T)op.gprev[tid] : T(0);
  }
  __syncthreads();
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) tma_issue<T>(M, blockIdx.x, info[0], col_s, val_s, smem_u32(bars));
  __syncthreads();
  const bool has_prev = LANCZOS && op.qprev != nullptr;
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  uint32_t par0 = 0u, par1 = 0u;  // phase parity of each mbarrier
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it & 1;
    if (tid == 0 && tile + gridDim.x < ntiles)  // next tile into the other buffer (consumed last iteration)
      tma_issue<T>(M, tile + gridDim.x, info[b ^ 1], col_s + (b ^ 1) * kTmaSlot, val_s + (b ^ 1) * kTmaSlot,
                   smem_u32(bars + (b ^ 1)));
    const int64_t row = tile * kTmaRows + tid;
    const bool own = row < M.nrows;
    int64_t rs = 0, re = 0;
    T xi[D], qp[D];
    T de = T(0);
    if (own) {  // row bounds and epilogue operands first: independent of the staging
      rs = __ldg(M.rowptr + row);
      re = __ldg(M.rowptr + row + 1);
      if constexpr (LANCZOS) {
        load_row<T, D>(op.x + row * D, xi);
        de = (T)op.eps * __ldg(op.Dv + row);
        if (has_prev) load_row<T, D>(op.qprev + row * D, qp);
      }
    }
    const TmaTile ti = info[b];
    const bool prefetched = tile + gridDim.x < ntiles && info[b ^ 1].staged;
    if (ti.staged) {
      if (!mbar_wait_bounded(smem_u32(bars + b), b ? par1 : par0)) {
        if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
        abort_s = 1;
      }
      if (b)
        par1 ^= 1u;
      else
        par0 ^= 1u;
    }
    __syncthreads();
    if (abort_s) {  // leave no bulk copy in flight into this CTA's shared memory
      if (tid == 0 && prefetched) mbar_wait_bounded(smem_u32(bars + (b ^ 1)), b ? par0 : par1);
      return;
    }
    T acc[D];
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = T(0);
    if (own) {
      const int* cp = ti.staged ? col_s + b * kTmaSlot - ti.cs : M.col;
      const T* vp = ti.staged ? val_s + b * kTmaSlot - ti.vs : M.val;
      constexpr int U = D >= 8 ? 2 : (D >= 4 ? 4 : 8);  // independent gathers in flight per thread
      int64_t k = rs;
      for (; k + U <= re; k += U) {
        int c[U];
        T a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          c[u] = cp[k + u];
          a[u] = vp[k + u];
        }
        T xv[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) load_row<T, D>(v + (int64_t)c[u] * D, xv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int q = 0; q < D; ++q) acc[q] = fma(a[u], xv[u][q], acc[q]);
      }
      if (k < re) {  // tail of fewer than U entries, loads first
        const int nt = (int)(re - k);
        int c[U];
        T a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          c[u] = u < nt ? cp[k + u] : 0;
          a[u] = u < nt ? vp[k + u] : T(0);
        }
        T xv[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (u < nt) {
            load_row<T, D>(v + (int64_t)c[u] * D, xv[u]);
          } else {
#pragma unroll
            for (int q = 0; q < D; ++q) xv[u][q] = T(0);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int q = 0; q < D; ++q) acc[q] = fma(a[u], xv[u][q], acc[q]);
      }
      if constexpr (LANCZOS) {
#pragma unroll
        for (int q = 0; q < D; ++q) acc[q] = fma(de, xi[q], acc[q]);
        if (has_prev) {
#pragma unroll
          for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) acc[r] = fma(-qp[c], g_s[r * D + c], acc[r]);
        }
        store_row<T, D>(op.out + row * D, acc);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int bb = 0; bb < D; ++bb) part[a * D + bb] = fma(xi[a], acc[bb], part[a * D + bb]);
      } else {
        store_row<T, D>(y + row * D, acc);
      }
    }
    __syncthreads();  // buffer b is refilled next iteration
  }
  if constexpr (LANCZOS) {
    double pd[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
    block_sum<NP>(pd, red_s, tot);
    if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
    if (last_block_reduce(red.part, NP, red.ticket, tot, red_s)) {
      if (threadIdx.x == 0) {
        double X[D * D];
        for (int a = 0; a < D; ++a)
          for (int bb = 0; bb < D; ++bb) X[a * D + bb] = 0.5 * (tot[a * D + bb] + tot[bb * D + a]);
        for (int k = 0; k < D * D; ++k) op.xi[k] = X[k];
        *op.xi_norm = sym_norm2(X, D);
      }
    }
  }
}

template <typename T, int D, bool LANCZOS>
static void launch_tma(const Csr<T>& M, const T* v, const StepOps<T>& op, T* y, const Red& red, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_spmm_tma<T, D, LANCZOS>);
  // the shared-memory limit is a per-device attribute: raised on each device in turn
  if (ensure_smem_limit(fn, tma_smem_bytes<T>()) != cudaSuccess) return;  // the caller's launch check reports it
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, tma_smem_bytes<T>());
  const int cap = std::max(1, std::min(per_sm, 8)) * std::max(sms, 1);  // resident CTAs of this instantiation
  const int64_t ntiles = (M.nrows + kTmaRows - 1) / kTmaRows;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, cap));
  k_spmm_tma<T, D, LANCZOS><<<grid, kThreads, tma_smem_bytes<T>(), s>>>(M, v, op, y, red);
}

unsigned spmm_wait_timeouts(bool clear) {
  unsigned v = 0;
  cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(unsigned));
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_wait_timeouts, &z, sizeof(unsigned));
  }
  return v;
}

#define NS_LANES_SWITCH(V, CALL) \
  switch (V) {                   \
    case 1: CALL(1); break;      \
    case 2: CALL(2); break;      \
    case 4: CALL(4); break;      \
    case 8: CALL(8); break;      \
    case 16: CALL(16); break;    \
    default: CALL(32); break;    \
  }

template <typename T, int D>
void spmm_plain(const Csr<T>& M, const T* v, T* y, cudaStream_t s) {
  if (M.nrows == 0) return;
  if (M.V == kSchedSell && M.sptr) {
    k_spmm_plain_sell<T, D><<<sell_grid(M.nrows), kThreads, 0, s>>>(M, v, y);
    return;
  }
  if (M.V == kSchedTma) {
    launch_tma<T, D, false>(M, v, StepOps<T>{}, y, Red{}, s);
    return;
  }
  const int grid = ceil_div(M.nrows * (int64_t)M.V, kThreads);
#define CALL(VV) k_spmm_plain<T, D, VV><<<grid, kThreads, 0, s>>>(M, v, y)
  NS_LANES_SWITCH(M.V, CALL)
#undef CALL
}

static int persistent_grid(int64_t nrows, int V) {
  const int64_t tiles = (nrows + (kThreads / V) - 1) / (kThreads / V);
  return (int)(tiles < kMaxBlocks ? (tiles > 0 ? tiles : 1) : kMaxBlocks);
}

template <typename T, int D>
void spmm_lanczos(const Csr<T>& M, const T* v, const StepOps<T>& op, const Red& red, cudaStream_t s) {
  if (M.V == kSchedSell && M.sptr) {
    k_spmm_lanczos_sell<T, D><<<sell_grid(M.nrows), kThreads, 0, s>>>(M, v, op, red);
    return;
  }
  if (M.V == kSchedTma) {
    launch_tma<T, D, true>(M, v, op, nullptr, red, s);
    return;
  }
  const int grid = persistent_grid(M.nrows, M.V);
#define CALL(VV) k_spmm_lanczos<T, D, VV><<<grid, kThreads, 0, s>>>(M, v, op, red)
  NS_LANES_SWITCH(M.V, CALL)
#undef CALL
}

template <typename T, int D>
void spmm_coldot(const Csr<T>& M, const T* v, T* y, const T* w, int sq, double* dots, const Red& red,
                 cudaStream_t s) {
  if constexpr (D == 16) {  // wide refinement panels: a lane per column
    k_spmm_panel<T, D><<<persistent_grid(M.nrows, D), kThreads, 0, s>>>(M, v, y, w, sq, red, dots);
    return;
  }
  const int V = (M.V == kSchedTma || M.V == kSchedSell) ? 1 : M.V;  // those serve the step products only
  const int grid = persistent_grid(M.nrows, V);
#define CALL(VV) k_spmm_coldot<T, D, VV><<<grid, kThreads, 0, s>>>(M, v, y, w, sq, red, dots)
  NS_LANES_SWITCH(V, CALL)
#undef CALL
}

// SpMM schedule autotuner: time y = M v for the TMA-staged schedule and V in
// {1, 2, 4, 8, 16} lanes per row
// on the actual matrix (CUDA events, one warm-up + two timed launches each) and
// return the fastest.
template <typename T, int D>
int tune_lanes(Csr<T> M, const T* v, T* y, cudaStream_t s) {
  if (M.nrows == 0) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = M.V;
  float best_ms = 1e30f;
  for (int V : {kSchedSell, kSchedTma, 1, 2, 4, 8, 16}) {
    if (V == kSchedSell && !M.sptr) continue;
    M.V = V;
    spmm_plain<T, D>(M, v, y, s);
    cudaEventRecord(e0, s);
    spmm_plain<T, D>(M, v, y, s);
    spmm_plain<T, D>(M, v, y, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = V;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

#define NS_INST_SPMM(T, D)                                                                            \
  template void spmm_plain<T, D>(const Csr<T>&, const T*, T*, cudaStream_t);                          \
  template void spmm_lanczos<T, D>(const Csr<T>&, const T*, const StepOps<T>&, const Red&, cudaStream_t); \
  template void spmm_coldot<T, D>(const Csr<T>&, const T*, T*, const T*, int, double*, const Red&, cudaStream_t); \
  template int tune_lanes<T, D>(Csr<T>, const T*, T*, cudaStream_t);
NS_INST_SPMM(double, 1)
NS_INST_SPMM(double, 2)
NS_INST_SPMM(double, 4)
NS_INST_SPMM(double, 8)
NS_INST_SPMM(float, 1)
NS_INST_SPMM(float, 2)
NS_INST_SPMM(float, 4)
NS_INST_SPMM(float, 8)
// wide panels for the refinement (column dots only)
template void spmm_coldot<double, 16>(const Csr<double>&, const double*, double*, const double*, int, double*,
                                      const Red&, cudaStream_t);
template void spmm_coldot<float, 16>(const Csr<float>&, const float*, float*, const float*, int, double*, const Red&,
                                     cudaStream_t);

// ---------------------------------------------------------------------------
// validation, norms, conversions
// ---------------------------------------------------------------------------
__global__ void k_validate(const int64_t* rowptr, const int* col, const double* val, int64_t m, int64_t n,
                           int64_t nnz, unsigned* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > m) return;
  if (r == 0 && rowptr[0] != 0) atomicOr(err, 1u);
  if (r == m) {
    if (rowptr[m] != nnz) atomicOr(err, 1u);
    return;
  }
  const int64_t s = rowptr[r], e = rowptr[r + 1];
  if (s > e || s < 0 || e > nnz) {
    atomicOr(err, 1u);
    return;
  }
  unsigned bad = 0;
  for (int64_t k = s; k < e; ++k) {
    const int c = col[k];
    if (c < 0 || (int64_t)c >= n) bad |= 2u;
    if (!isfinite(val[k])) bad |= 4u;
  }
  if (bad) atomicOr(err, bad);
}

void csr_validate(const int64_t* rowptr, const int* col, const double* val, int64_t m, int64_t n, int64_t nnz,
                  unsigned* err, cudaStream_t s) {
  k_validate<<<ceil_div(m + 1, kThreads), kThreads, 0, s>>>(rowptr, col, val, m, n, nnz, err);
}

__global__ void k_max_abs_row_sum(const int64_t* rowptr, const double* val, int64_t m, Red red, double* out) {
  __shared__ double red_s[kThreads / 32];
  __shared__ double tot[1];
  double mx = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += fabs(val[k]);
    mx = fmax(mx, s);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) red_s[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red_s[w]);
    red.part[blockIdx.x] = t;
  }
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(red.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t = fmax(t, __ldcg(red.part + b));
    *out = t;
    *red.ticket = 0u;
  }
}

void csr_max_abs_row_sum(const int64_t* rowptr, const double* val, int64_t m, double* out, const Red& red,
                         cudaStream_t s) {
  int grid = ceil_div(m, kThreads);
  if (grid > kMaxBlocks) grid = kMaxBlocks;
  if (grid < 1) grid = 1;
  k_max_abs_row_sum<<<grid, kThreads, 0, s>>>(rowptr, val, m, red, out);
}

__global__ void k_d2f(const double* a, float* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(const float* a, double* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
static int stream_grid(int64_t n) {
  int g = ceil_div(n, kThreads);
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : g;
}
void convert_d2f(const double* a, float* b, int64_t n, cudaStream_t s) {
  if (n > 0) k_d2f<<<stream_grid(n), kThreads, 0, s>>>(a, b, n);
}
void convert_f2d(const float* a, double* b, int64_t n, cudaStream_t s) {
  if (n > 0) k_f2d<<<stream_grid(n), kThreads, 0, s>>>(a, b, n);
}

// ---------------------------------------------------------------------------
// explicit transpose: column histogram -> exclusive scan -> scatter -> per-row
// sort by original position (so row i of A^T lists the rows of A in order)
// ---------------------------------------------------------------------------
__global__ void k_count_cols(const int* col, int64_t nnz, int* count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(count + col[e], 1);
}

constexpr int kScanChunk = 4096;

__global__ void k_chunk_totals(const int* count, int64_t n, int64_t* totals) {
  __shared__ double red_s[kThreads / 32];
  __shared__ double tot[1];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  double s = 0.0;
  for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x)
    if (base + i < n) s += (double)count[base + i];
  double v[1] = {s};
  block_sum<1>(v, red_s, tot);
  if (threadIdx.x == 0) totals[blockIdx.x] = (int64_t)tot[0];
}

__global__ void k_scan_totals(int64_t* totals, int nchunks) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int b = 0; b < nchunks; ++b) {
      const int64_t t = totals[b];
      totals[b] = run;
      run += t;
    }
  }
}

// rowptr_t[i+1] = offset(chunk) + inclusive prefix of count within the chunk
__global__ void k_chunk_scan(const int* count, int64_t n, const int64_t* offs, int64_t* rowptr_t) {
  constexpr int PER = kScanChunk / kThreads;  // 16
  __shared__ int64_t tsum[kThreads];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * PER;
  int64_t loc[PER];
  int64_t run = 0;
  for (int k = 0; k < PER; ++k) {
    run += (base + k < n) ? count[base + k] : 0;
    loc[k] = run;
  }
  tsum[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int t = 0; t < kThreads; ++t) {
      const int64_t v = tsum[t];
      tsum[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  const int64_t off = offs[blockIdx.x] + tsum[threadIdx.x];
  for (int k = 0; k < PER; ++k)
    if (base + k < n) rowptr_t[base + k + 1] = off + loc[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) rowptr_t[0] = 0;
}

__global__ void k_scatter(const int64_t* rowptr, const int* col, int64_t m, unsigned long long* cursor,
                          int64_t* perm, int* rowof) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      const unsigned long long pos = atomicAdd(cursor + col[e], 1ull);
      perm[pos] = e;
      rowof[pos] = (int)r;
    }
  }
}

__global__ void k_sort_rows(const int64_t* rowptr_t, int64_t n, int64_t* perm, int* rowof) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rowptr_t[r], e = rowptr_t[r + 1];
    for (int64_t i = s + 1; i < e; ++i) {  // insertion sort by original position
      const int64_t key = perm[i];
      const int ro = rowof[i];
      int64_t j = i - 1;
      while (j >= s && perm[j] > key) {
        perm[j + 1] = perm[j];
        rowof[j + 1] = rowof[j];
        --j;
      }
      perm[j + 1] = key;
      rowof[j + 1] = ro;
    }
  }
}

__global__ void k_gather_t(const int64_t* perm, const int* rowof, const double* val, int64_t nnz, int* col_t,
                           double* val_t) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
    col_t[p] = rowof[p];
    val_t[p] = val[perm[p]];
  }
}

__global__ void k_copy_i64_to_u64(const int64_t* a, unsigned long long* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (unsigned long long)a[i];
}

void csr_transpose(const int64_t* rowptr, const int* col, const double* val, int64_t m, int64_t n, int64_t nnz,
                   int64_t* rowptr_t, int* col_t, double* val_t, const TransposeWork& w, cudaStream_t s) {
  cudaMemsetAsync(w.count, 0, sizeof(int) * (size_t)(n + 1), s);
  if (nnz > 0) k_count_cols<<<stream_grid(nnz), kThreads, 0, s>>>(col, nnz, w.count);
  const int nchunks = ceil_div(n, kScanChunk);
  k_chunk_totals<<<nchunks, kThreads, 0, s>>>(w.count, n, w.blocksum);
  k_scan_totals<<<1, 32, 0, s>>>(w.blocksum, nchunks);
  k_chunk_scan<<<nchunks, kThreads, 0, s>>>(w.count, n, w.blocksum, rowptr_t);
  k_copy_i64_to_u64<<<stream_grid(n), kThreads, 0, s>>>(rowptr_t, (unsigned long long*)w.cursor, n);
  if (m > 0) k_scatter<<<stream_grid(m), kThreads, 0, s>>>(rowptr, col, m, (unsigned long long*)w.cursor, w.perm, w.rowof);
  k_sort_rows<<<stream_grid(n), kThreads, 0, s>>>(rowptr_t, n, w.perm, w.rowof);
  if (nnz > 0) k_gather_t<<<stream_grid(nnz), kThreads, 0, s>>>(w.perm, w.rowof, val, nnz, col_t, val_t);
}

}  // namespace ns

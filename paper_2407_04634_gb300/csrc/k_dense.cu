// Dense kernels of the Lanczos loop: random streams, block QR (CholQR2),
// CGS2 projections for partial reorthogonalization (Sec. 4.2), the W recurrence
// (one block), thick-restart GEMM and bookkeeping (Sec. 4.1), CG refinement.
#include "ns_common.cuh"
#include "ns_kernels.cuh"

#include <algorithm>
#include <type_traits>
#include <vector>

namespace ns {

static int stream_grid(int64_t n, int cap = 152 * 16) {
  int g = ceil_div(n, kThreads);
  if (g > cap) g = cap;
  return g < 1 ? 1 : g;
}
static int persistent_rows(int64_t n) { return stream_grid(n, kMaxBlocks); }

// ---------------------------------------------------------------------------
// Philox streams: uniforms (stream 0: D) and Box-Muller normals (stream 1: Omega)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_rng_uniform(uint64_t seed, uint32_t stream, T* out, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const U4 w = philox_at(seed, stream, (uint64_t)i);
    out[i] = (T)u53(w.x, w.y);
  }
}

template <typename T>
__global__ void k_rng_gauss(uint64_t seed, uint32_t stream, T* out, int64_t count) {
  const int64_t npairs = (count + 1) / 2;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * blockDim.x) {
    const U4 w = philox_at(seed, stream, (uint64_t)p);
    const uint64_t w0 = (uint64_t)w.x | ((uint64_t)w.y << 32);
    const uint64_t w1 = (uint64_t)w.z | ((uint64_t)w.w << 32);
    const double u1 = (double)((w0 >> 11) + 1) * 0x1.0p-53;
    const double u2 = (double)(w1 >> 11) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    out[2 * p] = (T)(r * cs);
    if (2 * p + 1 < count) out[2 * p + 1] = (T)(r * sn);
  }
}

template <typename T>
void rng_uniform(uint64_t seed, uint32_t stream, T* out, int64_t count, cudaStream_t s) {
  if (count > 0) k_rng_uniform<T><<<stream_grid(count), kThreads, 0, s>>>(seed, stream, out, count);
}
template <typename T>
void rng_gauss(uint64_t seed, uint32_t stream, T* out, int64_t count, cudaStream_t s) {
  if (count > 0) k_rng_gauss<T><<<stream_grid((count + 1) / 2), kThreads, 0, s>>>(seed, stream, out, count);
}
template void rng_uniform<double>(uint64_t, uint32_t, double*, int64_t, cudaStream_t);
template void rng_uniform<float>(uint64_t, uint32_t, float*, int64_t, cudaStream_t);
template void rng_gauss<double>(uint64_t, uint32_t, double*, int64_t, cudaStream_t);
template void rng_gauss<float>(uint64_t, uint32_t, float*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// CholQR passes on n x D panels
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_axpy_gram(T* __restrict__ qp, const T* __restrict__ x,
                                                        const double* __restrict__ Xi, int64_t n, double* R1,
                                                        unsigned* flags, Red red) {
  constexpr int NP = D * D;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  __shared__ T xi_s[NP];
  if (threadIdx.x < NP) xi_s[threadIdx.x] = (T)Xi[threadIdx.x];
  __syncthreads();
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T q[D], xr[D];
    load_row<T, D>(qp + i * D, q);
    load_row<T, D>(x + i * D, xr);
#pragma unroll
    for (int b = 0; b < D; ++b)
#pragma unroll
      for (int a = 0; a < D; ++a) q[b] = fma(-xr[a], xi_s[a * D + b], q[b]);
    store_row<T, D>(qp + i * D, q);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) part[a * D + b] = fma(q[a], q[b], part[a * D + b]);
  }
  double pd[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
  block_sum<NP>(pd, red_s, tot);
  if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, NP, red.ticket, tot, red_s))
    if (threadIdx.x == 0) finish_chol(tot, D, R1, nullptr, flags);
}

template <typename T, int D>
void axpy_gram(T* qp, const T* x, const double* Xi, int64_t n, double* R1, unsigned* flags, const Red& red,
               cudaStream_t s) {
  k_axpy_gram<T, D><<<persistent_rows(n), kThreads, 0, s>>>(qp, x, Xi, n, R1, flags, red);
}

// out = in R^{-1}; optional Gram of out with Cholesky into R2
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_scale_gram(const T* in, int64_t ldin, T* out, int64_t ldout,
                                                         const double* __restrict__ R, int64_t n, double* R2,
                                                         unsigned* flags, Red red) {
  constexpr int NP = D * D;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  __shared__ T ri_s[NP];
  if (threadIdx.x == 0) {
    double Rl[NP], Ri[NP];
    for (int k = 0; k < NP; ++k) Rl[k] = R[k];
    inv_upper(Rl, Ri, D);
    for (int k = 0; k < NP; ++k) ri_s[k] = (T)Ri[k];
  }
  __syncthreads();
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T a[D], o[D];
#pragma unroll
    for (int k = 0; k < D; ++k) a[k] = in[i * ldin + k];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k <= c; ++k) s = fma(a[k], ri_s[k * D + c], s);
      o[c] = s;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) out[i * ldout + k] = o[k];
    if (R2) {
#pragma unroll
      for (int p = 0; p < D; ++p)
#pragma unroll
        for (int q = 0; q < D; ++q) part[p * D + q] = fma(o[p], o[q], part[p * D + q]);
    }
  }
  if (!R2) return;  // uniform across the grid
  double pd[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
  block_sum<NP>(pd, red_s, tot);
  if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, NP, red.ticket, tot, red_s))
    if (threadIdx.x == 0) finish_chol(tot, D, R2, nullptr, flags);
}

template <typename T, int D>
void scale_gram(const T* in, int64_t ldin, T* out, int64_t ldout, const double* R, int64_t n, double* R2,
                unsigned* flags, const Red& red, cudaStream_t s, int) {
  k_scale_gram<T, D><<<persistent_rows(n), kThreads, 0, s>>>(in, ldin, out, ldout, R, n, R2, flags, red);
}

template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_gram_chol(const T* W, int64_t ld, int64_t n, double* R,
                                                        double* gdiag, unsigned* flags, Red red) {
  constexpr int NP = D * D;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T a[D];
#pragma unroll
    for (int k = 0; k < D; ++k) a[k] = W[i * ld + k];
#pragma unroll
    for (int p = 0; p < D; ++p)
#pragma unroll
      for (int q = 0; q < D; ++q) part[p * D + q] = fma(a[p], a[q], part[p * D + q]);
  }
  double pd[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
  block_sum<NP>(pd, red_s, tot);
  if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, NP, red.ticket, tot, red_s))
    if (threadIdx.x == 0) finish_chol(tot, D, R, gdiag, flags);
}

template <typename T, int D>
void gram_chol(const T* W, int64_t ld, int, int64_t n, double* R, double* gdiag, unsigned* flags, const Red& red,
               cudaStream_t s) {
  k_gram_chol<T, D><<<persistent_rows(n), kThreads, 0, s>>>(W, ld, n, R, gdiag, flags, red);
}

#define NS_INST_QR(T, D)                                                                                      \
  template void axpy_gram<T, D>(T*, const T*, const double*, int64_t, double*, unsigned*, const Red&,         \
                                cudaStream_t);                                                                \
  template void scale_gram<T, D>(const T*, int64_t, T*, int64_t, const double*, int64_t, double*, unsigned*, \
                                 const Red&, cudaStream_t, int);                                              \
  template void gram_chol<T, D>(const T*, int64_t, int, int64_t, double*, double*, unsigned*, const Red&,     \
                                cudaStream_t);
NS_INST_QR(double, 1)
NS_INST_QR(double, 2)
NS_INST_QR(double, 4)
NS_INST_QR(double, 8)
NS_INST_QR(float, 1)
NS_INST_QR(float, 2)
NS_INST_QR(float, 4)
NS_INST_QR(float, 8)

// ---------------------------------------------------------------------------
// projections against V = [X | Z] (classical Gram-Schmidt; CGS2 = two calls)
// W is a row-major panel of width W (leading dimension ldw); when Wp2 is given,
// columns [W/2, W) come from the second panel (two adjacent Lanczos blocks).
// Z holds panels of width P, so the column -> address map needs no division.
// ---------------------------------------------------------------------------
constexpr int kKT = 8;  // V columns per dots tile (a multiple of every P)

template <typename T, int W>
__device__ __forceinline__ void load_w(const T* Wp, const T* Wp2, int64_t ldw, int64_t i, T (&w)[W]) {
  if (Wp2 == nullptr) {
#pragma unroll
    for (int c = 0; c < W; ++c) w[c] = Wp[i * ldw + c];
  } else {
#pragma unroll
    for (int c = 0; c < W / 2; ++c) {
      w[c] = Wp[i * ldw + c];
      w[W / 2 + c] = Wp2[i * ldw + c];
    }
  }
}

template <typename T, int W>
__device__ __forceinline__ void store_w(T* Wp, T* Wp2, int64_t ldw, int64_t i, const T (&w)[W]) {
  if (Wp2 == nullptr) {
#pragma unroll
    for (int c = 0; c < W; ++c) Wp[i * ldw + c] = w[c];
  } else {
#pragma unroll
    for (int c = 0; c < W / 2; ++c) {
      Wp[i * ldw + c] = w[c];
      Wp2[i * ldw + c] = w[W / 2 + c];
    }
  }
}

// part[chunk][k][c] = sum over the rows of the chunk of V[i,k] W[i,c]
// V columns per dots tile: wide panels take 4 so the kKT * W accumulators stay in
// registers at 3+ CTAs per SM
template <int W>
constexpr int dots_kt() {
  return W >= 8 ? 4 : kKT;
}

template <typename T, int W, int P>
__global__ void __launch_bounds__(kThreads) k_proj_dots(VParts<T> V, const T* __restrict__ Wp,
                                                        const T* __restrict__ Wp2, int64_t ldw, int64_t n,
                                                        int64_t rows_per_chunk, double* part) {
  constexpr int KT = dots_kt<W>();
  constexpr int NP = KT * W;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  const int K = V.kx + V.kz;
  const int tilesX = (V.kx + KT - 1) / KT;
  const bool isX = (int)blockIdx.y < tilesX;
  const int k0 = isX ? blockIdx.y * KT : V.kx + (blockIdx.y - tilesX) * KT;  // first global column
  const int kend = isX ? V.kx : K;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk;
  if (r1 > n) r1 = n;
  T acc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) acc[k] = T(0);
  // column base pointers of this tile (element i of column kk at base[kk] + i * stride)
  const T* base[KT];
  int64_t stride = 1;
#pragma unroll
  for (int kk = 0; kk < KT; ++kk) {
    const int k = k0 + kk;
    if (isX) {
      base[kk] = V.X + (int64_t)(k < kend ? k : 0) * n;
    } else {
      const int kz = (k < kend ? k : V.kx) - V.kx;
      base[kk] = V.Z + (int64_t)(kz / P) * n * P + (kz % P);
    }
  }
  if (!isX) stride = P;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    T w[W];
    load_w<T, W>(Wp, Wp2, ldw, i, w);
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      const T v = (k0 + kk < kend) ? base[kk][i * stride] : T(0);
#pragma unroll
      for (int c = 0; c < W; ++c) acc[kk * W + c] = fma(v, w[c], acc[kk * W + c]);
    }
  }
  block_sum_t<T, NP>(acc, red_s, tot);
  for (int t = threadIdx.x; t < NP; t += blockDim.x) {
    const int k = k0 + t / W;
    if (k < kend) part[((size_t)blockIdx.x * K + k) * W + (t % W)] = tot[t];
  }
}

__global__ void k_dots_reduce(const double* part, int nchunks, int KW, double* C) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < KW; t += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * KW + t];
    C[t] = s;
  }
}

static int64_t dots_rows_per_chunk(int64_t n) {
  // at most ~128 rows per thread inside one chunk keeps FP32 partial sums short
  int64_t r = (int64_t)kThreads * 128;
  if (r > n) r = n > 0 ? n : 1;
  return r;
}

#define NS_P_SWITCH(P, CALL) \
  switch (P) {               \
    case 1: CALL(1); break;  \
    case 2: CALL(2); break;  \
    case 4: CALL(4); break;  \
    default: CALL(8); break; \
  }

template <typename T, int W>
void proj_dots(const VParts<T>& V, const T* Wp, const T* Wp2, int64_t ldw, int64_t n, double* C, double* part,
               cudaStream_t s, int64_t rows_per_chunk) {
  const int K = V.kx + V.kz;
  if (K == 0) return;
  int64_t rpc = dots_rows_per_chunk(n);
  if (rows_per_chunk == kDotsAutoChunks) {
    // enough (chunk, column tile) CTAs for 8 per SM, each chunk >= kDotsMinChunk rows
    const int kt = (std::is_same<T, double>::value && V.df) ? (W >= 16 ? 2 : W >= 8 ? 4 : 8) : dots_kt<W>();
    const int64_t tiles = ceil_div(V.kx, kt) + ceil_div(V.kz, kt);
    const int64_t want = (kMaxBlocks + tiles - 1) / tiles;
    int64_t r = (n + want - 1) / want;
    r = (r + kThreads - 1) / kThreads * kThreads;
    rpc = std::min<int64_t>(rpc, std::max<int64_t>(r, kDotsMinChunk));
  }
  if constexpr (std::is_same<T, double>::value) {
    if (V.df) {
      proj_dots_df<W>(V, Wp, Wp2, ldw, n, C, part, rpc, s);
      return;
    }
  }
  const int nchunks = ceil_div(n, rpc);
  constexpr int KT = dots_kt<W>();
  dim3 grid(nchunks, ceil_div(V.kx, KT) + ceil_div(V.kz, KT));
#define CALL(PP) k_proj_dots<T, W, PP><<<grid, kThreads, 0, s>>>(V, Wp, Wp2, ldw, n, rpc, part)
  NS_P_SWITCH(V.p, CALL)
#undef CALL
  k_dots_reduce<<<ceil_div((int64_t)K * W, kThreads), kThreads, 0, s>>>(part, nchunks, K * W, C);
}

// W -= V C (C: K x W row-major FP64, staged in dynamic shared memory) ; optional Gram + Cholesky
template <typename T, int W, int P, bool GRAM>
__global__ void __launch_bounds__(kThreads) k_proj_update(VParts<T> V, const double* __restrict__ C,
                                                          T* __restrict__ Wp, T* __restrict__ Wp2, int64_t ldw,
                                                          int64_t n, int gram, double* R, double* gdiag,
                                                          unsigned* flags, Red red) {
  constexpr int NP = GRAM ? W * W : 1;  // Gram accumulators only in the fused-CholQR variant
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* c_s = reinterpret_cast<T*>(smem_raw);
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  const int K = V.kx + V.kz;
  for (int t = threadIdx.x; t < K * W; t += blockDim.x) c_s[t] = (T)C[t];
  __syncthreads();
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  const int nzp = V.kz / P;  // whole panels of Z
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T w[W];
    load_w<T, W>(Wp, Wp2, ldw, i, w);
    // V streamed in batches: all loads of a batch are issued before its FMAs, so each
    // thread keeps 8 column loads in flight (the FMA chain on w is serial)
    int k = 0;
    for (; k + 8 <= V.kx; k += 8) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V.X[(int64_t)(k + u) * n + i];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int c = 0; c < W; ++c) w[c] = fma(-v[u], c_s[(k + u) * W + c], w[c]);
    }
    for (; k < V.kx; ++k) {
      const T v = V.X[(int64_t)k * n + i];
#pragma unroll
      for (int c = 0; c < W; ++c) w[c] = fma(-v, c_s[k * W + c], w[c]);
    }
    constexpr int PB = P >= 8 ? 1 : 8 / P;  // Z panels per batch
    int b = 0;
    for (; b + PB <= nzp; b += PB) {
      T zr[PB][P];
#pragma unroll
      for (int u = 0; u < PB; ++u) load_row<T, P>(V.Z + (int64_t)(b + u) * n * P + i * P, zr[u]);
#pragma unroll
      for (int u = 0; u < PB; ++u)
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const int kk = V.kx + (b + u) * P + q;
#pragma unroll
          for (int c = 0; c < W; ++c) w[c] = fma(-zr[u][q], c_s[kk * W + c], w[c]);
        }
    }
    for (; b < nzp; ++b) {
      T zr[P];
      load_row<T, P>(V.Z + (int64_t)b * n * P + i * P, zr);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int kk = V.kx + b * P + q;
#pragma unroll
        for (int c = 0; c < W; ++c) w[c] = fma(-zr[q], c_s[kk * W + c], w[c]);
      }
    }
    store_w<T, W>(Wp, Wp2, ldw, i, w);
    if constexpr (GRAM) {
#pragma unroll
      for (int p = 0; p < W; ++p)
#pragma unroll
        for (int q = 0; q < W; ++q) part[p * W + q] = fma(w[p], w[q], part[p * W + q]);
    }
  }
  (void)gram;
  if constexpr (!GRAM) return;
  double pd[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) pd[k] = (double)part[k];
  block_sum<NP>(pd, red_s, tot);
  if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, NP, red.ticket, tot, red_s))
    if (threadIdx.x == 0) finish_chol(tot, W, R, gdiag, flags);
}

template <typename T, int W>
cudaError_t proj_update(const VParts<T>& V, const double* C, T* Wp, T* Wp2, int64_t ldw, int64_t n, int gram,
                        double* R, double* gdiag, unsigned* flags, const Red& red, cudaStream_t s) {
  if constexpr (std::is_same<T, double>::value) {
    if (V.df) return proj_update_df<W>(V, C, Wp, Wp2, ldw, n, gram, R, gdiag, flags, red, s);
  }
  const int K = V.kx + V.kz;
  const size_t smem = sizeof(T) * (size_t)K * W;
  cudaError_t e = cudaSuccess;
#define CALL1(PP, GG)                                                                                    \
  do {                                                                                                   \
    const void* fn = reinterpret_cast<const void*>(k_proj_update<T, W, PP, GG>);                         \
    e = ensure_smem_limit(fn, smem);                                                                     \
    if (e != cudaSuccess) return e;                                                                      \
    k_proj_update<T, W, PP, GG><<<persistent_rows(n), kThreads, smem, s>>>(V, C, Wp, Wp2, ldw, n, gram, R, \
                                                                            gdiag, flags, red);          \
  } while (0)
#define CALL(PP)          \
  do {                    \
    if (gram)             \
      CALL1(PP, true);    \
    else                  \
      CALL1(PP, false);   \
  } while (0)
  NS_P_SWITCH(V.p, CALL)
#undef CALL
#undef CALL1
  return e;
}

// Raises the shared-memory limit of the single-panel update kernels (P = 1, with and
// without the fused Gram) to `bytes` on the current device ahead of time, so that a
// later launch needs no attribute change (e.g. while a stream is being captured).
template <typename T, int W>
cudaError_t proj_update_reserve_smem(size_t bytes) {
  cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(k_proj_update<T, W, 1, false>), bytes);
  if (e == cudaSuccess) e = ensure_smem_limit(reinterpret_cast<const void*>(k_proj_update<T, W, 1, true>), bytes);
  return e;
}

#define NS_INST_PROJ(T, W)                                                                                     \
  template void proj_dots<T, W>(const VParts<T>&, const T*, const T*, int64_t, int64_t, double*, double*,       \
                                cudaStream_t, int64_t);                                                        \
  template cudaError_t proj_update<T, W>(const VParts<T>&, const double*, T*, T*, int64_t, int64_t, int,        \
                                         double*, double*, unsigned*, const Red&, cudaStream_t);              \
  template cudaError_t proj_update_reserve_smem<T, W>(size_t);
NS_INST_PROJ(double, 1)
NS_INST_PROJ(double, 2)
NS_INST_PROJ(double, 4)
NS_INST_PROJ(double, 8)
NS_INST_PROJ(double, 16)
NS_INST_PROJ(float, 1)
NS_INST_PROJ(float, 2)
NS_INST_PROJ(float, 4)
NS_INST_PROJ(float, 8)
NS_INST_PROJ(float, 16)

// ---------------------------------------------------------------------------
// thick-restart GEMM: [Lnew | Znext] = Z(:, 0:R) V_Z(:, sel)
// ---------------------------------------------------------------------------
constexpr int kGR = 32;  // rows per block
constexpr int kGC = 32;  // output columns per pass

// Output tile: kRGR rows x kRGC selected columns per CTA; each thread holds a 4 x 4
// register tile.  The contraction over the R basis columns runs in chunks of kRGJ:
// Z is staged transposed (zt[j][r]) with coalesced loads (the rows of one panel
// block are contiguous), the selected columns of V_Z as vt[j][c].
constexpr int kRGR = 64, kRGC = 64, kRGJ = 64;

template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&v)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_restart_gemm(const T* __restrict__ Z, int d, int R,
                                                           const double* __restrict__ VZ, const int* __restrict__ sel,
                                                           int nsel, int nl, int64_t n, T* Lnew, T* Znext) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* zt = reinterpret_cast<T*>(smem_raw);  // kRGJ x kRGR
  T* vt = zt + kRGJ * kRGR;                // kRGJ x kRGC
  const int64_t i0 = (int64_t)blockIdx.x * kRGR;
  const int cg = threadIdx.x & 15, rg = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  const int per_blk = kRGR * d;
  for (int c0 = 0; c0 < nsel; c0 += kRGC) {
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int j0 = 0; j0 < R; j0 += kRGJ) {  // kRGJ is a multiple of every d, R a multiple of d
      const int jc = (R - j0) < kRGJ ? (R - j0) : kRGJ;
      __syncthreads();
      // Z(i0 + r, j), j = b d + q, lives at b n d + (i0 + r) d + q: contiguous over (r, q)
      for (int t = threadIdx.x; t < jc * kRGR; t += blockDim.x) {
        const int b = j0 / d + t / per_blk, rem = t % per_blk;
        const int r = rem / d, q = rem % d;
        zt[(b * d + q - j0) * kRGR + r] = (i0 + r < n) ? Z[(int64_t)b * n * d + i0 * d + rem] : T(0);
      }
      for (int t = threadIdx.x; t < jc * kRGC; t += blockDim.x) {
        const int jj = t / kRGC, c = t % kRGC;
        vt[t] = (c0 + c < nsel) ? (T)VZ[(int64_t)sel[c0 + c] * R + j0 + jj] : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int jj = 0; jj < jc; ++jj) {
        T zr[4], vr[4];
        lds4<T>(zt + jj * kRGR + rg * 4, zr);
        lds4<T>(vt + jj * kRGC + cg * 4, vr);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(zr[a], vr[b], acc[a][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + rg * 4 + a;
      if (i >= n) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = c0 + cg * 4 + b;
        if (c >= nsel) continue;
        if (c < nl) {
          Lnew[i * nl + c] = acc[a][b];
        } else {
          const int kc = c - nl;
          Znext[(int64_t)(kc / d) * n * d + i * d + (kc % d)] = acc[a][b];
        }
      }
    }
  }
}

// FP64: the FP64 pipe is the bound; this row-tile form (32 rows staged, one column
// per lane) measured faster than the 4 x 4 register tile above on GB300 (10.1 vs
// 12.3 ms at n = 1e6, R = 120); it stages all R columns, so R > 400 goes to the
// chunked kernel
__global__ void __launch_bounds__(kThreads) k_restart_gemm_fp64(const double* __restrict__ Z, int d, int R,
                                                           const double* __restrict__ VZ, const int* __restrict__ sel,
                                                           int nsel, int nl, int64_t n, double* Lnew, double* Znext) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* zs = reinterpret_cast<double*>(smem_raw);  // kGR x R
  double* vs = zs + kGR * R;                    // R x kGC
  const int64_t i0 = (int64_t)blockIdx.x * kGR;
  for (int t = threadIdx.x; t < kGR * R; t += blockDim.x) {
    const int r = t / R, j = t % R;
    const int64_t i = i0 + r;
    zs[t] = (i < n) ? Z[(int64_t)(j / d) * n * d + i * d + (j % d)] : 0.0;
  }
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps x 32 columns
  for (int c0 = 0; c0 < nsel; c0 += kGC) {
    __syncthreads();
    for (int t = threadIdx.x; t < R * kGC; t += blockDim.x) {
      const int j = t / kGC, c = t % kGC;
      vs[t] = (c0 + c < nsel) ? VZ[(int64_t)sel[c0 + c] * R + j] : 0.0;
    }
    __syncthreads();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < R; ++j) {
      const double v = vs[j * kGC + tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(zs[(ty + 8 * q) * R + j], v, acc[q]);
    }
    const int c = c0 + tx;
    if (c < nsel) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + ty + 8 * q;
        if (i >= n) continue;
        if (c < nl) {
          Lnew[i * nl + c] = acc[q];
        } else {
          const int kc = c - nl;
          Znext[(int64_t)(kc / d) * n * d + i * d + (kc % d)] = acc[q];
        }
      }
    }
  }
}


template <typename T>
cudaError_t restart_gemm(const T* Z, int d, int R, const double* VZ, const int* sel, int nsel, int nl, int64_t n,
                         T* Lnew, T* Znext, cudaStream_t s) {
  if (nsel == 0 || n == 0) return cudaSuccess;
  const size_t smem64 = sizeof(double) * (size_t)(kGR * R + R * kGC);
  if (sizeof(T) == 8 && smem64 <= 200 * 1024) {  // larger R (> 400) takes the chunked kernel
    const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(k_restart_gemm_fp64), smem64);
    if (e != cudaSuccess) return e;
    k_restart_gemm_fp64<<<ceil_div(n, kGR), kThreads, smem64, s>>>(reinterpret_cast<const double*>(Z), d, R, VZ, sel,
                                                                   nsel, nl, n, reinterpret_cast<double*>(Lnew),
                                                                   reinterpret_cast<double*>(Znext));
    return cudaSuccess;
  }
  const size_t smem = sizeof(T) * (size_t)kRGJ * (kRGR + kRGC);  // 32 KB
  const cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(k_restart_gemm<T>), smem);
  if (e != cudaSuccess) return e;
  k_restart_gemm<T><<<ceil_div(n, kRGR), kThreads, smem, s>>>(Z, d, R, VZ, sel, nsel, nl, n, Lnew, Znext);
  return cudaSuccess;
}
template cudaError_t restart_gemm<double>(const double*, int, int, const double*, const int*, int, int, int64_t,
                                          double*, double*, cudaStream_t);
template cudaError_t restart_gemm<float>(const float*, int, int, const double*, const int*, int, int, int64_t,
                                         float*, float*, cudaStream_t);

template <typename T>
__global__ void k_panel_to_cols(const T* P, int64_t ldp, int w, int64_t n, T* X, int c0) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < w; ++c) X[(int64_t)(c0 + c) * n + i] = P[i * ldp + c];
}
template <typename T>
void panel_to_cols(const T* P, int64_t ldp, int w, int64_t n, T* X, int c0, cudaStream_t s) {
  k_panel_to_cols<T><<<stream_grid(n), kThreads, 0, s>>>(P, ldp, w, n, X, c0);
}
template void panel_to_cols<double>(const double*, int64_t, int, int64_t, double*, int, cudaStream_t);
template void panel_to_cols<float>(const float*, int64_t, int, int64_t, float*, int, cudaStream_t);

template <typename T>
__global__ void k_cols_to_panel64(const T* X, int c0, int w, int64_t n, double* P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < w; ++c) P[i * w + c] = (double)X[(int64_t)(c0 + c) * n + i];
}
template <typename T>
void cols_to_panel64(const T* X, int c0, int w, int64_t n, double* P, cudaStream_t s) {
  k_cols_to_panel64<T><<<stream_grid(n), kThreads, 0, s>>>(X, c0, w, n, P);
}
template void cols_to_panel64<double>(const double*, int, int, int64_t, double*, cudaStream_t);
template void cols_to_panel64<float>(const float*, int, int, int64_t, double*, cudaStream_t);

// ---------------------------------------------------------------------------
// Lanczos step finalization: Gamma_j = R2 R1, its norms, and column j+1 of W
// (Sec. 4.2, three cases, readings R2-R6); one block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_step_finalize(OmegaArgs a, int mode) {
  __shared__ double sh[4];  // g, nXj, nGjm1, sumF
  __shared__ int bd;
  __shared__ int trig[2];
  const int d = a.d, j = a.j;
  const int nbp = a.nb + 1;
  if (threadIdx.x == 0) {
    double G[kMaxD * kMaxD];
    if (a.R2)
      matmul_dd(a.R2, a.R1, G, d);
    else
      for (int k = 0; k < d * d; ++k) G[k] = a.R1[k];
    double smax, smn;
    sv_minmax(G, d, &smax, &smn);
    bd = ((*a.flags & 1u) != 0u) || !(smn > a.bd_tol);
    if (bd) {
      for (int k = 0; k < d * d; ++k) G[k] = 0.0;
      smax = smn = 0.0;
    }
    for (int k = 0; k < d * d; ++k) a.Gam[(size_t)j * d * d + k] = G[k];
    a.nGam[j] = smax;
    a.sminGam[j] = smn;
    trig[0] = trig[1] = 0;
  }
  __syncthreads();
  if (mode == 1) return;
  if (bd) {
    if (threadIdx.x == 0) {
      atomicOr(a.flags, 1u);
      a.counters[2] += 1;
    }
    return;
  }
  double* cj = a.wz + (size_t)(j % 3) * nbp;
  double* cjm1 = a.wz + (size_t)((j + 2) % 3) * nbp;
  double* cn = a.wz + (size_t)((j + 1) % 3) * nbp;
  if (threadIdx.x == 0) {
    sh[0] = 1.0 / a.sminGam[j];
    sh[1] = a.nXi[j];
    sh[2] = a.nGam[j - 1];
    double s = 0.0;
    for (int i = 0; i < a.r0; ++i) s += cj[i] * a.nF[i];  // w_{i,j} ||F_i||, i < r0 < j
    sh[3] = s;
  }
  __syncthreads();
  const double g = sh[0], nXj = sh[1], nGjm1 = sh[2], sumF = sh[3];
  const double ud2 = 2.0 * a.u_d;
  // w(a, c) = W[a][c] for a < c, else 0 (strictly upper triangular W)
#define WZ(row, colptr, col) ((row) < (col) ? (colptr)[row] : 0.0)
  int tz = 0;
  for (int b = threadIdx.x; b <= j; b += blockDim.x) {
    double val;
    if (b < a.r0) {
      val = WZ(b, cj, j) * (a.nTheta[b] + nXj) + WZ(a.r0, cj, j) * a.nF[b] + WZ(b, cjm1, j - 1) * nGjm1 + ud2;
    } else if (b == a.r0) {
      val = WZ(b, cj, j) * (a.nXi[b] + nXj) + sumF + WZ(b + 1, cj, j) * a.nGam[b] + WZ(b, cjm1, j - 1) * nGjm1 +
            ud2;
    } else {
      val = WZ(b, cj, j) * (a.nXi[b] + nXj) + WZ(b + 1, cj, j) * a.nGam[b] + WZ(b - 1, cj, j) * a.nGam[b - 1] +
            WZ(b, cjm1, j - 1) * nGjm1 + ud2;
    }
    const double w = g * val;
    cn[b] = w;
    if (a.trace) a.trace[(size_t)(j + 1) * nbp + b] = w;
    if (!(w <= a.u_ro)) tz = 1;
  }
#undef WZ
  double* xj = a.wx + (size_t)(j % 3) * a.cap;
  double* xjm1 = a.wx + (size_t)((j + 2) % 3) * a.cap;
  double* xn = a.wx + (size_t)((j + 1) % 3) * a.cap;
  int tx = 0;
  for (int k = threadIdx.x; k < a.nlock; k += blockDim.x) {
    const double w = g * (xj[k] * (a.xtheta[k] + nXj) + a.xrho[k] + xjm1[k] * nGjm1 + ud2);
    xn[k] = w;
    if (!(w <= a.u_ro)) tx = 1;
  }
  if (tz) atomicOr(&trig[0], 1);
  if (tx) atomicOr(&trig[1], 1);
  __syncthreads();
  const int TZ = trig[0], TX = trig[1];
  if (TZ) {
    for (int b = threadIdx.x; b <= j; b += blockDim.x) {
      if (b < j) cj[b] = a.u_d;
      cn[b] = a.u_d;
    }
  }
  if (TX) {
    for (int k = threadIdx.x; k < a.nlock; k += blockDim.x) xj[k] = xn[k] = a.u_d;
  }
  if (threadIdx.x == 0) {
    unsigned f = 0;
    if (TZ) {
      f |= 2u;
      a.counters[0] += 1;
    }
    if (TX) {
      f |= 4u;
      a.counters[1] += 1;
    }
    if (f) atomicOr(a.flags, f);
  }
}

void step_finalize(const OmegaArgs& a, cudaStream_t s) { k_step_finalize<<<1, kThreads, 0, s>>>(a, 0); }

// store Gamma and its norms only (first step of a cycle, replacement blocks)
void gamma_store(const OmegaArgs& a, cudaStream_t s) { k_step_finalize<<<1, kThreads, 0, s>>>(a, 1); }

// W column `col`: rows b < upto set to val; locked rows too
__global__ void k_omega_fill(double* wz, double* wx, int nb, int cap, int col, int upto, int nlock, double val) {
  double* cz = wz + (size_t)(col % 3) * (nb + 1);
  double* cx = wx + (size_t)(col % 3) * cap;
  for (int b = threadIdx.x; b < upto; b += blockDim.x) cz[b] = val;
  for (int k = threadIdx.x; k < nlock; k += blockDim.x) cx[k] = val;
}

void omega_init(double* wz, double* wx, int nb, int cap, int r0, int nlock, double u_d, cudaStream_t s) {
  k_omega_fill<<<1, kThreads, 0, s>>>(wz, wx, nb, cap, r0, r0, nlock, u_d);
  k_omega_fill<<<1, kThreads, 0, s>>>(wz, wx, nb, cap, r0 + 1, r0 + 1, nlock, u_d);
}

void omega_column(double* wz, double* wx, int nb, int cap, int col, int nlock, double u_d, cudaStream_t s) {
  k_omega_fill<<<1, kThreads, 0, s>>>(wz, wx, nb, cap, col, col, nlock, u_d);
}

// ---------------------------------------------------------------------------
// restart bookkeeping (one block each)
// ---------------------------------------------------------------------------
// T (R x R, column-major) of Eq. (defT): diag(Theta), arrow F (d x k0, row-major),
// blocks Xi_b on the diagonal and Gamma_b below it for b = k0/d .. R/d-1
__global__ void k_build_T(const double* Theta, const double* F, const double* Xi, const double* Gam, int k0, int d,
                          int R, double* T) {
  for (int t = threadIdx.x; t < R * R; t += blockDim.x) T[t] = 0.0;
  __syncthreads();
  for (int c = threadIdx.x; c < k0; c += blockDim.x) {
    T[(int64_t)c * R + c] = Theta[c];
    for (int r = 0; r < d; ++r) {
      const double f = F[r * k0 + c];
      T[(int64_t)c * R + (k0 + r)] = f;
      T[(int64_t)(k0 + r) * R + c] = f;
    }
  }
  const int nb = R / d, r0 = k0 / d;
  for (int t = threadIdx.x; t < (nb - r0) * d * d; t += blockDim.x) {
    const int b = r0 + t / (d * d), e = t % (d * d), i = e / d, k = e % d;
    T[(int64_t)(b * d + k) * R + (b * d + i)] = Xi[(size_t)b * d * d + e];
    if (b + 1 < nb) {
      const double gv = Gam[(size_t)b * d * d + e];  // Gamma_b(i,k): row (b+1)d+i, column b d + k
      T[(int64_t)(b * d + k) * R + ((b + 1) * d + i)] = gv;
      T[(int64_t)((b + 1) * d + i) * R + (b * d + k)] = gv;
    }
  }
}

void build_T(const double* Theta, const double* F, const double* Xi, const double* Gam, int k0, int d, int R,
             double* T, cudaStream_t s) {
  k_build_T<<<1, kThreads, 0, s>>>(Theta, F, Xi, Gam, k0, d, R, T);
}

// Ritz residual estimates ||Gamma_last V_Z(last d rows, i)||_2
__global__ void k_ritz_resid(const double* G, const double* VZ, int d, int R, double* res) {
  for (int i = threadIdx.x; i < R; i += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < d; ++r) {
      double t = 0.0;
      for (int k = 0; k < d; ++k) t += G[r * d + k] * VZ[(int64_t)i * R + (R - d + k)];
      s += t * t;
    }
    res[i] = sqrt(s);
  }
}
void ritz_resid(const double* Gam_last, const double* VZ, int d, int R, double* res, cudaStream_t s) {
  k_ritz_resid<<<1, kThreads, 0, s>>>(Gam_last, VZ, d, R, res);
}

// F = Rr Gamma_last V_Z(last d rows, keep) (reading R8), Theta = theta(keep), block norms
__global__ void k_make_F(const double* Rr, const double* G, const double* VZ, const int* keep, const double* theta,
                         int k0, int d, int R, double* F, double* Theta, double* nTheta, double* nF) {
  __shared__ double RG[kMaxD * kMaxD];
  if (threadIdx.x == 0) matmul_dd(Rr, G, RG, d);
  __syncthreads();
  for (int c = threadIdx.x; c < k0; c += blockDim.x) {
    const int col = keep[c];
    for (int r = 0; r < d; ++r) {
      double t = 0.0;
      for (int k = 0; k < d; ++k) t += RG[r * d + k] * VZ[(int64_t)col * R + (R - d + k)];
      F[r * k0 + c] = t;
    }
    Theta[c] = theta[col];
  }
  __syncthreads();
  for (int b = threadIdx.x; b < k0 / d; b += blockDim.x) {
    double th = 0.0, M[kMaxD * kMaxD];
    for (int k = 0; k < d; ++k) th = fmax(th, fabs(Theta[b * d + k]));
    for (int r = 0; r < d; ++r)
      for (int k = 0; k < d; ++k) M[r * d + k] = F[r * k0 + b * d + k];
    double smax, smn;
    sv_minmax(M, d, &smax, &smn);
    nTheta[b] = th;
    nF[b] = smax;
  }
}
void make_F(const double* Rr, const double* Gam_last, const double* VZ, const int* keep, const double* theta, int k0,
            int d, int R, double* F, double* Theta, double* nTheta, double* nF, cudaStream_t s) {
  k_make_F<<<1, kThreads, 0, s>>>(Rr, Gam_last, VZ, keep, theta, k0, d, R, F, Theta, nTheta, nF);
}

// ---------------------------------------------------------------------------
// CG / CGLS refinement helpers on row-major panels of width W (T = float for
// the inner iterations, double for the outer residual correction)
// ---------------------------------------------------------------------------
// delta += alpha p (np rows) ; r -= alpha q (nr rows) ; rr_new[c] = sum_i r_i[c]^2.
// Element-linear over the row-major panels, so every access is coalesced; W divides
// the grid stride, so each thread always meets the same column c = threadIdx.x % W
// and keeps one partial sum (FP32 over its few dozen elements, FP64 beyond).
template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_cg_update(T* delta, const T* p, int64_t np_, T* r, const T* q,
                                                        int64_t nr, const double* alpha, Red red, double* rr_new) {
  static_assert(kThreads % W == 0, "the column of an element must not depend on the grid stride");
  __shared__ double red_s[kThreads];
  __shared__ double tot[W];
  const int c = threadIdx.x % W;
  const T al = (T)alpha[c];
  const int64_t ep = np_ * W, er = nr * W, emax = ep > er ? ep : er;
  T part = T(0);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < emax; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < ep) delta[t] = fma(al, p[t], delta[t]);
    if (t < er) {
      const T v = fma(-al, q[t], r[t]);
      r[t] = v;
      part = fma(v, v, part);
    }
  }
  red_s[threadIdx.x] = (double)part;
  __syncthreads();
  if (threadIdx.x < W) {
    double sum = 0.0;
    for (int j = threadIdx.x; j < kThreads; j += W) sum += red_s[j];
    tot[threadIdx.x] = sum;
  }
  __syncthreads();
  if (threadIdx.x < W) red.part[(size_t)blockIdx.x * W + threadIdx.x] = tot[threadIdx.x];
  if (last_block_reduce(red.part, W, red.ticket, tot, red_s))
    if (threadIdx.x < W) rr_new[threadIdx.x] = tot[threadIdx.x];
}

template <typename T, int W>
void cg_update2(T* delta, const T* p, int64_t np_, T* r, const T* q, int64_t nr, const double* alpha, const Red& red,
                double* rr_new, cudaStream_t s) {
  k_cg_update<T, W><<<persistent_rows((np_ > nr ? np_ : nr) * W), kThreads, 0, s>>>(delta, p, np_, r, q, nr, alpha,
                                                                                      red, rr_new);
}

// p = s + beta p
template <typename T, int W>
__global__ void k_cg_direction(T* p, const T* sres, const double* beta, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * W; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % W);
    p[t] = fma((T)beta[c], p[t], sres[t]);
  }
}
template <typename T, int W>
void cg_direction2(T* p, const T* sres, const double* beta, int64_t n, cudaStream_t s) {
  k_cg_direction<T, W><<<stream_grid(n * W), kThreads, 0, s>>>(p, sres, beta, n);
}

// alpha[c] = num[c]/den[c] for active columns (else 0); same kernel for beta
__global__ void k_cg_scalars(const double* num, const double* den, const unsigned char* active, double* out, int w) {
  const int c = threadIdx.x;
  if (c < w) out[c] = (active[c] && den[c] > 0.0) ? num[c] / den[c] : 0.0;
}
void cg_scalars(const double* num, const double* den, const unsigned char* active, double* out, int w,
                cudaStream_t s) {
  k_cg_scalars<<<1, 32, 0, s>>>(num, den, active, out, w);
}

// active[c] &= rr[c] > tol2[c] (tol2 per column, or the scalar tol2s when tol2 == null)
__global__ void k_cg_check(const double* rr, const double* tol2, double tol2s, unsigned char* active, int* nactive,
                           int w) {
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int c = 0; c < w; ++c) {
      const unsigned char a = active[c] && (rr[c] > (tol2 ? tol2[c] : tol2s));
      active[c] = a;
      cnt += a;
    }
    *nactive = cnt;
  }
}
void cg_check(const double* rr, const double* tol2, double tol2s, unsigned char* active, int* nactive, int w,
              cudaStream_t s) {
  k_cg_check<<<1, 32, 0, s>>>(rr, tol2, tol2s, active, nactive, w);
}

// tol2[c] = f^2 rr[c]
__global__ void k_scale_vec(const double* rr, double f2, double* out, int w) {
  if (threadIdx.x < w) out[threadIdx.x] = f2 * rr[threadIdx.x];
}
void scale_vec(const double* rr, double f2, double* out, int w, cudaStream_t s) {
  k_scale_vec<<<1, 32, 0, s>>>(rr, f2, out, w);
}

// columns [c0, c0+w) of X (FP64 column-major) into a zero-padded row-major panel of width W
template <int W>
__global__ void k_cols_to_panel(const double* X, int c0, int w, int64_t n, double* P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < W; ++c) P[i * W + c] = (c < w) ? X[(int64_t)(c0 + c) * n + i] : 0.0;
}
template <int W>
void cols_to_panel_w(const double* X, int c0, int w, int64_t n, double* P, cudaStream_t s) {
  k_cols_to_panel<W><<<stream_grid(n), kThreads, 0, s>>>(X, c0, w, n, P);
}

// x -= delta (FP64 panel minus the FP32 correction)
template <int W>
__global__ void k_sub_correction(double* x, const float* dl, int64_t n) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * W; t += (int64_t)gridDim.x * blockDim.x)
    x[t] -= (double)dl[t];
}
template <int W>
void sub_correction(double* x, const float* dl, int64_t n, cudaStream_t s) {
  k_sub_correction<W><<<stream_grid(n * W), kThreads, 0, s>>>(x, dl, n);
}

// X[:, c0 + c] = P[:, c] for c < w
template <int W>
__global__ void k_panel_to_cols64(const double* P, double* X, int c0, int w, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < w; ++c) X[(int64_t)(c0 + c) * n + i] = P[i * W + c];
}
template <int W>
void panel_to_cols64(const double* P, double* X, int c0, int w, int64_t n, cudaStream_t s) {
  k_panel_to_cols64<W><<<stream_grid(n), kThreads, 0, s>>>(P, X, c0, w, n);
}

template void cg_update2<float, 16>(float*, const float*, int64_t, float*, const float*, int64_t, const double*,
                                    const Red&, double*, cudaStream_t);
template void cg_direction2<float, 16>(float*, const float*, const double*, int64_t, cudaStream_t);
template void cols_to_panel_w<16>(const double*, int, int, int64_t, double*, cudaStream_t);
template void sub_correction<16>(double*, const float*, int64_t, cudaStream_t);
template void panel_to_cols64<16>(const double*, double*, int, int, int64_t, cudaStream_t);

}  // namespace ns

namespace ns {

// ---------------------------------------------------------------------------
// Gram matrix G = X^T X of an FP64 column-major n x N basis (upper-triangular
// 32 x 32 tiles, split over row chunks; partials reduced in chunk order).  The
// products run in compensated FP32 pairs (df_split / df_fma) on the FP32 pipe:
// each staged FP64 element is split once into hi + lo words in shared memory, each
// thread keeps 4 pair accumulators.  A pair add has relative error 2^-48 of its
// running sum, so the pairs are flushed into FP64 accumulators every 1024 rows:
// each pair sum stays short, and the FP64 sum of the flushed segments is as
// accurate as a plain FP64 accumulation.
// ---------------------------------------------------------------------------
constexpr int kGT = 32;

__global__ void __launch_bounds__(kThreads) k_gram_tiles(const double* __restrict__ X, int64_t n, int N,
                                                         int64_t rows_per_chunk, const int2* __restrict__ pairs,
                                                         double* part) {
  __shared__ float2 xa[kGT][kGT + 1];
  __shared__ float2 xb[kGT][kGT + 1];
  const int2 pr = pairs[blockIdx.x];
  const int ca = pr.x * kGT, cb = pr.y * kGT;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk;
  if (r1 > n) r1 = n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int seg = 0;
  for (int64_t base = r0; base < r1; base += kGT) {
    if (++seg == 32) {  // 1024 rows into FP64
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += (double)sh[q] + (double)sl[q];
        sh[q] = sl[q] = 0.f;
      }
      seg = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kGT * kGT; t += blockDim.x) {
      const int r = t & 31, c = t >> 5;  // 32 consecutive rows of one column per warp
      const int64_t i = base + r;
      float h, l;
      df_split((i < r1 && ca + c < N) ? X[(int64_t)(ca + c) * n + i] : 0.0, h, l);
      xa[r][c] = make_float2(h, l);
      df_split((i < r1 && cb + c < N) ? X[(int64_t)(cb + c) * n + i] : 0.0, h, l);
      xb[r][c] = make_float2(h, l);
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kGT; ++r) {
      const float2 b = xb[r][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 a = xa[r][ty + 8 * q];
        df_fma(sh[q], sl[q], a.x, a.y, b.x, b.y);
      }
    }
  }
  double* out = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (kGT * kGT);
#pragma unroll
  for (int q = 0; q < 4; ++q) out[(ty + 8 * q) * kGT + tx] = acc[q] + ((double)sh[q] + (double)sl[q]);
}

__global__ void k_gram_reduce(const double* part, const int2* pairs, int npairs, int nchunks, int N, double* G) {
  const int64_t total = (int64_t)npairs * kGT * kGT;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(t / (kGT * kGT)), e = (int)(t % (kGT * kGT));
    // a diagonal tile holds both (i, j) and (j, i), summed in different orders: only
    // its upper triangle writes, so every entry of G has exactly one writer
    if (pairs[p].x == pairs[p].y && e / kGT > e % kGT) continue;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[((size_t)c * npairs + p) * (kGT * kGT) + e];
    const int i = pairs[p].x * kGT + e / kGT, j = pairs[p].y * kGT + e % kGT;
    if (i < N && j < N) {
      G[(int64_t)j * N + i] = s;
      G[(int64_t)i * N + j] = s;
    }
  }
}

size_t gram_part_doubles(int64_t n, int N) {
  const int nt = (N + kGT - 1) / kGT;
  const int npairs = nt * (nt + 1) / 2;
  int nchunks = (int)((152 * 4 + npairs - 1) / npairs);
  if (nchunks < 1) nchunks = 1;
  if ((int64_t)nchunks * kGT > n) nchunks = (int)std::max<int64_t>(1, n / kGT);
  return (size_t)nchunks * npairs * kGT * kGT + 2 * (size_t)npairs;
}

void gram64(const double* X, int64_t n, int N, double* G, double* part, cudaStream_t s) {
  const int nt = (N + kGT - 1) / kGT;
  const int npairs = nt * (nt + 1) / 2;
  int nchunks = (int)((152 * 4 + npairs - 1) / npairs);
  if (nchunks < 1) nchunks = 1;
  if ((int64_t)nchunks * kGT > n) nchunks = (int)std::max<int64_t>(1, n / kGT);
  int64_t rpc = (n + nchunks - 1) / nchunks;
  rpc = (rpc + kGT - 1) / kGT * kGT;
  int2* pairs = reinterpret_cast<int2*>(part + (size_t)nchunks * npairs * kGT * kGT);
  std::vector<int2> hp;
  for (int a = 0; a < nt; ++a)
    for (int b = a; b < nt; ++b) hp.push_back(make_int2(a, b));
  cudaMemcpyAsync(pairs, hp.data(), sizeof(int2) * hp.size(), cudaMemcpyHostToDevice, s);
  k_gram_tiles<<<dim3(npairs, nchunks), kThreads, 0, s>>>(X, n, N, rpc, pairs, part);
  k_gram_reduce<<<stream_grid((int64_t)npairs * kGT * kGT), kThreads, 0, s>>>(part, pairs, npairs, nchunks, N, G);
}

// ---------------------------------------------------------------------------
// first-order symmetric (Loewdin) re-orthonormalization:
//   Xout = X - 0.5 X E,  E = X^T X - I  (|E| small, so the product runs in FP32:
//   its relative error ~1e-7 is an absolute ~1e-7 |E|, far below FP64 rounding)
// One CTA: 64 rows x 64 output columns, K = N in chunks of 32, each thread a
// 4 x 4 register tile.  blockIdx.x walks the column blocks, so the CTAs that read
// the same 64-row strip of X run together and share it through L2.
// ---------------------------------------------------------------------------
constexpr int kLR = 64, kLC = 64, kLK = 32;

__global__ void __launch_bounds__(kThreads) k_lowdin(const double* __restrict__ X, int64_t n, int N,
                                                     const double* __restrict__ G, double* __restrict__ Xout) {
  __shared__ float xs[kLK][kLR + 4];  // xs[k][row]
  __shared__ float es[kLK][kLC + 4];  // es[k][col] = E(k0 + k, c0 + col)
  const int c0 = blockIdx.x * kLC;
  const int64_t i0 = (int64_t)blockIdx.y * kLR;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;  // rows tr*4.., columns tc*4..
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < N; k0 += kLK) {
    __syncthreads();
    for (int t = threadIdx.x; t < kLK * kLR; t += blockDim.x) {
      const int r = t % kLR, k = t / kLR;  // consecutive rows of one column: coalesced
      const int64_t i = i0 + r;
      xs[k][r] = (i < n && k0 + k < N) ? (float)X[(int64_t)(k0 + k) * n + i] : 0.f;
    }
    for (int t = threadIdx.x; t < kLK * kLC; t += blockDim.x) {
      const int k = t % kLK, c = t / kLK;  // E is symmetric: E(kk, j) = G[j * N + kk] - delta
      const int kk = k0 + k, j = c0 + c;
      es[k][c] = (kk < N && j < N) ? (float)(G[(int64_t)j * N + kk] - (kk == j ? 1.0 : 0.0)) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kLK; ++k) {
      const float4 xv = *reinterpret_cast<const float4*>(&xs[k][tr * 4]);
      const float4 ev = *reinterpret_cast<const float4*>(&es[k][tc * 4]);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, eb[4] = {ev.x, ev.y, ev.z, ev.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], eb[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int j = c0 + tc * 4 + b;
    if (j >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t i = i0 + tr * 4 + a;
      if (i < n) Xout[(int64_t)j * n + i] = X[(int64_t)j * n + i] - 0.5 * (double)acc[a][b];
    }
  }
}

void lowdin_update(const double* X, int64_t n, int N, const double* G, double* Xout, cudaStream_t s) {
  dim3 grid(ceil_div(N, kLC), ceil_div(n, kLR));
  k_lowdin<<<grid, kThreads, 0, s>>>(X, n, N, G, Xout);
}

// max_ij |G_ij - delta_ij| (one block)
__global__ void k_max_offdiag(const double* G, int N, double* out) {
  __shared__ double red_s[kThreads / 32];
  double m = 0.0;
  for (int64_t t = threadIdx.x; t < (int64_t)N * N; t += blockDim.x) {
    const int i = (int)(t % N), j = (int)(t / N);
    m = fmax(m, fabs(G[t] - (i == j ? 1.0 : 0.0)));
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red_s[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red_s[w]);
    *out = t;
  }
}
void max_offdiag(const double* G, int N, double* out, cudaStream_t s) { k_max_offdiag<<<1, kThreads, 0, s>>>(G, N, out); }

}  // namespace ns

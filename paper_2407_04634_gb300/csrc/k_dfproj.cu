// FP64 block Gram-Schmidt products in compensated FP32-pair arithmetic.
//
// The partial reorthogonalization of Sec. 4.2 (C = V^T W and W <- W - V C, V up to
// n x ~600, W n x 2..16) does one FMA per 8 bytes of V: far above the FP64 pipe's
// ridge point on this part (about 0.15 flop/B), far below the FP32 pipe's.  So the
// FP64 path runs these products on the FP32 pipe in compensated pair arithmetic:
//   * every FP64 operand x is split exactly, with integer operations only, into
//     x = hi + lo + r, hi holding the leading 24 significand bits, lo the next 24
//     (rounded), |r| <= 2^-48 |x|;
//   * a product a b is formed as p + e with p = fl(ah bh) and e the exact FMA
//     residual of ah bh plus the cross terms ah bl + al bh (al bl is below
//     2^-48 |a b| and is dropped);
//   * a running sum is kept as an unevaluated pair (sh, sl) updated by TwoSum
//     (Knuth) and renormalized by FastTwoSum (Dekker).
// Each thread accumulates 128 rows this way, then the partial sums are reduced in
// FP64 as before.  The error per inner product is about 2^-47 sum_i |v_i w_i|,
// below the sqrt(n) u sum |v_i w_i| of a plain FP64 accumulation at these lengths.
// The update forms the correction V C in pairs and subtracts it from W in FP64, so
// W itself keeps its full FP64 precision.
//
// All adds and multiplies of the error-free transformations use explicit
// round-to-nearest intrinsics so that the compiler cannot contract them into FMAs.
#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace ns {
namespace {

template <int W>
__device__ __forceinline__ void load_w2(const double* Wp, const double* Wp2, int64_t ldw, int64_t i, double (&w)[W]) {
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

template <int W>
__device__ __forceinline__ void store_w2(double* Wp, double* Wp2, int64_t ldw, int64_t i, const double (&w)[W]) {
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

// V columns per dots tile: the pair accumulators (2 KT W floats) stay in registers
template <int W>
constexpr int df_kt() {
  return W >= 16 ? 2 : W >= 8 ? 4 : 8;
}

// part[chunk][k][c] = sum over the chunk's rows of V[i,k] W[i,c] (pairs per thread,
// FP64 across threads)
template <int W, int P>
__global__ void __launch_bounds__(kThreads) k_proj_dots_df(VParts<double> V, const double* __restrict__ Wp,
                                                           const double* __restrict__ Wp2, int64_t ldw, int64_t n,
                                                           int64_t rows_per_chunk, double* part) {
  constexpr int KT = df_kt<W>();
  constexpr int NP = KT * W;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  const int K = V.kx + V.kz;
  const int tilesX = (V.kx + KT - 1) / KT;
  const bool isX = (int)blockIdx.y < tilesX;
  const int k0 = isX ? blockIdx.y * KT : V.kx + (blockIdx.y - tilesX) * KT;
  const int kend = isX ? V.kx : K;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk;
  if (r1 > n) r1 = n;
  float sh[NP], sl[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) sh[k] = sl[k] = 0.f;
  const double* base[KT];
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
    double w[W];
    load_w2<W>(Wp, Wp2, ldw, i, w);
    double v[KT];
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) v[kk] = (k0 + kk < kend) ? base[kk][i * stride] : 0.0;
    float wh[W], wl[W];
#pragma unroll
    for (int c = 0; c < W; ++c) df_split(w[c], wh[c], wl[c]);
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      float vh, vl;
      df_split(v[kk], vh, vl);
#pragma unroll
      for (int c = 0; c < W; ++c) df_fma(sh[kk * W + c], sl[kk * W + c], vh, vl, wh[c], wl[c]);
    }
  }
  double acc[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) acc[k] = (double)sh[k] + (double)sl[k];  // exact
  block_sum<NP>(acc, red_s, tot);
  for (int t = threadIdx.x; t < NP; t += blockDim.x) {
    const int k = k0 + t / W;
    if (k < kend) part[((size_t)blockIdx.x * K + k) * W + (t % W)] = tot[t];
  }
}

__global__ void k_dots_reduce_df(const double* part, int nchunks, int KW, double* C) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < KW; t += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * KW + t];
    C[t] = s;
  }
}

// W -= V C: the correction V C in pairs, subtracted in FP64; optional Gram + Cholesky
template <int W, int P, bool GRAM>
__global__ void __launch_bounds__(kThreads) k_proj_update_df(VParts<double> V, const double* __restrict__ C,
                                                             double* __restrict__ Wp, double* __restrict__ Wp2,
                                                             int64_t ldw, int64_t n, double* R, double* gdiag,
                                                             unsigned* flags, Red red) {
  constexpr int NP = GRAM ? W * W : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* c_s = reinterpret_cast<float2*>(smem_raw);  // C split into (hi, lo)
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  const int K = V.kx + V.kz;
  for (int t = threadIdx.x; t < K * W; t += blockDim.x) {
    float h, l;
    df_split(C[t], h, l);
    c_s[t] = make_float2(h, l);
  }
  __syncthreads();
  double part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = 0.0;
  const int nzp = V.kz / P;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float dh[W], dl[W];
#pragma unroll
    for (int c = 0; c < W; ++c) dh[c] = dl[c] = 0.f;
    int k = 0;
    for (; k + 8 <= V.kx; k += 8) {  // 8 independent column loads in flight
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = V.X[(int64_t)(k + u) * n + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float vh, vl;
        df_split(v[u], vh, vl);
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const float2 cc = c_s[(k + u) * W + c];
          df_fma(dh[c], dl[c], vh, vl, cc.x, cc.y);
        }
      }
    }
    for (; k < V.kx; ++k) {
      float vh, vl;
      df_split(V.X[(int64_t)k * n + i], vh, vl);
#pragma unroll
      for (int c = 0; c < W; ++c) {
        const float2 cc = c_s[k * W + c];
        df_fma(dh[c], dl[c], vh, vl, cc.x, cc.y);
      }
    }
    constexpr int PB = P >= 8 ? 1 : 8 / P;
    int b = 0;
    for (; b + PB <= nzp; b += PB) {
      double zr[PB][P];
#pragma unroll
      for (int u = 0; u < PB; ++u) load_row<double, P>(V.Z + (int64_t)(b + u) * n * P + i * P, zr[u]);
#pragma unroll
      for (int u = 0; u < PB; ++u)
#pragma unroll
        for (int q = 0; q < P; ++q) {
          float vh, vl;
          df_split(zr[u][q], vh, vl);
          const int kk = V.kx + (b + u) * P + q;
#pragma unroll
          for (int c = 0; c < W; ++c) {
            const float2 cc = c_s[kk * W + c];
            df_fma(dh[c], dl[c], vh, vl, cc.x, cc.y);
          }
        }
    }
    for (; b < nzp; ++b) {
      double zr[P];
      load_row<double, P>(V.Z + (int64_t)b * n * P + i * P, zr);
#pragma unroll
      for (int q = 0; q < P; ++q) {
        float vh, vl;
        df_split(zr[q], vh, vl);
        const int kk = V.kx + b * P + q;
#pragma unroll
        for (int c = 0; c < W; ++c) {
          const float2 cc = c_s[kk * W + c];
          df_fma(dh[c], dl[c], vh, vl, cc.x, cc.y);
        }
      }
    }
    double w[W];
    load_w2<W>(Wp, Wp2, ldw, i, w);
#pragma unroll
    for (int c = 0; c < W; ++c) w[c] -= (double)dh[c] + (double)dl[c];
    store_w2<W>(Wp, Wp2, ldw, i, w);
    if constexpr (GRAM) {
#pragma unroll
      for (int p = 0; p < W; ++p)
#pragma unroll
        for (int q = 0; q < W; ++q) part[p * W + q] = fma(w[p], w[q], part[p * W + q]);
    }
  }
  if constexpr (GRAM) {
    block_sum<NP>(part, red_s, tot);
    if (threadIdx.x < NP) red.part[(size_t)blockIdx.x * NP + threadIdx.x] = tot[threadIdx.x];
    if (last_block_reduce(red.part, NP, red.ticket, tot, red_s))
      if (threadIdx.x == 0) finish_chol(tot, W, R, gdiag, flags);
  }
}

int persistent_rows_df(int64_t n) {
  int g = ceil_div(n, kThreads);
  if (g > kMaxBlocks) g = kMaxBlocks;
  return g < 1 ? 1 : g;
}

}  // namespace

#define NS_P_SWITCH_DF(P, CALL) \
  switch (P) {                  \
    case 1: CALL(1); break;     \
    case 2: CALL(2); break;     \
    case 4: CALL(4); break;     \
    default: CALL(8); break;    \
  }

template <int W>
void proj_dots_df(const VParts<double>& V, const double* Wp, const double* Wp2, int64_t ldw, int64_t n, double* C,
                  double* part, int64_t rows_per_chunk, cudaStream_t s) {
  const int K = V.kx + V.kz;
  if (K == 0) return;
  const int nchunks = ceil_div(n, rows_per_chunk);
  constexpr int KT = df_kt<W>();
  dim3 grid(nchunks, ceil_div(V.kx, KT) + ceil_div(V.kz, KT));
#define CALL(PP) k_proj_dots_df<W, PP><<<grid, kThreads, 0, s>>>(V, Wp, Wp2, ldw, n, rows_per_chunk, part)
  NS_P_SWITCH_DF(V.p, CALL)
#undef CALL
  k_dots_reduce_df<<<ceil_div((int64_t)K * W, kThreads), kThreads, 0, s>>>(part, nchunks, K * W, C);
}

template <int W>
cudaError_t proj_update_df(const VParts<double>& V, const double* C, double* Wp, double* Wp2, int64_t ldw, int64_t n,
                           int gram, double* R, double* gdiag, unsigned* flags, const Red& red, cudaStream_t s) {
  const int K = V.kx + V.kz;
  const size_t smem = sizeof(float2) * (size_t)K * W;
  cudaError_t e = cudaSuccess;
#define CALL1(PP, GG)                                                                                       \
  do {                                                                                                      \
    e = ensure_smem_limit(reinterpret_cast<const void*>(k_proj_update_df<W, PP, GG>), smem);                 \
    if (e != cudaSuccess) return e;                                                                         \
    k_proj_update_df<W, PP, GG><<<persistent_rows_df(n), kThreads, smem, s>>>(V, C, Wp, Wp2, ldw, n, R, gdiag, \
                                                                              flags, red);                  \
  } while (0)
#define CALL(PP)       \
  do {                 \
    if (gram)          \
      CALL1(PP, true); \
    else               \
      CALL1(PP, false); \
  } while (0)
  NS_P_SWITCH_DF(V.p, CALL)
#undef CALL
#undef CALL1
  return e;
}

#define NS_INST_DF(W)                                                                                          \
  template void proj_dots_df<W>(const VParts<double>&, const double*, const double*, int64_t, int64_t, double*, \
                                double*, int64_t, cudaStream_t);                                               \
  template cudaError_t proj_update_df<W>(const VParts<double>&, const double*, double*, double*, int64_t,       \
                                         int64_t, int, double*, double*, unsigned*, const Red&, cudaStream_t);
NS_INST_DF(1)
NS_INST_DF(2)
NS_INST_DF(4)
NS_INST_DF(8)
NS_INST_DF(16)

}  // namespace ns

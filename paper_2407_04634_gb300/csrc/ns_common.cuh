// Shared device helpers of the null-space library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <map>
#include <mutex>
#include <utility>

namespace ns {

constexpr int kThreads = 256;  // block size of every streaming kernel
constexpr int kMaxD = 8;       // largest Lanczos block size

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85, ten rounds.
// Counter layout: (index lo, index hi, stream, 0); key: (seed lo, seed hi).
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox10(U4 c, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0;
    const uint32_t h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
    c = U4{h1 ^ c.y ^ k0, l1, h0 ^ c.w ^ k1, l0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ inline U4 philox_at(uint64_t seed, uint32_t stream, uint64_t i) {
  return philox10(U4{(uint32_t)i, (uint32_t)(i >> 32), stream, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// 53-bit uniform in [0,1) from two 32-bit words
__host__ __device__ inline double u53(uint32_t lo, uint32_t hi) {
  const uint64_t w = (uint64_t)lo | ((uint64_t)hi << 32);
  return (double)(w >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------
// numeric traits
// ---------------------------------------------------------------------------
template <typename T>
struct Unit;
template <>
struct Unit<double> {
  static constexpr double u = 0x1.0p-52;
};
template <>
struct Unit<float> {
  static constexpr double u = 0x1.0p-23;
};

// ---------------------------------------------------------------------------
// deterministic reductions
// ---------------------------------------------------------------------------
__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sums NV per-thread values over the block in a fixed order; the result is
// returned to thread 0 in out[0..NV) (out must hold NV doubles in shared memory
// and red must hold (blockDim/32)*NV doubles).
template <int NV>
__device__ inline void block_sum(const double (&v)[NV], double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = warp_sum(v[k]);
    if (lane == 0) red[warp * NV + k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * NV + k];
    out[k] = s;
  }
  __syncthreads();
}

// block_sum for partials held in T: the 32-lane step runs in T (FP32 shuffles and
// adds for float, which are cheap next to FP64 ones), the cross-warp sum in FP64
template <typename T, int NV>
__device__ inline void block_sum_t(const T (&v)[NV], double* red, double* out) {
  if constexpr (sizeof(T) == 8) {
    double d[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) d[k] = (double)v[k];
    block_sum<NV>(d, red, out);
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float s = (float)v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) red[warp * NV + k] = (double)s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NV; k += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w * NV + k];
      out[k] = s;
    }
    __syncthreads();
  }
}

// "Last block" protocol: each block writes NV partial sums to part[block*NV+k];
// the block that arrives last (atomic ticket) sums all partials in block order
// and returns true with the totals in tot[0..NV) (shared memory).  The ticket
// counter is reset by the last block, so the kernel can be relaunched.  In the last
// block warp w sums the values k = w, w + nwarps, ...: lane l adds blocks l, l + 32,
// ... in order, then a fixed butterfly combines the lanes, so the result does not
// depend on timing; there is one barrier however large NV is.
__device__ inline bool last_block_reduce(double* part, int NV, unsigned* ticket, double* tot, double* red) {
  (void)red;
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < NV; k += nw) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(part + (size_t)b * NV + k);
    s = warp_sum(s);
    if (lane == 0) tot[k] = s;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// small dense FP64 kernels for d x d blocks (row-major, d <= 8), one thread
// ---------------------------------------------------------------------------

// G = R^T R with R upper triangular, positive diagonal.  Returns false when a
// pivot is not positive (numerical rank deficiency).
__host__ __device__ inline bool chol_upper(const double* G, double* R, int d) {
  for (int i = 0; i < d * d; ++i) R[i] = 0.0;
  for (int j = 0; j < d; ++j) {
    double s = G[j * d + j];
    for (int k = 0; k < j; ++k) s -= R[k * d + j] * R[k * d + j];
    if (!(s > 0.0)) return false;
    const double rjj = sqrt(s);
    R[j * d + j] = rjj;
    for (int i = j + 1; i < d; ++i) {
      double t = G[j * d + i];
      for (int k = 0; k < j; ++k) t -= R[k * d + j] * R[k * d + i];
      R[j * d + i] = t / rjj;
    }
  }
  return true;
}

// inverse of an upper triangular matrix
__host__ __device__ inline void inv_upper(const double* R, double* Ri, int d) {
  for (int i = 0; i < d * d; ++i) Ri[i] = 0.0;
  for (int j = 0; j < d; ++j) {
    Ri[j * d + j] = 1.0 / R[j * d + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[i * d + k] * Ri[k * d + j];
      Ri[i * d + j] = -s / R[i * d + i];
    }
  }
}

// C = A B for d x d row-major
__host__ __device__ inline void matmul_dd(const double* A, const double* B, double* C, int d) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += A[i * d + k] * B[k * d + j];
      C[i * d + j] = s;
    }
}

// eigenvalues of a symmetric d x d matrix by cyclic Jacobi rotations
__host__ __device__ inline void sym_eigvals(const double* S, double* ev, int d) {
  double a[kMaxD * kMaxD];
  for (int i = 0; i < d * d; ++i) a[i] = S[i];
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        tot += a[i * d + j] * a[i * d + j];
        if (i != j) off += a[i * d + j] * a[i * d + j];
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < d - 1; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double apq = a[p * d + q];
        if (apq == 0.0) continue;
        const double theta = (a[q * d + q] - a[p * d + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < d; ++k) {  // columns p, q
          const double akp = a[k * d + p], akq = a[k * d + q];
          a[k * d + p] = c * akp - s * akq;
          a[k * d + q] = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {  // rows p, q
          const double apk = a[p * d + k], aqk = a[q * d + k];
          a[p * d + k] = c * apk - s * aqk;
          a[q * d + k] = s * apk + c * aqk;
        }
      }
  }
  for (int i = 0; i < d; ++i) ev[i] = a[i * d + i];
}

// spectral norm of a symmetric d x d matrix
__host__ __device__ inline double sym_norm2(const double* S, int d) {
  double ev[kMaxD];
  sym_eigvals(S, ev, d);
  double m = 0.0;
  for (int i = 0; i < d; ++i) m = fmax(m, fabs(ev[i]));
  return m;
}

// largest and smallest singular value of a general d x d matrix M
__host__ __device__ inline void sv_minmax(const double* M, int d, double* smax, double* smin) {
  double G[kMaxD * kMaxD], ev[kMaxD];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += M[k * d + i] * M[k * d + j];
      G[i * d + j] = s;
    }
  sym_eigvals(G, ev, d);
  double mx = 0.0, mn = 1e300;
  for (int i = 0; i < d; ++i) {
    mx = fmax(mx, ev[i]);
    mn = fmin(mn, ev[i]);
  }
  *smax = sqrt(fmax(mx, 0.0));
  *smin = sqrt(fmax(mn, 0.0));
}

// ---------------------------------------------------------------------------
// compensated FP32-pair arithmetic for FP64 data (the FP64 path's Gram-Schmidt and
// Gram products run on the FP32 pipe): an exact split of an FP64 value into two
// FP32 words, and a multiply-accumulate into an unevaluated pair (TwoProd through
// the FMA residual, TwoSum of Knuth, FastTwoSum of Dekker).  Explicit
// round-to-nearest intrinsics keep the compiler from contracting the transformations.
// ---------------------------------------------------------------------------
// exact split x = hi + lo + r, |r| <= 2^-48 |x|; |x| < 2^-126 gives 0 (such entries
// contribute below 2^-126 to a product of unit vectors)
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const int E = (int)((h32 >> 20) & 0x7FFu);
  const unsigned sgn = h32 & 0x80000000u;
  const int e32 = E - 896;  // FP32 biased exponent of x
  if (e32 <= 0 || e32 >= 255) {
    hi = e32 <= 0 ? 0.f : __uint_as_float(sgn | 0x7F800000u);
    lo = 0.f;
    return;
  }
  hi = __uint_as_float(sgn | ((unsigned)e32 << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
  const unsigned r = l32 & 0x1FFFFFFFu;  // the remaining 29 significand bits: r 2^(E - 1075)
  const int el = E - 1075 + 127;
  const float sc = el >= 1 ? __uint_as_float((unsigned)el << 23) : 0.f;
  lo = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(r), sc)) | sgn);
}

// (sh, sl) += (ah + al)(bh + bl)
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);  // exact: ah bh = p + e
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float s = __fadd_rn(sh, p);  // TwoSum(sh, p) = (s, t)
  const float v = __fsub_rn(s, sh);
  float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));
  t = __fadd_rn(t, __fadd_rn(sl, e));
  sh = __fadd_rn(s, t);  // FastTwoSum(s, t)
  sl = __fsub_rn(t, __fsub_rn(sh, s));
}

// pivot test shared by the last blocks of the CholQR kernels: Cholesky of the d x d
// Gram matrix G (d <= kMaxD); on failure R = I and flag bit 1 is set
__device__ inline void finish_chol(const double* G, int d, double* R, double* gdiag, unsigned* flags) {
  double Rl[kMaxD * kMaxD];
  const bool ok = chol_upper(G, Rl, d);
  if (gdiag)
    for (int i = 0; i < d; ++i) gdiag[i] = G[i * d + i];
  if (!ok) {
    for (int i = 0; i < d * d; ++i) Rl[i] = (i % (d + 1) == 0) ? 1.0 : 0.0;
    if (flags) atomicOr(flags, 1u);
  }
  for (int i = 0; i < d * d; ++i) R[i] = Rl[i];
}

// ---------------------------------------------------------------------------
// vector loads of one row of a row-major n x D panel
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&v)[D]) {
  if constexpr (sizeof(T) * D >= 16 && (sizeof(T) * D) % 16 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
    constexpr int NQ = (int)(sizeof(T) * D / 16);
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const float4 t = __ldg(q + k);
      reinterpret_cast<float4*>(v)[k] = t;
    }
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = __ldg(p + k);
  }
}

template <typename T, int D>
__device__ __forceinline__ void load_row_cg(const T* p, T (&v)[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k) v[k] = p[k];
}

template <typename T, int D>
__device__ __forceinline__ void store_row(T* p, const T (&v)[D]) {
  if constexpr (sizeof(T) * D >= 16 && (sizeof(T) * D) % 16 == 0) {
    constexpr int NQ = (int)(sizeof(T) * D / 16);
#pragma unroll
    for (int k = 0; k < NQ; ++k) reinterpret_cast<float4*>(p)[k] = reinterpret_cast<const float4*>(v)[k];
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) p[k] = v[k];
  }
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Raises the dynamic shared-memory limit of kernel `fn` to at least `bytes` on the
// current device.  The attribute belongs to the (function, device) pair, so it is
// tracked per device; calls from several host threads are serialized.  Any nonzero
// request is raised explicitly: the default 48 KiB covers static plus dynamic shared
// memory, so a kernel with static arrays can need the opt-in below 48 KiB of
// dynamic memory.  Returns the status of cudaFuncSetAttribute (cudaSuccess when
// nothing had to change).
inline cudaError_t ensure_smem_limit(const void* fn, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> raised;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = raised[std::make_pair(fn, dev)];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

}  // namespace ns

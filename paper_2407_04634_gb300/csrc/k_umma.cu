// Thick-restart product on the 5th-generation tensor cores (tcgen05, sm_103a):
//   out(:, c) = Z V_Z(:, sel_c),  Z: n x R Lanczos basis,  V_Z: R x R eigenvectors of T
// (Alg. 2, restart step of Sec. 4.1).  With n ~ 1e6 and R, nsel ~ 100 this is the one
// dense contraction of the method (~20 flop per byte of Z in FP32).
//
// Two kernels share the tcgen05 machinery below.
//
// Mixed path (FP32 basis): every operand is split into bf16 slices (x = x_0 + x_1 [+
// x_2], each slice the bf16 rounding of what the previous ones left), and the
// product is the compensated sum of the slice products x_p y_q with p + q < S
// (3 products for S = 2, 6 for S = 3), accumulated in FP32 in tensor memory.
//
// Tiling: one CTA owns a 128-row tile of Z (the MMA's M), all nsel output columns
// (N <= 256, one TMEM accumulator of N FP32 columns) and walks K = R in chunks of
// 64.  Per chunk every thread loads its share of the FP32 Z tile with coalesced
// loads, splits it and stores the slices into shared memory in the canonical
// K-major no-swizzle layout (8 x 16-byte core matrices); the B slices are copied
// from a pre-split image built once per launch (L2-resident).  One elected thread
// issues the tcgen05.mma instructions and commits them to an mbarrier that every
// thread waits on (bounded) before the shared memory is refilled.  Several CTAs per
// SM overlap one CTA's loads with another's MMAs; their number is capped so that
// their TMEM allocations always fit the SM's 512 columns.
#include <cuda_bf16.h>

#include <algorithm>

#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace ns {
namespace {

constexpr int kTM = 128;       // rows per tile: the MMA's M (cta_group::1)
constexpr int kKC = 64;        // K per chunk: 4 MMAs of K = 16 (bf16)
constexpr int kUThreads = 256; // 8 warps: 2 per TMEM lane quarter in the epilogue
constexpr int kSliceA = kTM * kKC * 2;  // bytes of one A slice per chunk (16 KB)
constexpr uint32_t kLBO = 128;          // byte step between core matrices along K
constexpr uint32_t kSBO = 1024;         // byte step between 8-row groups (8 core matrices of K)

// byte offset of element (row r, k) in a rows x 64 bf16 tile, canonical K-major layout
__host__ __device__ constexpr uint32_t canon(int r, int k) {
  return (uint32_t)((r >> 3) * kSBO + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, fixed version bits 0b001 at [46,49), no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait on an mbarrier phase; false when it gave up (about 0.2 s)
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__host__ __device__ constexpr int tmem_cols(int npad) {
  int c = 32;
  while (c < npad) c <<= 1;
  return c;
}

// split x into S bf16 slices, each the rounding of what the previous ones left
template <int S>
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 (&o)[S]) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    o[s] = __float2bfloat16_rn(x);
    x -= __bfloat162float(o[s]);  // exact: x - rn(x) is representable in FP32
  }
}

// pre-split image of V_Z(:, sel) for every K chunk: [chunk][slice][Npad x 64 canonical]
template <int S>
__global__ void k_umma_bimage(const double* __restrict__ VZ, const int* __restrict__ sel, int nsel, int R, int npad,
                              int nk, __nv_bfloat16* __restrict__ img) {
  const int per_chunk = npad * kKC;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nk * per_chunk; idx += gridDim.x * blockDim.x) {
    const int kc = idx / per_chunk, rem = idx % per_chunk;
    const int c = rem / kKC, kk = rem % kKC, k = kc * kKC + kk;
    double v = (c < nsel && k < R) ? VZ[(int64_t)sel[c] * R + k] : 0.0;
    const uint32_t e = canon(c, kk) / 2;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)v);
      v -= (double)__bfloat162float(b);
      img[((size_t)kc * S + s) * per_chunk + e] = b;
    }
  }
}

template <int S, int D>
__global__ void __launch_bounds__(kUThreads, 1)
    k_restart_umma(const float* __restrict__ Z, int R, int64_t n, const uint4* __restrict__ img, int npad, int nsel,
                   int nl, float* __restrict__ Lnew, float* __restrict__ Znext, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  unsigned char* As = sm;                         // S slices of 128 x 64
  unsigned char* Bs = sm + (size_t)S * kSliceA;   // S slices of npad x 64
  const uint32_t bslice = (uint32_t)npad * kKC * 2;
  const int ncols = tmem_cols(npad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (R + kKC - 1) / kKC;
  const int ksteps16 = (R + 15) / 16;  // MMAs of K = 16 that touch real columns
  constexpr int NP = S == 2 ? 3 : 6;
  constexpr int PA[6] = {0, 0, 1, 1, 0, 2};  // slice pairs (p, q) with p + q < S
  constexpr int PB[6] = {0, 1, 0, 1, 2, 0};
  const uint32_t idesc = idesc_bf16(kTM, npad);
  const uint32_t mbar_a = smem_u32(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_holder;
  uint32_t phase = 0;

  const int64_t ntiles = (n + kTM - 1) / kTM;
  const int r = threadIdx.x & (kTM - 1), half = threadIdx.x >> 7;  // A loader: row, which 4 of the 8 K-cores
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = tile * kTM, i = i0 + r;
    for (int kc = 0; kc < nk; ++kc) {
      // ---- A chunk: rows i0..i0+127, columns kc*64 .. +63 of Z, split into S slices ----
      float v[4][8];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = kc * kKC + (half * 4 + cc) * 8 + u;
          v[cc][u] = (i < n && k < R) ? __ldg(Z + (int64_t)(k / D) * n * D + i * D + (k % D)) : 0.f;
        }
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        __align__(16) __nv_bfloat16 sl[S][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          __nv_bfloat16 o[S];
          split_bf16<S>(v[cc][u], o);
#pragma unroll
          for (int s = 0; s < S; ++s) sl[s][u] = o[s];
        }
        const uint32_t off = canon(r, (half * 4 + cc) * 8);
#pragma unroll
        for (int s = 0; s < S; ++s)
          *reinterpret_cast<uint4*>(As + (size_t)s * kSliceA + off) = *reinterpret_cast<const uint4*>(sl[s]);
      }
      // ---- B chunk: straight copy of the pre-split image ----
      const int nq = S * npad * kKC * 2 / 16;
      const uint4* src = img + (size_t)kc * nq;
      for (int q = threadIdx.x; q < nq; q += blockDim.x) reinterpret_cast<uint4*>(Bs)[q] = __ldg(src + q);
      fence_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) {
        fence_after();
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (kc * 4 + t >= ksteps16) break;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const uint64_t ad = umma_desc(a0 + PA[p] * kSliceA + t * 256, kLBO, kSBO);
            const uint64_t bd = umma_desc(b0 + PB[p] * bslice + t * 256, kLBO, kSBO);
            mma_bf16(tmem, ad, bd, idesc, (kc | t | p) != 0 ? 1u : 0u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                     : "memory");
      }
      if (!mbar_wait(mbar_a, phase)) abort_flag = 1;
      phase ^= 1u;
      __syncthreads();
      if (abort_flag) break;
    }
    if (abort_flag) break;
    fence_after();
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows), half the columns ----
    {
      const int lq = warp & 3, ch = warp >> 2;
      const int64_t row = i0 + 32 * lq + lane;
      const int c_lo = ch * (npad / 2), c_hi = (ch + 1) * (npad / 2);
      for (int c0 = c_lo; c0 < c_hi; c0 += 8) {
        float acc[8];
        tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)c0, acc);
        if (row < n) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int c = c0 + k;
            if (c >= nsel) break;
            if (c < nl) {
              Lnew[row * nl + c] = acc[k];
            } else {
              const int kz = c - nl;
              Znext[(int64_t)(kz / D) * n * D + row * D + (kz % D)] = acc[k];
            }
          }
        }
      }
    }
    fence_before();
    __syncthreads();
  }
  if (abort_flag && threadIdx.x == 0) atomicOr(err, 1u);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// FP64 path: error-free slicing on the tensor cores (the scheme of Ozaki, Ogita,
// Oishi and Rump, 2012).  Row i of Z is written as sum_p zq_p 2^(e_i - 7(p+1)) with
// integer slices |zq_p| <= 127 (e_i: |z_ij| < 2^e_i over the row), column c of V_Z
// as sum_q vq_q 2^(f_c - 7(q+1)).  A product of two slices is an integer below
// 2^14, exact in bf16 x bf16 -> FP32, and the partial sums of the leading groups
// (the (s + 1) slice pairs with p + q = s, s <= 4) stay below 2^24 for R <= 208, so
// their FP32 accumulators hold exact integers (restart_ozaki_supported).  The eight groups s = 0..7 (the 36
// pairs with p + q <= 7) live in eight TMEM accumulators of 64 columns; the
// epilogue adds them exactly in int64 and scales by 2^(e_i + f_c - 63) in FP64.
// Dropped pairs (p + q >= 8) and the truncated tails of the slices leave an error
// below about 2^-47 R 2^(e_i + f_c): the rounding level of an FP64 product.
// ---------------------------------------------------------------------------
constexpr int kOzS = 8;                        // slices per operand
constexpr int kOzKC = 32;                      // K per chunk (2 MMAs of K = 16)
constexpr int kOzN = 64;                       // output columns per pass (8 groups x 64 = 512 TMEM columns)
constexpr int kOzSliceA = kTM * kOzKC * 2;     // 8 KB
constexpr int kOzSliceB = kOzN * kOzKC * 2;    // 4 KB
constexpr int kOzStage = kOzS * (kOzSliceA + kOzSliceB);  // 96 KB
constexpr uint32_t kOzSBO = (kOzKC / 8) * 128; // 512: 8-row groups of a 32-wide K chunk
constexpr int kOzThreads = 512;                // 16 warps: one CTA per SM holds all 512 TMEM
                                               // columns, so the loads in flight come from warps

__host__ __device__ constexpr uint32_t canon32(int r, int k) {
  return (uint32_t)((r >> 3) * kOzSBO + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2);
}

// biased exponent field of x (0 for zero and subnormals, which then slice to 0)
__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// the 8 slices of x relative to the biased exponent Emax of its row/column
// (|x| < 2^(Emax - 1022)), as bf16 bit patterns: sign | integer in [0, 127]
__device__ __forceinline__ void oz_slices(double x, int Emax, uint16_t (&o)[kOzS]) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  const uint16_t sgn = bits < 0 ? 0x8000 : 0;
  unsigned long long M = 0;
  if (E != 0 && Emax != 0) {
    const unsigned long long m = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - Emax + 3;  // M = |x| 2^(56 - e) with e = Emax - 1022, below 2^56
    M = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull);
  }
#pragma unroll
  for (int p = 0; p < kOzS; ++p) {
    const unsigned q = (unsigned)(M >> (49 - 7 * p)) & 127u;
    const float f = __uint_as_float(0x4B000000u | q) - 8388608.0f;  // exactly q
    o[p] = (uint16_t)(__float_as_uint(f) >> 16) | sgn;
  }
}

// 2^k as a double (0 below the normal range)
__device__ __forceinline__ double pow2(int k) {
  if (k < -1022) return 0.0;
  if (k > 1023) k = 1023;
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// largest exponent field of each row of Z (n x R in panels of width D)
template <int D>
__global__ void k_oz_rowexp(const double* __restrict__ Z, int R, int64_t n, int* __restrict__ emax) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int e = 0;
    for (int b = 0; b < R / D; ++b) {
      double v[D];
      load_row<double, D>(Z + (int64_t)b * n * D + i * D, v);
#pragma unroll
      for (int q = 0; q < D; ++q) e = max(e, exp_field(v[q]));
    }
    emax[i] = e;
  }
}

// V_Z(:, sel): column exponents and the slice image [nblock][chunk][slice][64 x 32 canonical]
__global__ void k_oz_bimage(const double* __restrict__ VZ, const int* __restrict__ sel, int nsel, int R, int nkc,
                            int nblk, uint16_t* __restrict__ img, int* __restrict__ fexp) {
  __shared__ int fe[kOzN];
  const int blk = blockIdx.x;  // one CTA per 64-column block
  for (int c = threadIdx.x; c < kOzN; c += blockDim.x) {
    const int cc = blk * kOzN + c;
    int e = 0;
    if (cc < nsel)
      for (int j = 0; j < R; ++j) e = max(e, exp_field(VZ[(int64_t)sel[cc] * R + j]));
    fe[c] = e;
    fexp[cc] = e;
  }
  __syncthreads();
  const int per = nkc * kOzN * kOzKC;
  for (int idx = threadIdx.x; idx < per; idx += blockDim.x) {
    const int kc = idx / (kOzN * kOzKC), rem = idx % (kOzN * kOzKC);
    const int c = rem / kOzKC, kk = rem % kOzKC, k = kc * kOzKC + kk, cc = blk * kOzN + c;
    const double v = (cc < nsel && k < R) ? VZ[(int64_t)sel[cc] * R + k] : 0.0;
    uint16_t o[kOzS];
    oz_slices(v, fe[c], o);
    const size_t base = ((size_t)blk * nkc + kc) * kOzS * (kOzN * kOzKC);
    const uint32_t e = canon32(c, kk) / 2;
#pragma unroll
    for (int p = 0; p < kOzS; ++p) img[base + (size_t)p * (kOzN * kOzKC) + e] = o[p];
  }
}

template <int D>
__global__ void __launch_bounds__(kOzThreads, 1)
    k_restart_ozaki(const double* __restrict__ Z, int R, int64_t n, const int* __restrict__ emax,
                    const uint4* __restrict__ img, const int* __restrict__ fexp, int nsel, int nl,
                    double* __restrict__ Lnew, double* __restrict__ Znext, unsigned* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  __shared__ int fe_s[kOzN];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkc = (R + kOzKC - 1) / kOzKC, nblk = (nsel + kOzN - 1) / kOzN;
  const int ksteps16 = (R + 15) / 16;
  const uint32_t idesc = idesc_bf16(kTM, kOzN);
  const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_holder;
  uint32_t ph[2] = {0u, 0u};  // next parity to wait for, per stage buffer
  int pending[2] = {0, 0};    // a commit on this buffer not yet waited for

  const int r = threadIdx.x & (kTM - 1), kcore = threadIdx.x >> 7;  // A stager: row, which 8 of the 32 K
  const int64_t ntiles = (n + kTM - 1) / kTM;
  for (int64_t tile = blockIdx.x; tile < ntiles && !abort_flag; tile += gridDim.x) {
    const int64_t i0 = tile * kTM, i = i0 + r;
    const int Erow = i < n ? __ldg(emax + i) : 0;
    for (int blk = 0; blk < nblk && !abort_flag; ++blk) {
      __syncthreads();
      if (threadIdx.x < kOzN) fe_s[threadIdx.x] = fexp[blk * kOzN + threadIdx.x < nsel ? blk * kOzN + threadIdx.x : 0];
      for (int kc = 0; kc < nkc; ++kc) {
        const int sb = kc & 1;
        unsigned char* As = sm + (size_t)sb * kOzStage;
        unsigned char* Bs = As + kOzS * kOzSliceA;
        const uint32_t mb = sb ? mb1 : mb0;
        if (pending[sb]) {  // the MMAs that last read this buffer must be done
          if (!mbar_wait(mb, ph[sb])) abort_flag = 1;
          ph[sb] ^= 1u;
          pending[sb] = 0;
        }
        // A: 8 values of row r (one K-core), split into 8 integer slices each
        {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = kc * kOzKC + kcore * 8 + u;
            v[u] = (i < n && k < R) ? __ldg(Z + (int64_t)(k / D) * n * D + i * D + (k % D)) : 0.0;
          }
          __align__(16) uint16_t sl[kOzS][8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            uint16_t o[kOzS];
            oz_slices(v[u], Erow, o);
#pragma unroll
            for (int p = 0; p < kOzS; ++p) sl[p][u] = o[p];
          }
          const uint32_t off = canon32(r, kcore * 8);
#pragma unroll
          for (int p = 0; p < kOzS; ++p)
            *reinterpret_cast<uint4*>(As + (size_t)p * kOzSliceA + off) = *reinterpret_cast<const uint4*>(sl[p]);
        }
        // B: the pre-split image of this (column block, chunk)
        const int nq = kOzS * kOzSliceB / 16;
        const uint4* src = img + ((size_t)blk * nkc + kc) * nq;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) reinterpret_cast<uint4*>(Bs)[q] = __ldg(src + q);
        fence_async_smem();
        __syncthreads();
        if (abort_flag) break;
        if (threadIdx.x == 0) {
          fence_after();
          const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            if (kc * 2 + t >= ksteps16) break;
#pragma unroll
            for (int sg = 0; sg < kOzS; ++sg)
#pragma unroll
              for (int pa = 0; pa <= sg; ++pa) {
                const uint64_t ad = umma_desc(a0 + pa * kOzSliceA + t * 256, kLBO, kOzSBO);
                const uint64_t bd = umma_desc(b0 + (sg - pa) * kOzSliceB + t * 256, kLBO, kOzSBO);
                mma_bf16(tmem + (uint32_t)(sg * kOzN), ad, bd, idesc, (kc | t | pa) != 0 ? 1u : 0u);
              }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                       : "memory");
        }
        pending[sb] = 1;
      }
      // all MMAs of this column block done
      for (int sb = 0; sb < 2; ++sb)
        if (pending[sb]) {
          if (!mbar_wait(sb ? mb1 : mb0, ph[sb])) abort_flag = 1;
          ph[sb] ^= 1u;
          pending[sb] = 0;
        }
      __syncthreads();
      if (abort_flag) break;
      fence_after();
      // epilogue: warp w reads lanes 32 (w % 4) .. +31, 16 of the 64 columns
      const int lq = warp & 3, chh = warp >> 2;
      const int64_t row = i0 + 32 * lq + lane;
      const int Er = row < n ? __ldg(emax + row) : 0;
      for (int c0 = chh * 16; c0 < chh * 16 + 16; c0 += 8) {
        float g[kOzS][8];
#pragma unroll
        for (int sg = 0; sg < kOzS; ++sg)
          tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(sg * kOzN + c0), g[sg]);
        if (row < n) {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int c = blk * kOzN + c0 + k;
            if (c >= nsel) break;
            long long V = 0;
#pragma unroll
            for (int sg = 0; sg < kOzS; ++sg) {
              const long long a = (long long)__float2int_rn(g[sg][k]);  // exact integer
              const int shl = 38 - 7 * sg;  // groups 6, 7 lose their lowest 4 / 11 bits (below 2^-58 relative)
              V += shl >= 0 ? a * (1ll << shl) : (a >> -shl);
            }
            const int Ec = fe_s[c0 + k];
            const double out =
                (Er == 0 || Ec == 0) ? 0.0 : (double)V * pow2((Er - 1022) + (Ec - 1022) - 52);
            if (c < nl) {
              Lnew[row * nl + c] = out;
            } else {
              const int kz = c - nl;
              Znext[(int64_t)(kz / D) * n * D + row * D + (kz % D)] = out;
            }
          }
        }
      }
      fence_before();
      __syncthreads();
    }
  }
  if (abort_flag && threadIdx.x == 0) atomicOr(err, 1u);
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

template <int S>
size_t umma_smem(int npad) {
  return (size_t)S * kSliceA + (size_t)S * npad * kKC * 2;
}

}  // namespace

size_t restart_umma_image_bytes(int R, int nsel, int slices) {
  const int npad = (nsel + 15) / 16 * 16;
  return (size_t)((R + kKC - 1) / kKC) * slices * npad * kKC * 2 + 256;
}

bool restart_umma_supported(int R, int nsel) { return R >= 1 && nsel >= 1 && (nsel + 15) / 16 * 16 <= 256; }

template <int S, int D>
static cudaError_t launch_umma(const float* Z, int R, int64_t n, const uint4* img, int npad, int nsel, int nl,
                               float* Lnew, float* Znext, unsigned* err, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(k_restart_umma<S, D>);
  const int ncols = tmem_cols(npad);
  const int max_ctas = std::max(1, std::min(4, 512 / ncols));  // TMEM: 512 columns per SM
  // the dynamic shared memory is padded so that at most max_ctas CTAs fit on an SM
  // (then every tcgen05.alloc is served without waiting)
  const size_t need = umma_smem<S>(npad);
  const size_t cap_smem = 227 * 1024;
  size_t smem = std::max(need, (size_t)(233472 / (max_ctas + 1)) + 1);
  if (smem > cap_smem) smem = std::max(need, cap_smem);
  cudaError_t e = ensure_smem_limit(fn, smem);
  if (e != cudaSuccess) return e;
  // the whole unified L1 / shared array as shared memory, so that the occupancy query
  // (and the launch) see the largest carveout
  e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // resident CTAs per SM from the kernel's own registers and shared memory (plus the
  // 1 KB the driver reserves per CTA), capped by the TMEM columns
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  const int regs_cta = ((fa.numRegs + 7) / 8) * 8 * kUThreads;
  const int by_regs = regs_cta > 0 ? 65536 / regs_cta : 1;
  const int by_smem = (int)((size_t)smem_sm / (smem + fa.sharedSizeBytes + 1024));
  const int per_sm = std::max(1, std::min({by_regs, by_smem, max_ctas}));
  const int64_t ntiles = (n + kTM - 1) / kTM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sms * per_sm));
  k_restart_umma<S, D><<<grid, kUThreads, smem, s>>>(Z, R, n, img, npad, nsel, nl, Lnew, Znext, err);
  return cudaSuccess;
}

size_t restart_ozaki_scratch_bytes(int64_t n, int R, int nsel) {
  const int nkc = (R + kOzKC - 1) / kOzKC, nblk = (nsel + kOzN - 1) / kOzN;
  return (size_t)nblk * nkc * kOzS * kOzSliceB + sizeof(int) * ((size_t)nblk * kOzN + (size_t)n) + 512;
}

// Exactness of the slice-pair sums: group s adds (s + 1) pairs over R terms below
// 2^14 each, so groups s <= 4 stay below 2^24 (exact in FP32) for R <= 208.  Groups
// s >= 5 may round, but they weigh 2^(-7 s - 14) relative to the leading group, so
// their FP32 rounding stays below 2^-56 of the result: beyond FP64 precision.
bool restart_ozaki_supported(int R, int nsel) { return R >= 1 && R <= 208 && nsel >= 1; }

cudaError_t restart_gemm_ozaki(const double* Z, int d, int R, const double* VZ, const int* sel, int nsel, int nl,
                               int64_t n, double* Lnew, double* Znext, void* scratch, unsigned* err, cudaStream_t s) {
  if (nsel == 0 || n == 0) return cudaSuccess;
  if (!restart_ozaki_supported(R, nsel)) return cudaErrorInvalidValue;
  const int nkc = (R + kOzKC - 1) / kOzKC, nblk = (nsel + kOzN - 1) / kOzN;
  unsigned char* sc = static_cast<unsigned char*>(scratch);
  uint16_t* img = reinterpret_cast<uint16_t*>(sc);
  int* fexp = reinterpret_cast<int*>(sc + (size_t)nblk * nkc * kOzS * kOzSliceB);
  int* emax = fexp + (size_t)nblk * kOzN;
  const int g = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  switch (d) {
    case 1: k_oz_rowexp<1><<<g, 256, 0, s>>>(Z, R, n, emax); break;
    case 2: k_oz_rowexp<2><<<g, 256, 0, s>>>(Z, R, n, emax); break;
    case 4: k_oz_rowexp<4><<<g, 256, 0, s>>>(Z, R, n, emax); break;
    default: k_oz_rowexp<8><<<g, 256, 0, s>>>(Z, R, n, emax); break;
  }
  k_oz_bimage<<<nblk, 256, 0, s>>>(VZ, sel, nsel, R, nkc, nblk, img, fexp);
  const size_t smem = 2 * (size_t)kOzStage;  // two stage buffers; one CTA per SM (all 512 TMEM columns)
  const void* fn;
  switch (d) {
    case 1: fn = reinterpret_cast<const void*>(k_restart_ozaki<1>); break;
    case 2: fn = reinterpret_cast<const void*>(k_restart_ozaki<2>); break;
    case 4: fn = reinterpret_cast<const void*>(k_restart_ozaki<4>); break;
    default: fn = reinterpret_cast<const void*>(k_restart_ozaki<8>); break;
  }
  cudaError_t e = ensure_smem_limit(fn, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (n + kTM - 1) / kTM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms));
  const uint4* im = reinterpret_cast<const uint4*>(img);
  switch (d) {
    case 1: k_restart_ozaki<1><<<grid, kOzThreads, smem, s>>>(Z, R, n, emax, im, fexp, nsel, nl, Lnew, Znext, err); break;
    case 2: k_restart_ozaki<2><<<grid, kOzThreads, smem, s>>>(Z, R, n, emax, im, fexp, nsel, nl, Lnew, Znext, err); break;
    case 4: k_restart_ozaki<4><<<grid, kOzThreads, smem, s>>>(Z, R, n, emax, im, fexp, nsel, nl, Lnew, Znext, err); break;
    default: k_restart_ozaki<8><<<grid, kOzThreads, smem, s>>>(Z, R, n, emax, im, fexp, nsel, nl, Lnew, Znext, err); break;
  }
  return cudaSuccess;
}

cudaError_t restart_gemm_umma(const float* Z, int d, int R, const double* VZ, const int* sel, int nsel, int nl,
                              int64_t n, float* Lnew, float* Znext, void* image, unsigned* err, int slices,
                              cudaStream_t s) {
  if (nsel == 0 || n == 0) return cudaSuccess;
  if (!restart_umma_supported(R, nsel) || !(slices == 2 || slices == 3)) return cudaErrorInvalidValue;
  const int npad = (nsel + 15) / 16 * 16;
  const int nk = (R + kKC - 1) / kKC;
  __nv_bfloat16* img = static_cast<__nv_bfloat16*>(image);
  const int total = nk * npad * kKC;
  const int g = std::min(1024, (total + 255) / 256);
  if (slices == 2)
    k_umma_bimage<2><<<g, 256, 0, s>>>(VZ, sel, nsel, R, npad, nk, img);
  else
    k_umma_bimage<3><<<g, 256, 0, s>>>(VZ, sel, nsel, R, npad, nk, img);
  const uint4* im = static_cast<const uint4*>(image);
#define NS_UMMA(SS, DD) return launch_umma<SS, DD>(Z, R, n, im, npad, nsel, nl, Lnew, Znext, err, s)
  if (slices == 2) {
    switch (d) {
      case 1: NS_UMMA(2, 1);
      case 2: NS_UMMA(2, 2);
      case 4: NS_UMMA(2, 4);
      default: NS_UMMA(2, 8);
    }
  }
  switch (d) {
    case 1: NS_UMMA(3, 1);
    case 2: NS_UMMA(3, 2);
    case 4: NS_UMMA(3, 4);
    default: NS_UMMA(3, 8);
  }
#undef NS_UMMA
}

}  // namespace ns

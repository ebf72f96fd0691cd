// Batched form: thousands of independent SPD matrices (graph Laplacians) solved in
// ONE persistent launch.  Each CTA pops an instance index from an atomic work queue
// (instances ordered by decreasing nnz) and runs the whole method for it on its
// own: B = A + eps D applied by a CTA-wide SpMV, the single-vector Lanczos
// recurrence (d = 1), the W recurrence of Sec. 4.2 with partial
// reorthogonalization, the projected eigenproblem (FP64 parallel Jacobi in shared
// memory), locking, thick restart (Sec. 4.1, retention capped at dimK/2), the
// stopping rule of Sec. 4.3, and the FP64 CG projection onto null(A) followed by
// FP64 re-orthonormalization.  Vectors are FP32, every scalar of the projected
// problem FP64.  No CTA ever waits for another one.
#include <algorithm>

#include "../../include/nullspace.h"
#include "ns_common.cuh"
#include "ns_kernels.cuh"
#include "ns_batch.cuh"

namespace ns {

// ---------------------------------------------------------------------------
// CTA-level helpers (every thread of the block calls them)
// ---------------------------------------------------------------------------
struct CtaRed {
  double w[kBThreads / 32];
  double out[4];
};

__device__ inline double cta_sum(double v, CtaRed& r) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) r.w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += r.w[k];
    r.out[0] = s;
  }
  __syncthreads();
  const double res = r.out[0];
  __syncthreads();
  return res;
}

__device__ inline double cta_max(double v, CtaRed& r) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) r.w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s = fmax(s, r.w[k]);
    r.out[0] = s;
  }
  __syncthreads();
  const double res = r.out[0];
  __syncthreads();
  return res;
}

// two sums at once
__device__ inline void cta_sum2(double a, double b, CtaRed& r, double& ra, double& rb) {
  a = warp_sum(a);
  b = warp_sum(b);
  __shared__ double w2[kBThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    r.w[threadIdx.x >> 5] = a;
    w2[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s += r.w[k];
      t += w2[k];
    }
    r.out[0] = s;
    r.out[1] = t;
  }
  __syncthreads();
  ra = r.out[0];
  rb = r.out[1];
  __syncthreads();
}

// Philox normals of the start / replacement vectors (same recipe as the streams of
// the single-instance path: Box-Muller on pairs, element e takes the pair e/2)
__device__ inline float gauss_at(uint64_t seed, uint32_t stream, int64_t e) {
  const U4 w = philox_at(seed, stream, (uint64_t)(e >> 1));
  const uint64_t w0 = (uint64_t)w.x | ((uint64_t)w.y << 32);
  const uint64_t w1 = (uint64_t)w.z | ((uint64_t)w.w << 32);
  const double u1 = (double)((w0 >> 11) + 1) * 0x1.0p-53;
  const double u2 = (double)(w1 >> 11) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return (float)((e & 1) ? r * sn : r * cs);
}

// y_i = sum_k a_ik x_k + eps D_i x_i - beta xprev_i ; returns per-thread partial of x_i y_i.
// LANES threads share one row.
template <int LANES>
__device__ inline double cta_apply(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                   const float* __restrict__ val, int n, const float* __restrict__ x,
                                   const float* __restrict__ Dv, float eps, const float* __restrict__ xprev,
                                   float beta, float* __restrict__ y) {
  float part = 0.f;
  if constexpr (LANES == 1) {  // thread per row, two rows at a time, four entries of each per round
    const int nt = blockDim.x;
    for (int i0 = threadIdx.x; i0 < n; i0 += 2 * nt) {
      const int i1 = i0 + nt;
      const bool h1 = i1 < n;
      int64_t k0 = rp[i0];
      const int64_t e0 = rp[i0 + 1];
      int64_t k1 = h1 ? rp[i1] : 0;
      const int64_t e1 = h1 ? rp[i1 + 1] : 0;
      float s0 = 0.f, s1 = 0.f;
      while (k0 < e0 || k1 < e1) {
        int c0[4], c1[4];
        float v0[4], v1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool a0 = k0 + u < e0, a1 = k1 + u < e1;
          c0[u] = a0 ? __ldg(col + k0 + u) : i0;
          v0[u] = a0 ? __ldg(val + k0 + u) : 0.f;
          c1[u] = a1 ? __ldg(col + k1 + u) : i0;
          v1[u] = a1 ? __ldg(val + k1 + u) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          s0 = fmaf(v0[u], x[c0[u]], s0);
          s1 = fmaf(v1[u], x[c1[u]], s1);
        }
        k0 += 4;
        k1 += 4;
      }
      {
        const float xi = x[i0];
        s0 = fmaf(eps * Dv[i0], xi, s0);
        if (xprev) s0 = fmaf(-beta, xprev[i0], s0);
        y[i0] = s0;
        part = fmaf(xi, s0, part);
      }
      if (h1) {
        const float xi = x[i1];
        s1 = fmaf(eps * Dv[i1], xi, s1);
        if (xprev) s1 = fmaf(-beta, xprev[i1], s1);
        y[i1] = s1;
        part = fmaf(xi, s1, part);
      }
    }
    return (double)part;
  }
  const int lane = threadIdx.x % LANES, grp = threadIdx.x / LANES, ngrp = blockDim.x / LANES;
  for (int base = 0; base < n; base += ngrp) {  // uniform trip count for the shuffles
    const int i = base + grp;
    float s = 0.f;
    if (i < n) {
      const int64_t e = rp[i + 1];
      for (int64_t k = rp[i] + lane; k < e; k += LANES) s = fmaf(__ldg(val + k), x[__ldg(col + k)], s);
    }
    if constexpr (LANES > 1) {
#pragma unroll
      for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0 && i < n) {
      const float xi = x[i];
      s = fmaf(eps * Dv[i], xi, s);
      if (xprev) s = fmaf(-beta, xprev[i], s);
      y[i] = s;
      part = fmaf(xi, s, part);
    }
  }
  return (double)part;
}

// FP64 SpMV y = A x for the refinement (LANES = 1, thread per row)
__device__ inline void cta_spmv64(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                  const double* __restrict__ val, int n, const double* __restrict__ x,
                                  double* __restrict__ y) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s = fma(__ldg(val + k), x[__ldg(col + k)], s);
    y[i] = s;
  }
}

// ---------------------------------------------------------------------------
// projected eigenproblem: cyclic Jacobi with the round-robin ordering (R/2
// disjoint rotations per round, applied in parallel), FP64, shared memory.
// A (R x R, row-major) is destroyed; on return th[] holds the eigenvalues in
// ascending order and V[i*R + k] component i of eigenvector k.
// ---------------------------------------------------------------------------
struct JacobiScratch {
  int p[kBMaxR / 2 + 1], q[kBMaxR / 2 + 1];
  double c[kBMaxR / 2 + 1], s[kBMaxR / 2 + 1];
  int perm[kBMaxR];
};

// Cyclic Jacobi sweeps in precision F on A (R x R, row-major, symmetric); V
// accumulates the rotations (V <- V J).  Stops when the squared off-diagonal
// mass is at most rel * the squared Frobenius norm, or after max_sweeps.
template <typename F>
__device__ int cta_jacobi_sweeps(F* A, F* V, int R, bool init_identity, double rel, int max_sweeps,
                                 JacobiScratch& js, CtaRed& cr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (init_identity) {
    for (int t = tid; t < R * R; t += nt) V[t] = (t / R == t % R) ? F(1) : F(0);
    __syncthreads();
  }
  const int Rp = R + (R & 1);  // one dummy index when R is odd
  const int np = Rp / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int t = tid; t < R * R; t += nt) {
      const double a = (double)A[t];
      tot += a * a;
      if (t / R != t % R) off += a * a;
    }
    cta_sum2(off, tot, cr, off, tot);
    if (off <= rel * tot || off == 0.0) break;
    for (int round = 0; round < Rp - 1; ++round) {
      if (tid < np) {  // circle method: position 0 fixed, the others rotate
        const int k = tid;
        const int a = (k == 0) ? 0 : 1 + (k - 1 + round) % (Rp - 1);
        const int kk = Rp - 1 - k;
        const int b = 1 + (kk - 1 + round) % (Rp - 1);
        const int pp = a < b ? a : b, qq = a < b ? b : a;
        F c = F(1), sn = F(0);
        if (qq < R) {
          const F apq = A[pp * R + qq];
          if (apq != F(0)) {
            const F theta = (A[qq * R + qq] - A[pp * R + pp]) / (F(2) * apq);
            const F t = (theta >= F(0) ? F(1) : F(-1)) / (fabs(theta) + sqrt(theta * theta + F(1)));
            c = F(1) / sqrt(t * t + F(1));
            sn = t * c;
          }
        }
        js.p[k] = pp;
        js.q[k] = qq < R ? qq : pp;
        js.c[k] = (double)c;
        js.s[k] = (qq < R) ? (double)sn : 0.0;
      }
      __syncthreads();
      // the np rotations of a round act on disjoint index pairs, so A <- M A M^T is
      // applied in one pass: thread -> 2 x 2 block (pairs a, b), new block =
      // M_a X M_b^T; V <- V M^T on the pairs' columns in the same pass.  A dummy
      // pair (odd R) has q == p and the identity rotation.
      for (int t = tid; t < np * np; t += nt) {
        const int a = t / np, b = t % np;
        const int pa = js.p[a], qa = js.q[a], pb = js.p[b], qb = js.q[b];
        const F ca = (F)js.c[a], sa = (F)js.s[a], cb = (F)js.c[b], sb = (F)js.s[b];
        const bool ra = qa != pa, rb = qb != pb;
        const F x00 = A[pa * R + pb];
        const F x01 = rb ? A[pa * R + qb] : F(0);
        const F x10 = ra ? A[qa * R + pb] : F(0);
        const F x11 = (ra && rb) ? A[qa * R + qb] : F(0);
        const F y00 = ca * x00 - sa * x10, y01 = ca * x01 - sa * x11;  // rows: M_a X
        const F y10 = sa * x00 + ca * x10, y11 = sa * x01 + ca * x11;
        A[pa * R + pb] = cb * y00 - sb * y01;  // columns: (M_a X) M_b^T
        if (rb) A[pa * R + qb] = sb * y00 + cb * y01;
        if (ra) A[qa * R + pb] = cb * y10 - sb * y11;
        if (ra && rb) A[qa * R + qb] = sb * y10 + cb * y11;
      }
      for (int t = tid; t < np * R; t += nt) {
        const int k = t / R, i = t % R;
        const int pp = js.p[k], qq = js.q[k];
        if (pp == qq) continue;
        const F c = (F)js.c[k], sn = (F)js.s[k];
        const F vip = V[i * R + pp], viq = V[i * R + qq];
        V[i * R + pp] = c * vip - sn * viq;
        V[i * R + qq] = sn * vip + c * viq;
      }
      __syncthreads();
    }
  }
  return sweep;
}

// Projected eigenproblem of T (Alg. 2 (the projected matrix T)), FP64 result at a fraction of the
// FP64 work of a cold FP64 Jacobi:
//   1. Jacobi in FP32 on a rounded copy of T           -> V32 (orthogonal to ~1e-7)
//   2. FP64: V = V32 (3I - V32^T V32)/2 (one Newton-Schulz step, orthonormal in FP64)
//   3. FP64: B = V^T T V (T applied from its arrow + tridiagonal structure)
//   4. FP64 Jacobi on B (nearly diagonal: one or two sweeps) -> Q
//   5. eigenvalues diag(B), eigenvectors V Q, sorted ascending.
// As holds T on entry (row-major) and is destroyed; Wt is R*R doubles of scratch.
// On return th[k] is the k-th smallest eigenvalue and Vs[i*R + k] component i of
// its eigenvector.
__device__ int2 cta_eig(double* As, double* Vs, double* Wt, double* th, int R, int r0, const double* diag,
                        const double* F, const double* beta, JacobiScratch& js, CtaRed& cr) {
  const int tid = threadIdx.x, nt = blockDim.x, RR = R * R;
  float* A32 = reinterpret_cast<float*>(Wt);
  float* V32 = A32 + RR;
  for (int t = tid; t < RR; t += nt) A32[t] = (float)As[t];
  __syncthreads();
  const int sw32 = cta_jacobi_sweeps<float>(A32, V32, R, true, 1e-11, 12, js, cr);
  for (int t = tid; t < RR; t += nt) Vs[t] = (double)V32[t];
  __syncthreads();
  for (int t = tid; t < RR; t += nt) {  // As = 1.5 I - 0.5 V^T V
    const int r = t / R, c = t % R;
    double g = 0.0;
    for (int k = 0; k < R; ++k) g = fma(Vs[k * R + r], Vs[k * R + c], g);
    As[t] = (r == c ? 1.5 : 0.0) - 0.5 * g;
  }
  __syncthreads();
  for (int t = tid; t < RR; t += nt) {  // Wt = V As
    const int r = t / R, c = t % R;
    double g = 0.0;
    for (int k = 0; k < R; ++k) g = fma(Vs[r * R + k], As[k * R + c], g);
    Wt[t] = g;
  }
  __syncthreads();
  for (int t = tid; t < RR; t += nt) {  // Vs = T Wt
    const int r = t / R, c = t % R;
    double g = diag[r] * Wt[t];
    if (r < r0) g = fma(F[r], Wt[r0 * R + c], g);
    if (r == r0)
      for (int i = 0; i < r0; ++i) g = fma(F[i], Wt[i * R + c], g);
    if (r >= r0 && r + 1 < R) g = fma(beta[r], Wt[(r + 1) * R + c], g);
    if (r - 1 >= r0) g = fma(beta[r - 1], Wt[(r - 1) * R + c], g);
    Vs[t] = g;
  }
  __syncthreads();
  for (int t = tid; t < RR; t += nt) {  // As = Wt^T (T Wt)
    const int r = t / R, c = t % R;
    double g = 0.0;
    for (int k = 0; k < R; ++k) g = fma(Wt[k * R + r], Vs[k * R + c], g);
    As[t] = g;
  }
  __syncthreads();
  for (int t = tid; t < RR; t += nt) {  // exact symmetry
    const int r = t / R, c = t % R;
    if (r < c) {
      const double m = 0.5 * (As[t] + As[c * R + r]);
      As[t] = m;
      As[c * R + r] = m;
    }
  }
  __syncthreads();
  const int sw64 = cta_jacobi_sweeps<double>(As, Vs, R, true, 1e-28, 20, js, cr);
  for (int k = tid; k < R; k += nt) th[k] = As[k * R + k];
  __syncthreads();
  if (tid == 0) {  // ascending order (insertion sort on indices)
    for (int i = 0; i < R; ++i) js.perm[i] = i;
    for (int i = 1; i < R; ++i) {
      const int key = js.perm[i];
      const double kv = th[key];
      int j = i - 1;
      while (j >= 0 && th[js.perm[j]] > kv) {
        js.perm[j + 1] = js.perm[j];
        --j;
      }
      js.perm[j + 1] = key;
    }
  }
  __syncthreads();
  for (int t = tid; t < RR; t += nt) {  // As = Wt Q, columns in ascending order
    const int r = t / R, c = js.perm[t % R];
    double g = 0.0;
    for (int k = 0; k < R; ++k) g = fma(Wt[r * R + k], Vs[k * R + c], g);
    As[t] = g;
  }
  __syncthreads();
  for (int k = tid; k < R; k += nt) Wt[k] = th[js.perm[k]];
  __syncthreads();
  for (int k = tid; k < R; k += nt) th[k] = Wt[k];
  for (int t = tid; t < RR; t += nt) Vs[t] = As[t];
  __syncthreads();
  return make_int2(sw32, sw64);
}

// ---------------------------------------------------------------------------
// one classical Gram-Schmidt pass of q against X(:, 0:kx) and Z(:, 0:kz)
// (column-major, leading dimension n); coefficients accumulated in FP64
// ---------------------------------------------------------------------------
constexpr int kBChunk = 8;
constexpr int kBCoef = kBMaxR + kBMaxLock + kBChunk;  // coefficient slots per vector

__device__ inline float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One classical Gram-Schmidt pass of NV (1 or 2) vectors against X(:, 0:kx) and
// Z(:, 0:kz) (column-major, leading dimension n), FP32 throughout.  Both vectors
// share every column load; each row issues kBChunk (dots) or 16 (update)
// independent loads before its FMA chain, so L2 latency overlaps.
template <int NV>
__device__ void cta_cgs_n(float* q0, float* q1, const float* X, int kx, const float* Z, int kz, int n,
                          float* coef) {
  __shared__ float w8[kBThreads / 32][2 * kBChunk];
  const int K = kx + kz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k0 = 0; k0 < K; k0 += kBChunk) {
    const float* cp[kBChunk];
#pragma unroll
    for (int c = 0; c < kBChunk; ++c) {
      const int k = min(k0 + c, K - 1);
      cp[c] = (k < kx) ? X + (int64_t)k * n : Z + (int64_t)(k - kx) * n;
    }
    float acc[NV][kBChunk];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
      for (int c = 0; c < kBChunk; ++c) acc[t][c] = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float v[kBChunk];
#pragma unroll
      for (int c = 0; c < kBChunk; ++c) v[c] = cp[c][i];
      const float qa = q0[i];
#pragma unroll
      for (int c = 0; c < kBChunk; ++c) acc[0][c] = fmaf(v[c], qa, acc[0][c]);
      if constexpr (NV > 1) {
        const float qb = q1[i];
#pragma unroll
        for (int c = 0; c < kBChunk; ++c) acc[NV - 1][c] = fmaf(v[c], qb, acc[NV - 1][c]);
      }
    }
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
      for (int c = 0; c < kBChunk; ++c) {
        const float r = warp_sum_f(acc[t][c]);
        if (lane == 0) w8[warp][t * kBChunk + c] = r;
      }
    __syncthreads();
    if (threadIdx.x < NV * kBChunk) {
      const int t = threadIdx.x / kBChunk, c = threadIdx.x % kBChunk;
      if (k0 + c < K) {
        float sm = 0.f;
        for (int w = 0; w < nw; ++w) sm += w8[w][threadIdx.x];
        coef[t * kBCoef + k0 + c] = sm;
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float va = q0[i], vb = 0.f;
    if constexpr (NV > 1) vb = q1[i];
    for (int k0 = 0; k0 < K; k0 += 16) {
      float b[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int k = k0 + c;
        b[c] = (k < K) ? ((k < kx) ? X[(int64_t)k * n + i] : Z[(int64_t)(k - kx) * n + i]) : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int k = k0 + c;
        if (k < K) {
          va = fmaf(-coef[k], b[c], va);
          if constexpr (NV > 1) vb = fmaf(-coef[kBCoef + k], b[c], vb);
        }
      }
    }
    q0[i] = va;
    if constexpr (NV > 1) q1[i] = vb;
  }
  __syncthreads();
}

__device__ inline void cta_cgs(float* q, const float* X, int kx, const float* Z, int kz, int n, float* coef,
                               CtaRed&) {
  cta_cgs_n<1>(q, nullptr, X, kx, Z, kz, n, coef);
}

// ||q||_2 (FP64 accumulation of FP32 squares)
__device__ inline double cta_norm(const float* q, int n, CtaRed& cr) {
  double loc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) loc += (double)q[i] * (double)q[i];
  return sqrt(cta_sum(loc, cr));
}

__device__ inline void cta_scale_to(const float* q, float* out, float f, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = q[i] * f;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// one instance, the whole method (all threads of the CTA)
// ---------------------------------------------------------------------------
struct BState {
  double alpha[kBMaxR + 1], beta[kBMaxR + 1];  // Xi_j, Gamma_j (d = 1)
  double theta_keep[kBMaxR], F[kBMaxR];        // retained Ritz values and the arrow row
  double th[kBMaxR], res[kBMaxR];              // eigenvalues of T, Ritz residuals
  double tdiag[kBMaxR];                        // diagonal of T
  double wz[3][kBMaxR + 1];                    // rotating columns of W (active blocks)
  double wx[3][kBMaxLock];                     // ... rows of the locked vectors
  double xth[kBMaxLock], xrho[kBMaxLock];
  float coef[2 * kBCoef];
  int lock_list[kBMaxR], keep_list[kBMaxR];
  int ncand, nkeep, nsmall, flags;
};

__device__ void replace_vec(float* dst, uint64_t seed, uint32_t stream, int n, const float* X, int nlock,
                            const float* Z, int kz, BState& S, CtaRed& cr) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = gauss_at(seed, stream, i);
  __syncthreads();
  cta_cgs(dst, X, nlock, Z, kz, n, S.coef, cr);
  cta_cgs(dst, X, nlock, Z, kz, n, S.coef, cr);
  const double nr = cta_norm(dst, n, cr);
  cta_scale_to(dst, dst, (float)(1.0 / nr), n);
}

template <int LANES>
__device__ void solve_instance(const BatchArgs& a, int inst, float* ws32, double* ws64, double* As, double* Vs,
                               double* Wt, BState& S, JacobiScratch& js, CtaRed& cr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long clk0 = clock64();
  const int n = a.nrows[inst];
  const int64_t* rp = a.rowptr + a.rp_off[inst];
  const int* col = a.col + a.nz_off[inst];
  const float* val = a.val + a.nz_off[inst];
  const double* val64 = a.val64 + a.nz_off[inst];
  const int R = a.R;
  const uint64_t seed = a.seed + (uint64_t)inst;  // instance i draws from the streams of seed + i
  float* Z = ws32;                        // n x (R+1) Lanczos basis, column-major
  float* Zt = Z + (int64_t)n * (R + 1);   // n x R restart / locking scratch
  float* X = Zt + (int64_t)n * R;         // n x kBMaxLock locked vectors
  float* Dv = X + (int64_t)n * kBMaxLock; // perturbation diagonal
  float* qp = Dv + n;                     // Q'
  const float eps = (float)a.eps;

  // ||A||_inf and the longest row, D ~ U[0,1), start vector ~ N(0,1)
  double mx = 0.0, ml = 0.0;
  for (int i = tid; i < n; i += nt) {
    double sm = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) sm += fabs(val64[k]);
    mx = fmax(mx, sm);
    ml = fmax(ml, (double)(rp[i + 1] - rp[i]));
    const U4 w = philox_at(seed, 0u, (uint64_t)i);
    Dv[i] = (float)u53(w.x, w.y);
    Z[i] = gauss_at(seed, 1u, i);
  }
  const double normB = cta_max(mx, cr) + a.eps;
  const double maxrow = cta_max(ml, cr);
  const double u = 0x1.0p-23;
  const double u_d = sqrt(fmax(maxrow, 1.0)) * u * normB, u_ro = sqrt(u), bd_tol = 100.0 * u_d;
  const double tol_eff = fmax(a.tol, 1e-5);
  const long long max_mv = a.max_matvec > 0 ? (long long)a.max_matvec : min(100LL * n + 50LL * R, 1000000LL);
  {
    const double nq = cta_norm(Z, n, cr);
    cta_scale_to(Z, Z, (float)(1.0 / nq), n);
  }
  int k0 = 0, nlock = 0, status = 0;
  // SM cycles by phase (thread 0; every boundary follows a barrier):
  // 0 Lanczos steps, 1 partial reorthogonalization, 2 projected eigenproblem,
  // 3 locking, 4 thick restart, 5 refinement
  long long cyc[6] = {0, 0, 0, 0, 0, 0};
  long long tmark = clock64();
  long long sweeps32 = 0, sweeps64 = 0;
#define PHASE(k)                      \
  do {                                \
    const long long tnow = clock64(); \
    cyc[k] += tnow - tmark;           \
    tmark = tnow;                     \
  } while (0)
  uint32_t bdcount = 0;
  long long matvecs = 0, restarts = 0, reorths = 0, ev_first = -1, ev_last = -1;
  int ev_first_k = 0, ev_total = 0, ev_count = 0;
  double theta_max = 0.0;
  while (true) {
    const int r0 = k0;
    // ---- first step of the cycle (Alg. 2 (the first step of a cycle)) ----
    {
      const float* q = Z + (int64_t)r0 * n;
      const double al = cta_sum(cta_apply<LANES>(rp, col, val, n, q, Dv, eps, nullptr, 0.f, qp), cr);
      ++matvecs;
      cta_cgs(qp, X, nlock, Z, r0 + 1, n, S.coef, cr);
      cta_cgs(qp, X, nlock, Z, r0 + 1, n, S.coef, cr);
      double b = cta_norm(qp, n, cr);
      float* qn = Z + (int64_t)(r0 + 1) * n;
      if (b <= bd_tol) {
        replace_vec(qn, seed, 2u + bdcount++, n, X, nlock, Z, r0 + 1, S, cr);
        b = 0.0;
      } else {
        cta_scale_to(qp, qn, (float)(1.0 / b), n);
      }
      if (tid == 0) {
        S.alpha[r0] = al;
        S.beta[r0] = b;
      }
      for (int t = tid; t <= r0; t += nt) {
        if (t < r0) S.wz[r0 % 3][t] = u_d;
        S.wz[(r0 + 1) % 3][t] = u_d;
      }
      for (int k = tid; k < nlock; k += nt) S.wx[r0 % 3][k] = S.wx[(r0 + 1) % 3][k] = u_d;
      __syncthreads();
    }
    // ---- inner steps (Alg. 2 (the block recurrence of a cycle)) ----
    for (int j = r0 + 1; j < R; ++j) {
      float* qj = Z + (int64_t)j * n;
      const float* qm = Z + (int64_t)(j - 1) * n;
      float* qn = Z + (int64_t)(j + 1) * n;
      const double al = cta_sum(cta_apply<LANES>(rp, col, val, n, qj, Dv, eps, qm, (float)S.beta[j - 1], qp), cr);
      ++matvecs;
      double loc = 0.0;
      for (int i = tid; i < n; i += nt) {
        const float v = fmaf(-(float)al, qj[i], qp[i]);
        qp[i] = v;
        loc += (double)v * (double)v;
      }
      const double b = sqrt(cta_sum(loc, cr));
      if (tid == 0) S.alpha[j] = al;
      if (b <= bd_tol) {  // breakdown: fresh direction, coupling zero, column j+1 of W reset
        replace_vec(qn, seed, 2u + bdcount++, n, X, nlock, Z, j + 1, S, cr);
        if (tid == 0) S.beta[j] = 0.0;
        for (int t = tid; t <= j; t += nt) S.wz[(j + 1) % 3][t] = u_d;
        for (int k = tid; k < nlock; k += nt) S.wx[(j + 1) % 3][k] = u_d;
        __syncthreads();
        continue;
      }
      cta_scale_to(qp, qn, (float)(1.0 / b), n);
      if (tid == 0) {
        S.beta[j] = b;
        S.flags = 0;
      }
      __syncthreads();
      // W recurrence, column j+1 (Sec. 4.2; d = 1 so every block norm is a scalar)
      const double g = 1.0 / b, nXj = fabs(al), nGjm1 = S.beta[j - 1], ud2 = 2.0 * u_d;
      double* cj = S.wz[j % 3];
      double* cjm1 = S.wz[(j + 2) % 3];
      double* cn = S.wz[(j + 1) % 3];
#define WB(row, colp, colidx) ((row) < (colidx) ? (colp)[row] : 0.0)
      double sumF = 0.0;
      for (int i = 0; i < r0; ++i) sumF += cj[i] * fabs(S.F[i]);
      int tz = 0, tx = 0;
      for (int bb = tid; bb <= j; bb += nt) {
        double v;
        if (bb < r0)
          v = WB(bb, cj, j) * (fabs(S.theta_keep[bb]) + nXj) + WB(r0, cj, j) * fabs(S.F[bb]) +
              WB(bb, cjm1, j - 1) * nGjm1 + ud2;
        else if (bb == r0)
          v = WB(bb, cj, j) * (fabs(S.alpha[bb]) + nXj) + sumF + WB(bb + 1, cj, j) * S.beta[bb] +
              WB(bb, cjm1, j - 1) * nGjm1 + ud2;
        else
          v = WB(bb, cj, j) * (fabs(S.alpha[bb]) + nXj) + WB(bb + 1, cj, j) * S.beta[bb] +
              WB(bb - 1, cj, j) * S.beta[bb - 1] + WB(bb, cjm1, j - 1) * nGjm1 + ud2;
        cn[bb] = g * v;
        if (!(g * v <= u_ro)) tz = 1;
      }
#undef WB
      double* xj = S.wx[j % 3];
      double* xjm1 = S.wx[(j + 2) % 3];
      double* xn = S.wx[(j + 1) % 3];
      for (int k = tid; k < nlock; k += nt) {
        const double v = g * (xj[k] * (S.xth[k] + nXj) + S.xrho[k] + xjm1[k] * nGjm1 + ud2);
        xn[k] = v;
        if (!(v <= u_ro)) tx = 1;
      }
      if (tz) atomicOr(&S.flags, 1);
      if (tx) atomicOr(&S.flags, 2);
      __syncthreads();
      const int fl = S.flags;
      if (fl) {  // one CGS pass of Q_j and Q_{j+1} against [X, Z_{j-1}] (semi-orthogonal blocks)
        PHASE(0);
        const int kx = (fl & 2) ? nlock : 0, kz = (fl & 1) ? j : 0;
        cta_cgs_n<2>(qj, qn, X, kx, Z, kz, n, S.coef);
        double nr = cta_norm(qj, n, cr);
        cta_scale_to(qj, qj, (float)(1.0 / nr), n);
        nr = cta_norm(qn, n, cr);
        cta_scale_to(qn, qn, (float)(1.0 / nr), n);
        if (fl & 1)
          for (int t = tid; t <= j; t += nt) {
            if (t < j) cj[t] = u_d;
            cn[t] = u_d;
          }
        if (fl & 2)
          for (int k = tid; k < nlock; k += nt) xj[k] = xn[k] = u_d;
        ++reorths;
        __syncthreads();
        PHASE(1);
      }
    }
    // ---- restart (Alg. 2 (the thick restart)) with locking ----
    PHASE(0);
    for (int t = tid; t < R * R; t += nt) {
      const int r = t / R, c = t % R;
      double v = 0.0;
      if (r == c) v = (r < r0) ? S.theta_keep[r] : S.alpha[r];
      else if (r < r0 && c == r0) v = S.F[r];
      else if (c < r0 && r == r0) v = S.F[c];
      else if (r >= r0 && c >= r0 && (r == c + 1 || c == r + 1)) v = S.beta[r < c ? r : c];
      As[t] = v;
    }
    __syncthreads();
    for (int r = tid; r < R; r += nt) S.tdiag[r] = (r < r0) ? S.theta_keep[r] : S.alpha[r];
    __syncthreads();
    const int2 sw = cta_eig(As, Vs, Wt, S.th, R, r0, S.tdiag, S.F, S.beta, js, cr);
    sweeps32 += sw.x;
    sweeps64 += sw.y;
    PHASE(2);
    for (int c = tid; c < R; c += nt) S.res[c] = S.beta[R - 1] * fabs(Vs[(R - 1) * R + c]);
    __syncthreads();
    theta_max = fmax(theta_max, S.th[R - 1]);
    if (tid == 0) {
      int nsm = 0, nc = 0;
      for (int c = 0; c < R; ++c)
        if (S.th[c] < 3.0 * a.eps) {
          ++nsm;
          if (S.res[c] <= tol_eff * normB) S.lock_list[nc++] = c;
        }
      S.nsmall = nsm;
      S.ncand = nc;
    }
    __syncthreads();
    const int ncand = S.ncand;
    float* V32 = reinterpret_cast<float*>(As);  // FP32 copy of the eigenvectors (As is free now)
    for (int t = tid; t < R * R; t += nt) V32[t] = (float)Vs[t];
    __syncthreads();
    int locked_now = 0;
    for (int ci = 0; ci < ncand; ++ci) {
      if (nlock >= kBMaxLock) {
        status = 8;  // more null vectors than the per-instance capacity
        break;
      }
      const int c = S.lock_list[ci];
      for (int i = tid; i < n; i += nt) {
        float sm = 0.f;
        for (int jj = 0; jj < R; ++jj) sm = fmaf(Z[(int64_t)jj * n + i], V32[jj * R + c], sm);
        Zt[i] = sm;
      }
      __syncthreads();
      const double n0 = cta_norm(Zt, n, cr);
      cta_cgs(Zt, X, nlock, Z, 0, n, S.coef, cr);
      cta_cgs(Zt, X, nlock, Z, 0, n, S.coef, cr);
      const double n1 = cta_norm(Zt, n, cr);
      if (!(n1 >= 0.5 * n0)) continue;  // a copy of a locked vector (ghost)
      cta_scale_to(Zt, X + (int64_t)nlock * n, (float)(1.0 / n1), n);
      if (tid == 0) {
        S.xth[nlock] = S.th[c];
        S.xrho[nlock] = S.res[c];
      }
      ++nlock;
      ++locked_now;
    }
    if (locked_now) {
      if (ev_first < 0) {
        ev_first = matvecs;
        ev_first_k = locked_now;
      }
      ev_last = matvecs;
      ev_total += locked_now;
      ++ev_count;
    }
    const int n_unl = S.nsmall - ncand;
    PHASE(3);
    if (tid == 0) {  // retained set (reading R7b), most converged small pairs first
      int nk = (n_unl + R) / 2;
      nk = max(nk, 1);
      nk = min(nk, R - 2);
      {  // reading R7b: the unlocked small pairs when they fit in 3R/4, else R/2
        const int cap = (n_unl > R / 2 && n_unl <= 3 * R / 4) ? n_unl : R / 2;
        nk = min(nk, max(1, cap));
      }
      int cnt = 0;
      // small, not candidates, by residual
      for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < R && cnt < R; ++c) {
          bool cand = false;
          for (int ci = 0; ci < ncand; ++ci) cand |= (S.lock_list[ci] == c);
          if (cand) continue;
          const bool sm = S.th[c] < 3.0 * a.eps;
          if ((pass == 0) != sm) continue;
          S.keep_list[cnt++] = c;
        }
        if (pass == 0) {  // insertion sort of the small ones by residual
          for (int x = 1; x < cnt; ++x) {
            const int key = S.keep_list[x];
            int y = x - 1;
            while (y >= 0 && S.res[S.keep_list[y]] > S.res[key]) {
              S.keep_list[y + 1] = S.keep_list[y];
              --y;
            }
            S.keep_list[y + 1] = key;
          }
        }
      }
      S.nkeep = min(nk, cnt);
    }
    __syncthreads();
    const int nk = S.nkeep;
    for (int i = tid; i < n; i += nt) {  // Z_new = Z V(:, keep), eight kept columns per pass over row i
      for (int c0 = 0; c0 < nk; c0 += 8) {
        float acc[8];
        int kc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          acc[c] = 0.f;
          kc[c] = S.keep_list[min(c0 + c, nk - 1)];
        }
        for (int jj = 0; jj < R; ++jj) {
          const float z = Z[(int64_t)jj * n + i];
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[c] = fmaf(z, V32[jj * R + kc[c]], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c0 + c < nk) Zt[(int64_t)(c0 + c) * n + i] = acc[c];
      }
      for (int c = 0; c < nk; ++c) Z[(int64_t)c * n + i] = Zt[(int64_t)c * n + i];
    }
    __syncthreads();
    {  // Q_{l+1} against [X, Z_new] -> block nk (Alg. 2 (the re-orthogonalized next block))
      float* ql = Z + (int64_t)R * n;
      cta_cgs(ql, X, nlock, Z, nk, n, S.coef, cr);
      cta_cgs(ql, X, nlock, Z, nk, n, S.coef, cr);
      double rho = cta_norm(ql, n, cr);
      float* qk = Z + (int64_t)nk * n;
      if (rho <= bd_tol) {
        replace_vec(qk, seed, 2u + bdcount++, n, X, nlock, Z, nk, S, cr);
        rho = 0.0;
      } else {
        cta_scale_to(ql, qk, (float)(1.0 / rho), n);
      }
      for (int c = tid; c < nk; c += nt) {
        const int kc = S.keep_list[c];
        S.F[c] = rho * S.beta[R - 1] * Vs[(R - 1) * R + kc];
        S.theta_keep[c] = S.th[kc];
      }
      __syncthreads();
    }
    k0 = nk;
    PHASE(4);
    ++restarts;
    // stopping rule (Sec. 4.3)
    double sv = (double)R;
    if (ev_count >= 2) sv = (double)(ev_last - ev_first) / fmax(1.0, (double)(ev_total - ev_first_k));
    sv = fmax(sv, (double)R);
    const long long since = matvecs - (ev_last >= 0 ? ev_last : 0);
    if (status) break;
    // before the first lock: also wait for the smallest Ritz value to converge at or
    // above 3 eps (the direct test of Sec. 4.3)
    const bool settled = ev_count > 0 || (S.th[0] >= 3.0 * a.eps && S.res[0] <= tol_eff * normB);
    if (n_unl == 0 && locked_now == 0 && (double)since > a.stop_factor * sv && settled) break;
    if (matvecs >= max_mv) {
      status = 4;
      break;
    }
  }
  // ---- FP64 projection of every locked vector onto null(A), then MGS twice ----
  PHASE(4);
  double* out = a.basis + a.out_off[inst];
  double* r = ws64;
  double* p = r + n;
  double* Ap = p + n;
  const double tol2 = (a.refine_tol * theta_max) * (a.refine_tol * theta_max);
  long long iters_max = 0;
  for (int k = 0; k < nlock; ++k) {
    double* z = out + (int64_t)k * n;  // CG on A z = 0 from z = x keeps the null component of x
    for (int i = tid; i < n; i += nt) z[i] = (double)X[(int64_t)k * n + i];
    __syncthreads();
    cta_spmv64(rp, col, val64, n, z, Ap);
    double loc = 0.0;
    for (int i = tid; i < n; i += nt) {
      r[i] = -Ap[i];
      p[i] = r[i];
      loc += r[i] * r[i];
    }
    double rr = cta_sum(loc, cr);
    int it = 0;
    for (; it < a.refine_maxit && rr > tol2; ++it) {
      cta_spmv64(rp, col, val64, n, p, Ap);
      double l2 = 0.0;
      for (int i = tid; i < n; i += nt) l2 += p[i] * Ap[i];
      const double pAp = cta_sum(l2, cr);
      if (!(pAp > 0.0)) break;
      const double alpha = rr / pAp;
      double l3 = 0.0;
      for (int i = tid; i < n; i += nt) {
        z[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
        l3 += r[i] * r[i];
      }
      const double rn = cta_sum(l3, cr);
      const double beta = rn / rr;
      for (int i = tid; i < n; i += nt) p[i] = r[i] + beta * p[i];
      rr = rn;
      __syncthreads();
    }
    iters_max = max(iters_max, (long long)it);
    if (rr > tol2 && status == 0) status = 7;
  }
  for (int k = 0; k < nlock; ++k) {
    double* zk = out + (int64_t)k * n;
    for (int pass = 0; pass < 2; ++pass)
      for (int jj = 0; jj < k; ++jj) {
        const double* zj = out + (int64_t)jj * n;
        double loc = 0.0;
        for (int i = tid; i < n; i += nt) loc += zj[i] * zk[i];
        const double c = cta_sum(loc, cr);
        for (int i = tid; i < n; i += nt) zk[i] -= c * zj[i];
        __syncthreads();
      }
    double loc = 0.0;
    for (int i = tid; i < n; i += nt) loc += zk[i] * zk[i];
    const double nr = sqrt(cta_sum(loc, cr));
    for (int i = tid; i < n; i += nt) zk[i] /= nr;
    __syncthreads();
  }
  if (tid == 0) {
    a.nullity[inst] = nlock;
    a.status[inst] = status;
    long long* st = a.istats + kBStats * (int64_t)inst;
    st[0] = matvecs;
    st[1] = restarts;
    st[2] = reorths;
    st[3] = iters_max;
    st[4] = clock64() - clk0;
    PHASE(5);
    for (int k = 0; k < 6; ++k) st[5 + k] = cyc[k];
    st[11] = sweeps32;
    st[12] = sweeps64;
  }
  __syncthreads();
#undef PHASE
}

template <int LANES, int BT>
__global__ void __launch_bounds__(BT, BT <= 128 ? 4 : 2) k_batched(BatchArgs a) {
  extern __shared__ __align__(16) double dyn[];
  __shared__ BState S;
  __shared__ JacobiScratch js;
  __shared__ CtaRed cr;
  __shared__ int next;
  double* As = dyn;
  double* Vs = dyn + a.R * a.R;
  double* Wt = Vs + a.R * a.R;
  float* ws32 = a.ws32 + (int64_t)blockIdx.x * a.ws32_stride;
  double* ws64 = a.ws64 + (int64_t)blockIdx.x * a.ws64_stride;
  while (true) {  // work queue: no CTA waits for another
    if (threadIdx.x == 0) next = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int k = next;
    __syncthreads();
    if (k >= a.count) break;
    solve_instance<LANES>(a, a.order[k], ws32, ws64, As, Vs, Wt, S, js, cr);
  }
}

template <int L, int BT>
static const void* kfun() {
  return reinterpret_cast<const void*>(k_batched<L, BT>);
}

static const void* batched_fn(int lanes, int block) {
  if (block == 128) return lanes == 1 ? kfun<1, 128>() : lanes == 2 ? kfun<2, 128>() : kfun<4, 128>();
  return lanes == 1 ? kfun<1, 256>() : lanes == 2 ? kfun<2, 256>() : kfun<4, 256>();
}

cudaError_t batched_prepare(int lanes, int block, int R, int* blocks_per_sm) {
  const int smem = (int)(sizeof(double) * 3 * (size_t)R * R);
  const void* f = batched_fn(lanes, block);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * kBMaxR * kBMaxR * 8);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, block, smem);
}

void batched_launch(const BatchArgs& a, int lanes, int block, int grid, cudaStream_t s) {
  const size_t smem = sizeof(double) * 3 * (size_t)a.R * a.R;
  if (block == 128) {
    switch (lanes) {
      case 1: k_batched<1, 128><<<grid, 128, smem, s>>>(a); break;
      case 2: k_batched<2, 128><<<grid, 128, smem, s>>>(a); break;
      default: k_batched<4, 128><<<grid, 128, smem, s>>>(a); break;
    }
  } else {
    switch (lanes) {
      case 1: k_batched<1, 256><<<grid, 256, smem, s>>>(a); break;
      case 2: k_batched<2, 256><<<grid, 256, smem, s>>>(a); break;
      default: k_batched<4, 256><<<grid, 256, smem, s>>>(a); break;
    }
  }
}

// ---------------------------------------------------------------------------
// ingest and output helpers of the batched form (one CTA per instance)
// ---------------------------------------------------------------------------
// every entry: column inside the instance, finite value (bit 2: column, bit 4: value)
__global__ void k_batch_validate(const int64_t* __restrict__ rowptr, const int64_t* __restrict__ rp_off,
                                 const int64_t* __restrict__ nz_off, const int* __restrict__ nrows,
                                 const int* __restrict__ col, const double* __restrict__ val, int count,
                                 unsigned* err) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const int n = nrows[i];
    const int64_t* rp = rowptr + rp_off[i];
    const int64_t e0 = rp[0], e1 = rp[n];
    const int* c = col + nz_off[i];
    const double* v = val + nz_off[i];
    unsigned bad = 0;
    for (int64_t k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
      const int cc = c[k];
      if (cc < 0 || cc >= n) bad |= 2u;
      if (!isfinite(v[k])) bad |= 4u;
    }
    if (bad) atomicOr(err, bad);
  }
}

// instance i's first N_i basis columns (n_i x N_i, column-major, contiguous at
// basis + out_off[i]) to packed + poff[i]
__global__ void k_batch_pack(const double* __restrict__ basis, const int64_t* __restrict__ out_off,
                             const int64_t* __restrict__ poff, const int64_t* __restrict__ plen, int count,
                             double* __restrict__ packed) {
  for (int i = blockIdx.x; i < count; i += gridDim.x) {
    const double* src = basis + out_off[i];
    double* dst = packed + poff[i];
    for (int64_t k = threadIdx.x; k < plen[i]; k += blockDim.x) dst[k] = src[k];
  }
}

void batch_validate(const BatchArgs& a, unsigned* err, cudaStream_t s) {
  k_batch_validate<<<std::min(a.count, 152 * 16), 256, 0, s>>>(a.rowptr, a.rp_off, a.nz_off, a.nrows, a.col,
                                                               a.val64, a.count, err);
}

void batch_pack(const double* basis, const int64_t* out_off, const int64_t* poff, const int64_t* plen, int count,
                double* packed, cudaStream_t s) {
  k_batch_pack<<<std::min(count, 152 * 16), 256, 0, s>>>(basis, out_off, poff, plen, count, packed);
}

size_t batched_ws32_per_slot(int nmax, int R) { return (size_t)nmax * (2 * R + 1 + kBMaxLock + 2) + 64; }
size_t batched_ws64_per_slot(int nmax) { return (size_t)nmax * 3 + 64; }

}  // namespace ns

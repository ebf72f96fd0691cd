// Symmetric eigensolver for the projected matrix T of Alg. 2 (the projected matrix T) (ascending
// eigenvalues, orthonormal eigenvectors), FP64.
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so a serial
// algorithm (a QR bulge chase, a one-SM Jacobi) is slow no matter how it is
// tuned.  The stages here therefore spread the FP64 work over many SMs:
//   1. Householder reduction T = Q Tri Q^T       (one CTA, matrix in shared memory)
//   2. eigenvalue i of Tri by Sturm-count multisection (one block per eigenvalue;
//      128 shifts per round, division-free determinant recurrence)
//   3. eigenvector of Tri by inverse iteration with a pivoted tridiagonal LU
//      (one block per eigenvector)
//   4. CGS2 inside clusters of close eigenvalues (gap < 1e-3 ||T||), which
//      restores orthogonality where inverse iteration cannot resolve directions
//   5. back-transformation by the Householder reflectors (one block per column).
#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace ns {

constexpr int kEigSmemMaxN = 160;  // tridiagonalization keeps T in shared memory up to this size
constexpr int kBisThreads = 128;   // shifts evaluated per multisection round
constexpr int kBisRounds = 8;      // 129^8 > 1e16 relative narrowing

// work layout (doubles): Hv n*n | a n | e n | e2 n | tau n | W n*n | misc 64
size_t syev_work_doubles(int n) { return 2 * (size_t)n * n + 4 * (size_t)n + 64; }

struct EigWork {
  double *Hv, *a, *e, *e2, *tau, *W, *misc;  // misc: [0] lo, [1] hi, [2] normT, [3] status
  __host__ __device__ EigWork(double* w, int n) {
    Hv = w;
    a = Hv + (size_t)n * n;
    e = a + n;
    e2 = e + n;
    tau = e2 + n;
    W = tau + n;
    misc = W + (size_t)n * n;
  }
};

__device__ inline double dsign(double a, double b) { return b >= 0.0 ? fabs(a) : -fabs(a); }

__device__ double block_sum_d(double v, double* red, double* out1) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out1 = s;
  }
  __syncthreads();
  const double r = *out1;
  __syncthreads();
  return r;
}

// ---- 1. Householder tridiagonalization -------------------------------------
__global__ void __launch_bounds__(kThreads) k_tridiag(const double* __restrict__ T, int n, double* work) {
  extern __shared__ __align__(16) double As[];
  __shared__ double red[kThreads / 32];
  __shared__ double one;
  __shared__ double pv[512];
  EigWork w(work, n);
  double* A = (n <= kEigSmemMaxN) ? As : w.Hv;  // column-major n x n
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < n * n; t += nt) {
    const int i = t % n, j = t / n;
    A[t] = (i >= j) ? T[(size_t)j * n + i] : T[(size_t)i * n + j];
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = A + (size_t)k * n + (k + 1);
    double loc = 0.0;
    for (int i = tid + 1; i < m; i += nt) loc += x[i] * x[i];
    const double tail = block_sum_d(loc, red, &one);
    const double x0 = x[0];
    if (tail == 0.0) {
      if (tid == 0) {
        w.tau[k] = 0.0;
        w.e[k] = x0;
      }
      __syncthreads();
      continue;
    }
    const double alpha = -dsign(sqrt(tail + x0 * x0), x0);
    const double v0 = x0 - alpha;
    const double tk = 2.0 / (tail + v0 * v0);
    __syncthreads();
    if (tid == 0) {
      x[0] = v0;
      w.tau[k] = tk;
      w.e[k] = alpha;
    }
    __syncthreads();
    double lk = 0.0;
    for (int i = tid; i < m; i += nt) {  // p = tau S v
      double s = 0.0;
      for (int j = 0; j < m; ++j) s = fma(A[(size_t)(k + 1 + j) * n + (k + 1 + i)], x[j], s);
      pv[i] = tk * s;
      lk += x[i] * pv[i];
    }
    const double K = 0.5 * tk * block_sum_d(lk, red, &one);
    for (int i = tid; i < m; i += nt) pv[i] -= K * x[i];  // w = p - K v
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
      const int i = t % m, j = t / m;
      if (j <= i) {  // lower triangle of the symmetric trailing block
        const double nv = A[(size_t)(k + 1 + j) * n + (k + 1 + i)] - (x[i] * pv[j] + pv[i] * x[j]);
        A[(size_t)(k + 1 + j) * n + (k + 1 + i)] = nv;
        A[(size_t)(k + 1 + i) * n + (k + 1 + j)] = nv;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) w.a[i] = A[(size_t)i * n + i];
  if (tid == 0) {
    if (n >= 2) w.e[n - 2] = A[(size_t)(n - 2) * n + (n - 1)];
    w.e[n - 1] = 0.0;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) w.e2[i] = w.e[i] * w.e[i];
  if (A == As)
    for (int t = tid; t < n * n; t += nt) w.Hv[t] = As[t];  // reflectors for stage 5
  __syncthreads();
  if (tid == 0) {  // Gershgorin interval of Tri
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? fabs(w.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(w.e[i]) : 0.0);
      lo = fmin(lo, w.a[i] - r);
      hi = fmax(hi, w.a[i] + r);
    }
    const double nt2 = fmax(fabs(lo), fabs(hi));
    w.misc[0] = lo - 1e-14 * nt2 - 1e-300;
    w.misc[1] = hi + 1e-14 * nt2 + 1e-300;
    w.misc[2] = nt2;
  }
}

// number of eigenvalues of Tri below x: sign changes of the leading principal
// minors P_0 = 1, P_1 = a_0 - x, P_{k+1} = (a_k - x) P_k - e_{k-1}^2 P_{k-1}
__device__ inline int sturm_count(const double* a, const double* e2, int n, double x) {
  double pm = 1.0, p = a[0] - x;
  int cnt = (__double2hiint(p) < 0);
  bool neg = cnt != 0;
  for (int k = 1; k < n; ++k) {
    const double pn = fma(a[k] - x, p, -e2[k - 1] * pm);
    const bool ng = __double2hiint(pn) < 0;
    cnt += (ng != neg);
    neg = ng;
    pm = p;
    p = pn;
    if ((k & 15) == 0) {  // keep the minors in range
      const double s = fabs(p) + fabs(pm);
      if (s > 1e150) {
        p *= 1e-150;
        pm *= 1e-150;
      } else if (s < 1e-150 && s > 0.0) {
        p *= 1e150;
        pm *= 1e150;
      }
    }
  }
  return cnt;
}

// ---- 2. eigenvalue i by multisection ----------------------------------------
__global__ void __launch_bounds__(kBisThreads) k_bisect(const double* work_c, int n, double* theta) {
  EigWork w(const_cast<double*>(work_c), n);
  __shared__ double as[512], e2s[512];
  __shared__ int cnt_s[kBisThreads];
  __shared__ double lohi[2];
  const int i = blockIdx.x, t = threadIdx.x;
  for (int k = t; k < n; k += blockDim.x) {
    as[k] = w.a[k];
    e2s[k] = w.e2[k];
  }
  if (t == 0) {
    lohi[0] = w.misc[0];
    lohi[1] = w.misc[1];
  }
  __syncthreads();
  for (int round = 0; round < kBisRounds; ++round) {
    const double lo = lohi[0], hi = lohi[1];
    const double x = lo + (hi - lo) * (double)(t + 1) / (double)(kBisThreads + 1);
    cnt_s[t] = sturm_count(as, e2s, n, x);
    __syncthreads();
    if (t == 0) {
      int j = 0;
      while (j < kBisThreads && cnt_s[j] <= i) ++j;  // first shift with more than i eigenvalues below
      const double h = (hi - lo) / (double)(kBisThreads + 1);
      lohi[0] = lo + h * (double)j;
      lohi[1] = (j < kBisThreads) ? lo + h * (double)(j + 1) : hi;
    }
    __syncthreads();
  }
  if (t == 0) theta[i] = 0.5 * (lohi[0] + lohi[1]);
}

// ---- 3. inverse iteration for eigenvector i ---------------------------------
__global__ void __launch_bounds__(32) k_inviter(double* work, int n, const double* theta) {
  EigWork w(work, n);
  __shared__ double u0[512], u1[512], u2[512], lm[512], x[512];
  __shared__ unsigned char sw[512];
  __shared__ double red[1], one[1];
  const int i = blockIdx.x, lane = threadIdx.x;
  const double th = theta[i];
  const double tiny = 0x1.0p-52 * fmax(w.misc[2], 1e-300);
  if (lane == 0) {  // LU of Tri - th I with partial pivoting (U has two superdiagonals)
    double d = w.a[0] - th, f1 = (n > 1) ? w.e[0] : 0.0, f2 = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
      const double ek = w.e[k], c1 = w.a[k + 1] - th, e1 = (k + 2 < n) ? w.e[k + 1] : 0.0;
      if (fabs(d) >= fabs(ek)) {
        if (d == 0.0) d = tiny;
        const double l = ek / d;
        u0[k] = d;
        u1[k] = f1;
        u2[k] = f2;
        lm[k] = l;
        sw[k] = 0;
        d = c1 - l * f1;
        f1 = e1 - l * f2;
        f2 = 0.0;
      } else {
        const double l = d / ek;
        u0[k] = ek;
        u1[k] = c1;
        u2[k] = e1;
        lm[k] = l;
        sw[k] = 1;
        const double nd = f1 - l * c1, nf1 = f2 - l * e1;
        d = nd;
        f1 = nf1;
        f2 = 0.0;
      }
    }
    if (fabs(d) < tiny) d = (d < 0.0) ? -tiny : tiny;
    u0[n - 1] = d;
    for (int k = 0; k < n; ++k) u0[k] = 1.0 / (fabs(u0[k]) < tiny ? dsign(tiny, u0[k]) : u0[k]);  // reciprocals
  }
  // deterministic start vector with all components nonzero
  for (int k = lane; k < n; k += 32) x[k] = 1.0 + 0.37 * (double)((k * 2654435761u + i * 40503u) % 1000u) / 1000.0;
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (lane == 0) {
      for (int k = 0; k + 1 < n; ++k) {  // forward: row swaps and eliminations
        if (sw[k]) {
          const double tmp = x[k];
          x[k] = x[k + 1];
          x[k + 1] = tmp;
        }
        x[k + 1] -= lm[k] * x[k];
      }
      for (int k = n - 1; k >= 0; --k) {  // back substitution
        double s = x[k];
        if (k + 1 < n) s -= u1[k] * x[k + 1];
        if (k + 2 < n) s -= u2[k] * x[k + 2];
        x[k] = s * u0[k];
      }
    }
    __syncwarp();
    double loc = 0.0;
    for (int k = lane; k < n; k += 32) loc += x[k] * x[k];
    loc = warp_sum(loc);
    const double inv = 1.0 / sqrt(loc);
    for (int k = lane; k < n; k += 32) x[k] *= inv;
    __syncwarp();
  }
  for (int k = lane; k < n; k += 32) w.W[(size_t)i * n + k] = x[k];
  (void)red;
  (void)one;
}

// ---- 4. CGS2 inside clusters -------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_cluster_orth(double* work, int n, const double* theta) {
  EigWork w(work, n);
  __shared__ double red[kThreads / 32];
  __shared__ double one;
  __shared__ double cf[512];
  const int s = blockIdx.x;
  const double gtol = 1e-3 * w.misc[2];
  if (s > 0 && theta[s] - theta[s - 1] <= gtol) return;  // not the start of a cluster
  int e = s + 1;
  while (e < n && theta[e] - theta[e - 1] <= gtol) ++e;
  if (e - s < 2) return;
  for (int j = s + 1; j < e; ++j) {
    double* xj = w.W + (size_t)j * n;
    for (int pass = 0; pass < 2; ++pass) {
      // coefficients against all earlier cluster members (one warp per coefficient)
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int k = s + warp; k < j; k += nw) {
        const double* xk = w.W + (size_t)k * n;
        double d = 0.0;
        for (int r = lane; r < n; r += 32) d += xk[r] * xj[r];
        d = warp_sum(d);
        if (lane == 0) cf[k - s] = d;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double v = xj[r];
        for (int k = s; k < j; ++k) v -= cf[k - s] * w.W[(size_t)k * n + r];
        xj[r] = v;
      }
      __syncthreads();
    }
    double loc = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) loc += xj[r] * xj[r];
    const double nrm = sqrt(block_sum_d(loc, red, &one));
    for (int r = threadIdx.x; r < n; r += blockDim.x) xj[r] /= nrm;
    __syncthreads();
  }
}

// ---- 5. back-transformation V = Q W ------------------------------------------
__global__ void __launch_bounds__(128) k_backtransform(const double* work_c, int n, double* V) {
  EigWork w(const_cast<double*>(work_c), n);
  __shared__ double x[512];
  __shared__ double red[4];
  __shared__ double one;
  const int j = blockIdx.x;
  for (int r = threadIdx.x; r < n; r += blockDim.x) x[r] = w.W[(size_t)j * n + r];
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const double tk = w.tau[k];
    if (tk == 0.0) continue;  // uniform
    const double* v = w.Hv + (size_t)k * n + (k + 1);
    double loc = 0.0;
    for (int r = threadIdx.x; r < n - k - 1; r += blockDim.x) loc += v[r] * x[k + 1 + r];
    const double dot = block_sum_d(loc, red, &one);
    for (int r = threadIdx.x; r < n - k - 1; r += blockDim.x) x[k + 1 + r] -= tk * dot * v[r];
    __syncthreads();
  }
  for (int r = threadIdx.x; r < n; r += blockDim.x) V[(size_t)j * n + r] = x[r];
}

void syev(const double* T, int n, double* theta, double* V, double* work, cudaStream_t s) {
  const size_t smem = (n <= kEigSmemMaxN) ? sizeof(double) * (size_t)n * n : 0;
  if (ensure_smem_limit(reinterpret_cast<const void*>(k_tridiag), smem) != cudaSuccess) return;  // launch fails; caller checks
  k_tridiag<<<1, kThreads, smem, s>>>(T, n, work);
  k_bisect<<<n, kBisThreads, 0, s>>>(work, n, theta);
  k_inviter<<<n, 32, 0, s>>>(work, n, theta);
  k_cluster_orth<<<n, kThreads, 0, s>>>(work, n, theta);
  k_backtransform<<<n, 128, 0, s>>>(work, n, V);
}

}  // namespace ns

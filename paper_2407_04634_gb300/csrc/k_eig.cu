// Symmetric eigensolver for the projected matrix T of Alg. 2 line 13 (ascending
// eigenvalues and orthonormal eigenvectors), one CTA, FP64:
//   1. Householder reduction to tridiagonal form  T = Q Tri Q^T,
//   2. explicit accumulation of Q,
//   3. implicit symmetric QR steps with the Wilkinson shift on Tri (bulge chasing
//      with Givens rotations), rotations accumulated into Q,
//   4. sort ascending.
// The rotations of one QR step are computed by one thread and applied by all
// threads to their own rows of Q (rows are independent), so each step costs two
// block barriers.
#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace ns {

size_t syev_work_doubles(int k) { return (size_t)k * k + 8 * (size_t)k + 64; }

__device__ inline double dsign(double a, double b) { return b >= 0.0 ? fabs(a) : -fabs(a); }

__global__ void __launch_bounds__(kThreads) k_syev(const double* __restrict__ T, int n, double* theta, double* V,
                                                   double* work, int* status) {
  double* A = work;                   // n x n column-major, Householder vectors below the diagonal
  double* a = A + (size_t)n * n;      // diagonal
  double* e = a + n;                  // sub-diagonal (e[i] couples i and i+1)
  double* tau = e + n;                // reflector scalars
  double* p = tau + n;                // scratch vectors
  double* cs = p + n;                 // rotations (c, s) of one QR step: 2n
  int* perm = reinterpret_cast<int*>(cs + 2 * n);  // n ints (fits in 2n doubles of slack)
  __shared__ double red_s[kThreads / 32];
  __shared__ double sh[4];
  __shared__ int win[3];  // p, q, done
  const int tid = threadIdx.x, nt = blockDim.x;

  // symmetric copy from the lower triangle
  for (int t = tid; t < n * n; t += nt) {
    const int i = t % n, j = t / n;
    A[t] = (i >= j) ? T[(size_t)j * n + i] : T[(size_t)i * n + j];
  }
  __syncthreads();

  auto block_sum1 = [&](double v) -> double {
    v = warp_sum(v);
    if ((tid & 31) == 0) red_s[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) s += red_s[w];
      sh[3] = s;
    }
    __syncthreads();
    const double r = sh[3];
    __syncthreads();
    return r;
  };

  // ---- 1. Householder tridiagonalization ----
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = A + (size_t)k * n + (k + 1);  // column k below the diagonal
    double loc = 0.0, loc_tail = 0.0;
    for (int i = tid; i < m; i += nt) {
      loc += x[i] * x[i];
      if (i > 0) loc_tail += x[i] * x[i];
    }
    const double ss = block_sum1(loc);
    const double tail = block_sum1(loc_tail);
    const double x0 = x[0];
    if (tail == 0.0) {  // already reduced in this column
      if (tid == 0) {
        tau[k] = 0.0;
        e[k] = x0;
      }
      __syncthreads();
      continue;
    }
    const double alpha = -dsign(sqrt(ss), x0);
    const double v0 = x0 - alpha;
    const double tk = 2.0 / (tail + v0 * v0);
    __syncthreads();
    if (tid == 0) {
      x[0] = v0;  // x now holds v
      tau[k] = tk;
      e[k] = alpha;
    }
    __syncthreads();
    // p = tau S v with S = A[k+1:, k+1:]
    double lk = 0.0;
    for (int i = tid; i < m; i += nt) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += A[(size_t)(k + 1 + j) * n + (k + 1 + i)] * x[j];
      p[i] = tk * s;
      lk += x[i] * p[i];
    }
    const double K = 0.5 * tk * block_sum1(lk);
    for (int i = tid; i < m; i += nt) p[i] -= K * x[i];  // w = p - K v
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
      const int i = t % m, j = t / m;
      A[(size_t)(k + 1 + j) * n + (k + 1 + i)] -= x[i] * p[j] + p[i] * x[j];
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) a[i] = A[(size_t)i * n + i];
  if (tid == 0 && n >= 2) e[n - 2] = A[(size_t)(n - 2) * n + (n - 1)];
  if (tid == 0) e[n - 1] = 0.0;
  __syncthreads();

  // ---- 2. Q = H_0 H_1 ... H_{n-3} (applied right to left to the identity) ----
  for (int t = tid; t < n * n; t += nt) V[t] = (t % n == t / n) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = n - 3; k >= 0; --k) {
    const double tk = tau[k];
    if (tk == 0.0) continue;  // uniform
    const int m = n - k - 1;
    const double* v = A + (size_t)k * n + (k + 1);
    for (int j = tid; j < m; j += nt) {  // u_j = v^T V[k+1:, k+1+j]
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += v[i] * V[(size_t)(k + 1 + j) * n + (k + 1 + i)];
      p[j] = tk * s;
    }
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
      const int i = t % m, j = t / m;
      V[(size_t)(k + 1 + j) * n + (k + 1 + i)] -= v[i] * p[j];
    }
    __syncthreads();
  }

  // ---- 3. implicit symmetric QR with Wilkinson shift ----
  if (tid == 0) {
    win[0] = 0;
    win[1] = n - 1;
    win[2] = 0;
  }
  __syncthreads();
  int steps = 0;
  const int max_steps = 60 * n + 100;
  while (true) {
    if (tid == 0) {
      int q = win[1];
      bool done = false;
      while (true) {
        for (int i = 0; i < q; ++i) {
          const double scale = fabs(a[i]) + fabs(a[i + 1]);
          if (fabs(e[i]) <= 0x1.0p-53 * scale || fabs(e[i]) < 1e-300) e[i] = 0.0;
        }
        while (q > 0 && e[q - 1] == 0.0) --q;
        if (q == 0) {
          done = true;
          break;
        }
        break;
      }
      win[1] = q;
      win[2] = done ? 1 : 0;
      if (!done) {
        int pp = q - 1;
        while (pp > 0 && e[pp - 1] != 0.0) --pp;
        win[0] = pp;
        // Wilkinson shift from the trailing 2 x 2 block
        const double dlt = 0.5 * (a[q - 1] - a[q]);
        const double b2 = e[q - 1] * e[q - 1];
        const double den = dlt + dsign(hypot(dlt, e[q - 1]), dlt == 0.0 ? 1.0 : dlt);
        const double mu = a[q] - b2 / den;
        double x = a[pp] - mu, z = e[pp], bulge = 0.0;
        for (int k = pp; k < q; ++k) {
          if (k > pp) {
            x = e[k - 1];
            z = bulge;
          }
          const double r = hypot(x, z);
          double c = 1.0, s = 0.0;
          if (r > 0.0) {
            c = x / r;
            s = -z / r;
          }
          if (k > pp) e[k - 1] = r;
          const double ak = a[k], ak1 = a[k + 1], ek = e[k];
          a[k] = c * c * ak - 2.0 * c * s * ek + s * s * ak1;
          a[k + 1] = s * s * ak + 2.0 * c * s * ek + c * c * ak1;
          e[k] = c * s * (ak - ak1) + (c * c - s * s) * ek;
          if (k + 1 < q) {
            bulge = -s * e[k + 1];
            e[k + 1] = c * e[k + 1];
          }
          cs[2 * k] = c;
          cs[2 * k + 1] = s;
        }
      }
    }
    __syncthreads();
    if (win[2]) break;
    const int pp = win[0], q = win[1];
    for (int r = tid; r < n; r += nt) {
      for (int k = pp; k < q; ++k) {
        const double c = cs[2 * k], s = cs[2 * k + 1];
        double* vk = V + (size_t)k * n + r;
        double* vk1 = V + (size_t)(k + 1) * n + r;
        const double x0 = *vk, x1 = *vk1;
        *vk = c * x0 - s * x1;
        *vk1 = s * x0 + c * x1;
      }
    }
    __syncthreads();
    if (++steps > max_steps) {
      if (tid == 0) *status = 1;
      break;
    }
  }
  __syncthreads();

  // ---- 4. sort ascending (stable on ties by index) ----
  if (tid == 0) {
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = 1; i < n; ++i) {
      const int key = perm[i];
      int j = i - 1;
      while (j >= 0 && a[perm[j]] > a[key]) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = key;
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) theta[i] = a[perm[i]];
  // permute columns of V into A (reuse), then copy back
  for (int t = tid; t < n * n; t += nt) {
    const int r = t % n, c = t / n;
    A[t] = V[(size_t)perm[c] * n + r];
  }
  __syncthreads();
  for (int t = tid; t < n * n; t += nt) V[t] = A[t];
}

void syev(const double* T, int k, double* theta, double* V, double* work, cudaStream_t s) {
  int* status = reinterpret_cast<int*>(work + syev_work_doubles(k) - 2);
  cudaMemsetAsync(status, 0, sizeof(int), s);
  k_syev<<<1, kThreads, 0, s>>>(T, k, theta, V, work, status);
}

}  // namespace ns

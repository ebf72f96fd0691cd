// Outer preconditioning of the SPD form (Sec. 4.4.2): B_R = L^-1 A~ L^-T + eps D.
//
// A~ = Pi^T A Pi is A renumbered colour by colour, the colours a Jones-Plassmann
// colouring of A's graph; L is the IC(0) factor of A~ + alpha diag(A~) (zero fill,
// diagonal compensation alpha as in Eq. defichol).  No two vertices of a colour
// are adjacent, so row i of L (columns of lower colours) and row i of L^T (higher
// colours) never reference a row of the same colour: the factorization and the
// two triangular solves run one launch per colour, a thread per row.
#include <cuda_runtime.h>

#include "ns_common.cuh"
#include "ns_kernels.cuh"

namespace ns {

static int rows_grid(int64_t rows) {
  const int64_t b = (rows + kThreads - 1) / kThreads;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

// ---------------------------------------------------------------------------
// Jones-Plassmann round: an uncoloured vertex whose (priority, index) beats every
// uncoloured neighbour takes the smallest colour absent among its coloured
// neighbours.  Colours are read from the previous round (cin) and written to cout
// (a copy of cin): a vertex coloured in this round is never a neighbour of another
// one coloured in this round, but a losing vertex must not see it either.
// ---------------------------------------------------------------------------
__global__ void k_jp_round(const int64_t* __restrict__ rowptr, const int* __restrict__ col, int64_t n,
                           const double* __restrict__ prio, const int* __restrict__ cin, int* __restrict__ cout,
                           unsigned* remaining) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (cin[v] >= 0) continue;
    const double pv = prio[v];
    const int64_t s = rowptr[v], e = rowptr[v + 1];
    bool top = true;
    for (int64_t k = s; k < e && top; ++k) {
      const int u = col[k];
      if (u == v || cin[u] >= 0) continue;
      const double pu = prio[u];
      if (pu > pv || (pu == pv && u > v)) top = false;
    }
    if (!top) {
      atomicAdd(remaining, 1u);
      continue;
    }
    for (int base = 0;; base += 64) {
      unsigned long long used = 0ull;
      for (int64_t k = s; k < e; ++k) {
        const int u = col[k];
        const int c = cin[u];
        if (u != v && c >= base && c < base + 64) used |= 1ull << (c - base);
      }
      if (~used) {
        cout[v] = base + __ffsll((long long)~used) - 1;
        break;
      }
    }
  }
}

void jp_round(const int64_t* rowptr, const int* col, int64_t n, const double* prio, const int* cin, int* cout,
              unsigned* remaining, cudaStream_t s) {
  k_jp_round<<<rows_grid(n), kThreads, 0, s>>>(rowptr, col, n, prio, cin, cout, remaining);
}

// ---------------------------------------------------------------------------
// IC(0), rows r0..r1 of one colour.  Row i of L holds its columns ascending with the
// diagonal last, initialised to the entries of tril(A~) and a_ii (1 + alpha).  Each
// off-diagonal l_ij = (a_ij - sum_k l_ik l_jk) / l_jj, the sum over the columns
// k < j kept in both rows (a merge of the two sorted rows); rows j have lower
// colours and are final.  Then l_ii = sqrt(a_ii (1 + alpha) - sum_j l_ij^2); a
// non-positive pivot sets *fail and stores 1.
// ---------------------------------------------------------------------------
__global__ void k_ic0_rows(const int64_t* __restrict__ rp, const int* __restrict__ col, double* val, int64_t r0,
                           int64_t r1, unsigned* fail) {
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = rp[i], pd = rp[i + 1] - 1;
    for (int64_t p = p0; p < pd; ++p) {
      const int j = col[p];
      double s = val[p];
      int64_t a = p0, b = rp[j];
      const int64_t be = rp[j + 1] - 1;
      while (a < p && b < be) {
        const int ca = col[a], cb = col[b];
        if (ca == cb) {
          s -= val[a] * val[b];
          ++a;
          ++b;
        } else if (ca < cb) {
          ++a;
        } else {
          ++b;
        }
      }
      val[p] = s / val[be];
    }
    double d = val[pd];
    for (int64_t p = p0; p < pd; ++p) d -= val[p] * val[p];
    if (!(d > 0.0)) {
      atomicOr(fail, 1u);
      d = 1.0;
    }
    val[pd] = sqrt(d);
  }
}

void ic0_rows(const int64_t* rp, const int* col, double* val, int64_t r0, int64_t r1, unsigned* fail,
              cudaStream_t s) {
  if (r1 > r0) k_ic0_rows<<<rows_grid(r1 - r0), kThreads, 0, s>>>(rp, col, val, r0, r1, fail);
}

__global__ void k_gather_vals(const double* __restrict__ src, const int64_t* __restrict__ map, double* dst,
                              int64_t count) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[map[t]];
}
void gather_vals(const double* src, const int64_t* map, double* dst, int64_t count, cudaStream_t s) {
  if (count > 0) k_gather_vals<<<rows_grid(count), kThreads, 0, s>>>(src, map, dst, count);
}

// ---------------------------------------------------------------------------
// Triangular solves on an n x D row-major block, rows r0..r1 of one colour.
// Lower: x_i = (b_i - sum_{j<i} l_ij x_j) / l_ii, the diagonal last in the row.
// Upper: x_i = (b_i - sum_{j>i} u_ij x_j) / u_ii, the diagonal first.  The rows
// read (other colours) are final; b may alias x.
// ---------------------------------------------------------------------------
template <typename T, int D, bool LOWER>
__global__ void __launch_bounds__(kThreads) k_trsv_color(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                         const T* __restrict__ val, int64_t r0, int64_t r1,
                                                         const T* b, T* x) {
  for (int64_t i = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[i], e = rp[i + 1];
    const int64_t ps = LOWER ? s : s + 1, pe = LOWER ? e - 1 : e;
    T acc[D];
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = b[i * D + q];
    for (int64_t p = ps; p < pe; ++p) {
      const T l = __ldg(val + p);
      const int64_t j = __ldg(col + p);
#pragma unroll
      for (int q = 0; q < D; ++q) acc[q] = fma(-l, x[j * D + q], acc[q]);
    }
    const T dg = __ldg(val + (LOWER ? e - 1 : s));
#pragma unroll
    for (int q = 0; q < D; ++q) x[i * D + q] = acc[q] / dg;
  }
}

template <typename T, int D>
void trsv_colors(const int64_t* rp, const int* col, const T* val, const int64_t* cstart, int ncolors, bool lower,
                 const T* b, T* x, cudaStream_t s) {
  for (int k = 0; k < ncolors; ++k) {
    const int c = lower ? k : ncolors - 1 - k;
    const int64_t r0 = cstart[c], r1 = cstart[c + 1];
    if (r1 <= r0) continue;
    // the first colour processed reads only b; later ones read x of earlier colours
    if (lower)
      k_trsv_color<T, D, true><<<rows_grid(r1 - r0), kThreads, 0, s>>>(rp, col, val, r0, r1, b, x);
    else
      k_trsv_color<T, D, false><<<rows_grid(r1 - r0), kThreads, 0, s>>>(rp, col, val, r0, r1, b, x);
  }
}

// ---------------------------------------------------------------------------
// Lanczos step epilogue on a product already formed (w = L^-1 A~ L^-T x):
// out = w + eps D x - qprev gprev^T, Xi = sym(x^T out).  The same arithmetic as the
// epilogue of the fused SpMM kernels, without the gather.
// ---------------------------------------------------------------------------
template <typename T, int D>
__global__ void __launch_bounds__(kThreads) k_lanczos_epilogue(const T* __restrict__ w, int64_t n, StepOps<T> op,
                                                               Red red) {
  constexpr int NP = D * D;
  __shared__ double red_s[(kThreads / 32) * NP];
  __shared__ double tot[NP];
  __shared__ T g_s[D * D];
  if (threadIdx.x < D * D) g_s[threadIdx.x] = op.gprev ? (T)op.gprev[threadIdx.x] : T(0);
  __syncthreads();
  const bool has_prev = op.qprev != nullptr;
  T part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = T(0);
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    T xi[D], acc[D];
    load_row<T, D>(op.x + row * D, xi);
    load_row<T, D>(w + row * D, acc);
    const T de = (T)op.eps * __ldg(op.Dv + row);
#pragma unroll
    for (int q = 0; q < D; ++q) acc[q] = fma(de, xi[q], acc[q]);
    if (has_prev) {
      T qp[D];
      load_row<T, D>(op.qprev + row * D, qp);
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

template <typename T, int D>
void lanczos_epilogue(const T* w, int64_t n, const StepOps<T>& op, const Red& red, cudaStream_t s) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  const int grid = (int)(b < kMaxBlocks ? (b > 0 ? b : 1) : kMaxBlocks);
  k_lanczos_epilogue<T, D><<<grid, kThreads, 0, s>>>(w, n, op, red);
}

// rows back to the original numbering: out[perm[i] + c n] = in[i + c n], c < ncols
template <typename T>
__global__ void k_unpermute_cols(const T* __restrict__ in, const int64_t* __restrict__ perm, int64_t n, int ncols,
                                 T* __restrict__ out) {
  const int64_t total = n * (int64_t)ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / n, i = t % n;
    out[perm[i] + c * n] = in[t];
  }
}
void unpermute_cols(const double* in, const int64_t* perm, int64_t n, int ncols, double* out, cudaStream_t s) {
  if (n * (int64_t)ncols > 0) k_unpermute_cols<double><<<rows_grid(n * (int64_t)ncols), kThreads, 0, s>>>(in, perm, n, ncols, out);
}

// columns c0 .. c0 + w of X (n x ., column-major) into an n x w row-major panel
template <typename T>
__global__ void k_cols_to_panel_t(const T* __restrict__ X, int c0, int w, int64_t n, T* __restrict__ P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < w; ++c) P[i * w + c] = X[(int64_t)(c0 + c) * n + i];
}
template <typename T>
void cols_to_panel_t(const T* X, int c0, int w, int64_t n, T* P, cudaStream_t s) {
  if (n > 0) k_cols_to_panel_t<T><<<rows_grid(n), kThreads, 0, s>>>(X, c0, w, n, P);
}

// ---------------------------------------------------------------------------
// Inner preconditioning of the normal form (Sec. 4.4.1) with P_L = diag(A A^T):
// s_i = 1 / ||a_i||_2 per row of A (0 for a zero row), then S A (each entry times
// its row's s) and A^T S (each entry of A^T times the s of its column, which is the
// row of A it came from).
// ---------------------------------------------------------------------------
__global__ void k_row_inv_norms(const int64_t* __restrict__ rowptr, const double* __restrict__ val, int64_t m,
                                double* __restrict__ s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    double q = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) q = fma(val[e], val[e], q);
    s[i] = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  }
}
__global__ void k_scale_rows(const int64_t* __restrict__ rowptr, const double* __restrict__ val, int64_t m,
                             const double* __restrict__ s, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = s[i];
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) out[e] = val[e] * si;
  }
}
__global__ void k_scale_by_col(const int* __restrict__ col, const double* __restrict__ val, int64_t nnz,
                               const double* __restrict__ s, double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = val[e] * s[col[e]];
}
void inner_scaling(const int64_t* rowptr, const double* val, int64_t m, const int* col_t, const double* val_t,
                   int64_t nnz, double* s, double* val_s, double* val_t_s, cudaStream_t st) {
  if (m > 0) {
    k_row_inv_norms<<<rows_grid(m), kThreads, 0, st>>>(rowptr, val, m, s);
    k_scale_rows<<<rows_grid(m), kThreads, 0, st>>>(rowptr, val, m, s, val_s);
  }
  if (nnz > 0) k_scale_by_col<<<rows_grid(nnz), kThreads, 0, st>>>(col_t, val_t, nnz, s, val_t_s);
}

#define NS_INST_PC(T, D)                                                                                           \
  template void trsv_colors<T, D>(const int64_t*, const int*, const T*, const int64_t*, int, bool, const T*, T*, \
                                  cudaStream_t);                                                                 \
  template void lanczos_epilogue<T, D>(const T*, int64_t, const StepOps<T>&, const Red&, cudaStream_t);
NS_INST_PC(double, 1)
NS_INST_PC(double, 2)
NS_INST_PC(double, 4)
NS_INST_PC(double, 8)
NS_INST_PC(float, 1)
NS_INST_PC(float, 2)
NS_INST_PC(float, 4)
NS_INST_PC(float, 8)
#undef NS_INST_PC
template void cols_to_panel_t<double>(const double*, int, int, int64_t, double*, cudaStream_t);
template void cols_to_panel_t<float>(const float*, int, int, int64_t, float*, cudaStream_t);

}  // namespace ns

// Launch wrappers of the null-space library's kernels (host side declarations).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ns {

// CSR matrix resident on the device; V = lanes cooperating on one row (1..32)
template <typename T>
struct Csr {
  const int64_t* rowptr = nullptr;
  const int* col = nullptr;
  const T* val = nullptr;
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int V = 8;  // lanes per row (1..32), kSchedTma (TMA-staged) or kSchedSell (sliced ELLPACK)
  // sliced ELLPACK copy of the same matrix, or null: slices of kSellC consecutive rows,
  // each padded to its longest row and stored column-major (entry j of row
  // kSellC s + l at sptr[s] + j kSellC + l); padding has col 0 and value 0
  const int64_t* sptr = nullptr;
  const int* scol = nullptr;
  const T* sval = nullptr;
};

// Reduction workspace: partial sums and an atomic ticket for the last-block protocol
struct Red {
  double* part = nullptr;  // >= kMaxBlocks * 64 doubles
  unsigned* ticket = nullptr;
};

constexpr int kMaxBlocks = 152 * 8;  // persistent grid cap of reducing kernels
constexpr int kSchedTma = 64;        // SpMM schedule code of the TMA-staged kernel
constexpr int kSchedSell = 128;      // SpMM schedule code of the sliced-ELLPACK kernels
constexpr int kSellC = 32;           // rows per ELLPACK slice: one warp, a row per lane
constexpr int kCsrPad = 16;          // padding entries after col/val (16-byte aligned bulk copies)
// bounded device waits that expired since the last call (clear: reset the count)
unsigned spmm_wait_timeouts(bool clear);

// Lanczos step epilogue operands (all device pointers)
template <typename T>
struct StepOps {
  const T* x = nullptr;       // Q_j (panel n x d)
  const T* Dv = nullptr;      // perturbation diagonal
  double eps = 0.0;
  const T* qprev = nullptr;   // Q_{j-1} or null
  const double* gprev = nullptr;  // Gamma_{j-1} (d x d, row-major) or null
  T* out = nullptr;           // Q'
  double* xi = nullptr;       // Xi_j output (d x d)
  double* xi_norm = nullptr;  // ||Xi_j||_2 output
};

// ---- sparse (k_sparse.cu) ----
int choose_lanes(int64_t nrows, int64_t nnz);
template <typename T, int D>
void spmm_plain(const Csr<T>& M, const T* v, T* y, cudaStream_t s);
// Lanczos fused step: out = M v + eps D x - qprev gprev^T ; Xi = sym(x^T out)
template <typename T, int D>
void spmm_lanczos(const Csr<T>& M, const T* v, const StepOps<T>& op, const Red& red, cudaStream_t s);
// column-wise dots: y = M v, dots[c] = sum_i w_i[c] y_i[c] (w = v if w == null) or
// norms (sq=1): dots[c] = sum_i y_i[c]^2
template <typename T, int D>
void spmm_coldot(const Csr<T>& M, const T* v, T* y, const T* w, int sq, double* dots, const Red& red,
                 cudaStream_t s);

// autotuner: fastest lanes-per-row for y = M v on this matrix (v: ncols x D, y: nrows x D)
template <typename T, int D>
int tune_lanes(Csr<T> M, const T* v, T* y, cudaStream_t s);

// transpose by counting sort; work buffers are caller-provided (device)
struct TransposeWork {
  int* count;        // ncols + 1
  int64_t* cursor;   // ncols
  int64_t* perm;     // nnz
  int* rowof;        // nnz
  int64_t* blocksum; // scan partials (>= 4096)
};
void csr_transpose(const int64_t* rowptr, const int* col, const double* val, int64_t m, int64_t n,
                   int64_t nnz, int64_t* rowptr_t, int* col_t, double* val_t, const TransposeWork& w,
                   cudaStream_t s);
// sliced-ELLPACK copy of a device CSR (nrows rows): slice lengths, offsets (scanned on
// the host), then the padded column-major entries.  Returns the number of entries
// (kSellC times the sum of the slice lengths) through *entries; sptr must hold
// ceil(nrows / kSellC) + 1 int64; scol / sval are filled by sell_fill.
void sell_lengths(const int64_t* rowptr, int64_t nrows, int* slice_len, cudaStream_t s);
void sell_fill(const int64_t* rowptr, const int* col, const double* val, int64_t nrows, const int64_t* sptr,
               int* scol, double* sval, cudaStream_t s);
// validation of a device CSR: err bit 1 rowptr, 2 colind, 4 values
void csr_validate(const int64_t* rowptr, const int* col, const double* val, int64_t m, int64_t n,
                  int64_t nnz, unsigned* err, cudaStream_t s);
// max_i sum_j |a_ij|  (into *out, device double); uses red
void csr_max_abs_row_sum(const int64_t* rowptr, const double* val, int64_t m, double* out, const Red& red,
                         cudaStream_t s);
// max row length (into *out, device int64 via double)
void convert_d2f(const double* a, float* b, int64_t n, cudaStream_t s);
void convert_f2d(const float* a, double* b, int64_t n, cudaStream_t s);

// ---- dense Lanczos kernels (k_dense.cu) ----
// Philox streams
template <typename T>
void rng_uniform(uint64_t seed, uint32_t stream, T* out, int64_t count, cudaStream_t s);
template <typename T>
void rng_gauss(uint64_t seed, uint32_t stream, T* out, int64_t count, cudaStream_t s);

// q'' = q' - x Xi (in place on qp), G = q''^T q'' ; last block: R1 = chol(G) (flag bit 1 on failure)
template <typename T, int D>
void axpy_gram(T* qp, const T* x, const double* Xi, int64_t n, double* R1, unsigned* flags, const Red& red,
               cudaStream_t s);
// out = in R^{-1} (R upper d x d FP64); if R2 != null: G = out^T out, last block R2 = chol(G)
template <typename T, int D>
void scale_gram(const T* in, int64_t ldin, T* out, int64_t ldout, const double* R, int64_t n, double* R2,
                unsigned* flags, const Red& red, cudaStream_t s, int w = D);
// G = W^T W (W panel, leading dim ld, width w<=D) ; last block: R = chol(G), diag saved in gdiag
template <typename T, int D>
void gram_chol(const T* W, int64_t ld, int w, int64_t n, double* R, double* gdiag, unsigned* flags,
               const Red& red, cudaStream_t s);

// projection against V = [X (n x kx, column-major, ld n) | Z (kz columns in panels of width p)]
template <typename T>
struct VParts {
  const T* X = nullptr;
  int kx = 0;
  const T* Z = nullptr;
  int kz = 0;
  int p = 1;
  int df = 0;  // FP64 only: 1 = the products in compensated FP32-pair arithmetic (k_dfproj.cu)
};
// C (K x w, FP64, row-major) = V^T W ; W panel with leading dim ldw; when Wp2 is
// given, columns [W/2, W) of W come from the panel Wp2 (same ldw)
// rows_per_chunk: 0 = 32768 rows per chunk (part needs ceil(n / 32768) K W doubles);
// kDotsAutoChunks = chosen so that the grid fills the GPU, never below
// kDotsMinChunk rows (part needs ceil(n / kDotsMinChunk) K W doubles)
constexpr int64_t kDotsAutoChunks = -1;
constexpr int64_t kDotsMinChunk = 2048;
template <typename T, int W>
void proj_dots(const VParts<T>& V, const T* Wp, const T* Wp2, int64_t ldw, int64_t n, double* C, double* part,
               cudaStream_t s, int64_t rows_per_chunk = 0);
// W -= V C ; if gram: G = W^T W partials, last block chol -> R (+gdiag)
// (returns the status of raising the kernel's shared-memory limit on this device;
// the launch itself is checked by the caller)
template <typename T, int W>
cudaError_t proj_update(const VParts<T>& V, const double* C, T* Wp, T* Wp2, int64_t ldw, int64_t n, int gram,
                        double* R, double* gdiag, unsigned* flags, const Red& red, cudaStream_t s);
// the FP64 products in compensated FP32-pair arithmetic (dispatched from proj_dots /
// proj_update when V.df is set)
template <int W>
void proj_dots_df(const VParts<double>& V, const double* Wp, const double* Wp2, int64_t ldw, int64_t n, double* C,
                  double* part, int64_t rows_per_chunk, cudaStream_t s);
template <int W>
cudaError_t proj_update_df(const VParts<double>& V, const double* C, double* Wp, double* Wp2, int64_t ldw, int64_t n,
                           int gram, double* R, double* gdiag, unsigned* flags, const Red& red, cudaStream_t s);
// raise the shared-memory limit of the P = 1 update kernels to `bytes` ahead of time
template <typename T, int W>
cudaError_t proj_update_reserve_smem(size_t bytes);

// restart GEMM: out_c = Z V_Z(:, sel_c), c < nl -> Lnew (row-major, width nl), else Znext panel (width d)
template <typename T>
cudaError_t restart_gemm(const T* Z, int d, int R, const double* VZ, const int* sel, int nsel, int nl, int64_t n,
                         T* Lnew, T* Znext, cudaStream_t s);
// the same product on the tensor cores (tcgen05, FP32 basis): operands split into
// `slices` bf16 slices (2: 3 products, 3: 6 products), FP32 accumulation in tensor
// memory; image = scratch of restart_umma_image_bytes(R, nsel, slices) bytes; err bit 1
// is set when a bounded mbarrier wait gave up.  Needs restart_umma_supported(R, nsel).
cudaError_t restart_gemm_umma(const float* Z, int d, int R, const double* VZ, const int* sel, int nsel, int nl,
                              int64_t n, float* Lnew, float* Znext, void* image, unsigned* err, int slices,
                              cudaStream_t s);
size_t restart_umma_image_bytes(int R, int nsel, int slices);
bool restart_umma_supported(int R, int nsel);
// the FP64 product on the tensor cores, error-free slicing (eight 7-bit integer slices
// per operand, exact FP32 group sums, int64 combination); R <= 128; scratch of
// restart_ozaki_scratch_bytes(n, R, nsel) bytes
cudaError_t restart_gemm_ozaki(const double* Z, int d, int R, const double* VZ, const int* sel, int nsel, int nl,
                               int64_t n, double* Lnew, double* Znext, void* scratch, unsigned* err, cudaStream_t s);
size_t restart_ozaki_scratch_bytes(int64_t n, int R, int nsel);
bool restart_ozaki_supported(int R, int nsel);
// copy w columns of a row-major panel (ld) into column-major X (ld n) starting at column c0
template <typename T>
void panel_to_cols(const T* P, int64_t ldp, int w, int64_t n, T* X, int c0, cudaStream_t s);
// gather columns [c0, c0+w) of column-major X (T) into an FP64 row-major panel of width w
template <typename T>
void cols_to_panel64(const T* X, int c0, int w, int64_t n, double* P, cudaStream_t s);

// Lanczos step finalization (one block): Gamma_j = R2 R1, norms, W recurrence, flags.
struct OmegaArgs {
  int j, r0, nb, d, nlock;
  double u_d, u_ro;
  const double* R1;
  const double* R2;      // null for a single CholQR pass
  double* Gam;           // Gamma blocks (nb+1) x d x d
  double* nGam;          // ||Gamma_b||
  double* sminGam;       // sigma_min(Gamma_b)
  const double* nXi;     // ||Xi_b||
  const double* nTheta;  // ||Theta_b|| of retained blocks
  const double* nF;      // ||F_b|| of retained blocks
  const double* xtheta;  // locked Ritz values
  const double* xrho;    // locked residuals
  double* wz;            // 3 x (nb+1) rotating columns of W
  double* wx;            // 3 x cap rotating columns of the locked rows
  int cap;
  double bd_tol;
  unsigned* flags;       // bit 1 breakdown, bit 2 reorth Z, bit 4 reorth X
  long long* counters;   // [0] reorth_Z, [1] reorth_X, [2] breakdowns
  double* trace = nullptr;  // optional record, (nb+1) x (nb+1) column-major: column j+1
                            // of W as the recurrence produced it, before any reset
};
void step_finalize(const OmegaArgs& a, cudaStream_t s);
// Gamma and its norms only (first step of a cycle)
void gamma_store(const OmegaArgs& a, cudaStream_t s);
// W columns r0 and r0+1 set to u_d (start of a cycle)
void omega_init(double* wz, double* wx, int nb, int cap, int r0, int nlock, double u_d, cudaStream_t s);
// W column col set to u_d (after a breakdown replacement)
void omega_column(double* wz, double* wx, int nb, int cap, int col, int nlock, double u_d, cudaStream_t s);

// restart bookkeeping: T assembly, Ritz residuals, F, Theta, norms
void build_T(const double* Theta, const double* F, const double* Xi, const double* Gam, int k0, int d, int R,
             double* T, cudaStream_t s);
void ritz_resid(const double* Gam_last, const double* VZ, int d, int R, double* res, cudaStream_t s);
void make_F(const double* Rr, const double* Gam_last, const double* VZ, const int* keep, const double* theta,
            int k0, int d, int R, double* F, double* Theta, double* nTheta, double* nF, cudaStream_t s);

// ---- eigensolver (k_eig.cu) ----
// symmetric k x k (column-major, lower triangle read) -> ascending theta, V (column-major)
void syev(const double* T, int k, double* theta, double* V, double* work, cudaStream_t s);
size_t syev_work_doubles(int k);

// ---- CG / CGLS refinement helpers on row-major panels of width W (k_dense.cu) ----
// delta += alpha p (np rows) ; r -= alpha q (nr rows) ; rr_new[c] = sum_i r_i[c]^2
template <typename T, int W>
void cg_update2(T* delta, const T* p, int64_t np_, T* r, const T* q, int64_t nr, const double* alpha, const Red& red,
                double* rr_new, cudaStream_t s);
// p = s + beta p
template <typename T, int W>
void cg_direction2(T* p, const T* sres, const double* beta, int64_t n, cudaStream_t s);
// out[c] = num[c] / den[c] on active columns, else 0
void cg_scalars(const double* num, const double* den, const unsigned char* active, double* out, int w,
                cudaStream_t s);
// active[c] &= rr[c] > tol2[c] (or > tol2s when tol2 is null) ; *nactive = number of active columns
void cg_check(const double* rr, const double* tol2, double tol2s, unsigned char* active, int* nactive, int w,
              cudaStream_t s);
// out[c] = f2 * rr[c]
void scale_vec(const double* rr, double f2, double* out, int w, cudaStream_t s);
// FP64 column-major <-> zero-padded row-major panel of width W; x -= FP32 correction
template <int W>
void cols_to_panel_w(const double* X, int c0, int w, int64_t n, double* P, cudaStream_t s);
template <int W>
void panel_to_cols64(const double* P, double* X, int c0, int w, int64_t n, cudaStream_t s);
template <int W>
void sub_correction(double* x, const float* dl, int64_t n, cudaStream_t s);

}  // namespace ns

namespace ns {
// ---- re-orthonormalization of the refined FP64 basis (k_dense.cu) ----
size_t gram_part_doubles(int64_t n, int N);
// G = X^T X (X column-major n x N FP64); part needs gram_part_doubles(n, N) doubles
void gram64(const double* X, int64_t n, int N, double* G, double* part, cudaStream_t s);
// Xout = X - 0.5 X (G - I)
void lowdin_update(const double* X, int64_t n, int N, const double* G, double* Xout, cudaStream_t s);
// *out = max |G - I|
void max_offdiag(const double* G, int N, double* out, cudaStream_t s);
// ---- outer preconditioning (k_precond.cu) ----
// one Jones-Plassmann colouring round (colours from cin, new ones written to cout,
// which starts as a copy of cin); *remaining counts vertices left uncoloured
void jp_round(const int64_t* rowptr, const int* col, int64_t n, const double* prio, const int* cin, int* cout,
              unsigned* remaining, cudaStream_t s);
// IC(0) of rows r0..r1 (one colour) of L (CSR, diagonal last, values initialised from
// tril(A~) with the compensated diagonal); *fail |= 1 on a non-positive pivot
void ic0_rows(const int64_t* rp, const int* col, double* val, int64_t r0, int64_t r1, unsigned* fail,
              cudaStream_t s);
void gather_vals(const double* src, const int64_t* map, double* dst, int64_t count, cudaStream_t s);
// x = L^-1 b (lower: diagonal last, colours ascending) or U^-1 b (upper: diagonal first,
// colours descending) on n x D row-major blocks; cstart: host array of ncolors + 1
template <typename T, int D>
void trsv_colors(const int64_t* rp, const int* col, const T* val, const int64_t* cstart, int ncolors, bool lower,
                 const T* b, T* x, cudaStream_t s);
// out = w + eps D x - qprev gprev^T, Xi = sym(x^T out) for a product w formed elsewhere
template <typename T, int D>
void lanczos_epilogue(const T* w, int64_t n, const StepOps<T>& op, const Red& red, cudaStream_t s);
void unpermute_cols(const double* in, const int64_t* perm, int64_t n, int ncols, double* out, cudaStream_t s);
// inner preconditioning with P_L = diag(A A^T): s = 1/||a_i|| (0 for a zero row),
// val_s = S A (A's CSR order), val_t_s = A^T S (A^T's CSR order, col_t its columns)
void inner_scaling(const int64_t* rowptr, const double* val, int64_t m, const int* col_t, const double* val_t,
                   int64_t nnz, double* s, double* val_s, double* val_t_s, cudaStream_t st);
template <typename T>
void cols_to_panel_t(const T* X, int c0, int w, int64_t n, T* P, cudaStream_t s);

}  // namespace ns

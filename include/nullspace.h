/*
 * nullspace.h -- C ABI of the GB300 (sm_103a) null-space library.
 *
 * The library computes an orthonormal basis of the null space of a sparse
 * matrix A (m x n, m >= n, CSR) with the randomized small-block Lanczos method
 * of Kressner & Shao ("On a randomized small-block Lanczos method for
 * large-scale null space computations"), Alg. 2 (restart + partial
 * reorthogonalization), extended by locking of converged null vectors and a
 * final FP64 projection onto null(A).
 *
 * Conventions shared by every call
 *   - Every call returns ns_status; nothing aborts or exits.  CUDA failures map
 *     to NS_ERR_CUDA and their text is kept for ns_last_error().
 *   - Input arrays are borrowed for the duration of the call and copied; the
 *     library never keeps a caller pointer.  Outputs go to caller-owned memory.
 *   - Host pointers are plain C arrays.  "Device" pointers are CUDA global memory
 *     of the current device.  Flags named *_on_device select which one is given.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - All GPU work of a handle runs on the stream given in ns_env (or the legacy
 *     default stream).  Calls return after that work completed unless stated.
 *   - The library needs a CUDA device of compute capability 10.3 (GB300); it has
 *     no CPU fallback and returns NS_ERR_CUDA when no such device is present.
 */
#ifndef NULLSPACE_H
#define NULLSPACE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NS_OK = 0,
  NS_ERR_INVALID_ARG = 1,   /* bad size, pointer or CSR structure; nothing changed */
  NS_ERR_OOM = 2,           /* device allocation failed (allocator returned NULL)  */
  NS_ERR_CUDA = 3,          /* a CUDA call failed; see ns_last_error()             */
  NS_ERR_NOT_CONVERGED = 4, /* max_matvec reached; basis holds what was locked     */
  NS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (no hang)             */
  NS_ERR_STATE = 6,         /* call out of order (e.g. basis before solve)         */
  NS_ERR_REFINE = 7,        /* some column missed the refinement tolerance          */
  NS_ERR_NUMERICAL = 8,     /* a block lost rank during reorthogonalization; a
                               numerical event of the iteration, not a CUDA failure */
  NS_ERR_IO = 9             /* a checkpoint file could not be written, or is missing,
                               truncated or corrupt (checksum)                     */
} ns_status;

typedef enum {
  NS_MODE_NORMAL = 0, /* B = A^T A + eps D              (Eq. defB)                   */
  NS_MODE_SPD = 1     /* B = A + eps D, A symmetric PSD (Sec. 5.1, graph Laplacians) */
} ns_mode;

typedef enum {
  NS_FP64 = 0,  /* everything in FP64                                               */
  NS_MIXED = 1, /* A values, Lanczos basis, SpMM and projections in FP32; projected
                   eigenproblem, W recurrence and final refinement in FP64          */
  NS_FP64_PAIRS = 2 /* ns_project only: FP64 data, products in compensated FP32 pairs
                   (the FP64 path's default arithmetic for its projections)          */
} ns_precision;

typedef enum {
  NS_REORTH_PARTIAL = 0, /* W recurrence of Sec. 4.2 decides (default)              */
  NS_REORTH_FULL = 1     /* project every new block against the whole basis         */
} ns_reorth;

/* Device memory and stream supplied by the caller (e.g. PyTorch's caching
 * allocator and current stream).  alloc must return 256-byte aligned device
 * memory or NULL; free receives the pointer and the size given to alloc.
 * A NULL ns_env (or NULL alloc) makes the library use cudaMalloc/cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* ctx;
  void* stream; /* cudaStream_t; NULL = legacy default stream */
} ns_env;

typedef struct {
  double eps;          /* perturbation strength (Sec. 5.3: 1e-3)                       */
  int precision;       /* ns_precision                                                */
  int reorth;          /* ns_reorth                                                   */
  int64_t max_matvec;  /* cap on B applications per column; <=0: min(100n+50R, 1e6) */
  double stop_factor;  /* stop after stop_factor * s matvecs without a new lock       */
  double lock_tol_mixed; /* lower bound of the lock tolerance on the mixed path         */
  int refine;          /* 1: FP64 projection of the basis onto null(A) (default 1)     */
  double refine_tol;   /* stop when ||A x|| <= refine_tol * ||A||_2 (default 1e-10)    */
  int refine_maxit;    /* CG / CGLS iteration cap per column (default 500)             */
  int refine_chunk;    /* columns refined together: 8, 16 or 32 (default 16)           */
  int use_graphs;      /* ns_solve: unused; ns_batch_solve: >= 0 replays the captured
                          graph (default 0), < 0 launches directly                  */
  int profile;         /* > 0: time every profile-th launch of each kernel class with
                          CUDA events on the library stream (ns_profile); 0 = off   */
  int batch_block;     /* ns_batch_solve: threads per CTA, 128 or 256; 0 = default (128) */
  int gemm;            /* thick-restart product Z V_Z (Sec. 4.1): NS_GEMM_* (default 0)  */
  int fp64_products;   /* FP64 path, Gram-Schmidt products V^T W and W - V C: 0 = compensated
                          FP32 pairs on the FP32 pipe (default; each FP64 operand split
                          exactly into two FP32 words, TwoProd / TwoSum accumulation, error
                          about 2^-47 sum |v w|), 1 = FP64 FMA                            */
  int spmm_schedule;   /* SpMM schedule of ns_solve's B applications: 0 = timed on this matrix
                          at the start of every solve (default); 1, 2, 4 or 8 threads per CSR
                          row, 64 = TMA-staged rows, 128 = sliced ELLPACK (8 threads per row
                          when ns_create did not build that layout).  Schedules sum a row in
                          different orders, and the timed choice can differ between runs:
                          a fixed schedule makes repeated solves bit-identical.            */
  int checkpoint_every;/* > 0: ns_solve writes its state to checkpoint_path after every
                          checkpoint_every-th thick restart, and at the restart where
                          max_matvec stops it; 0 = never (default)                         */
  int resume;          /* 1: ns_solve continues from the state in checkpoint_path instead of
                          drawing a start block; 0 = new solve (default)                  */
  const char* checkpoint_path; /* file of checkpoint_every / resume (NULL = none)          */
  int precond;         /* NS_MODE_SPD only: 1 = outer preconditioning (Sec. 4.4.2), the
                          method runs on B_R = L^-1 A~ L^-T + eps D with A~ = Pi^T A Pi
                          (Pi: renumbering by a Jones-Plassmann colouring of A's graph,
                          priorities from Philox stream 0x7FFFFFFF) and L the zero-fill
                          incomplete Cholesky factor of A~ + precond_shift diag(A~); the
                          basis is mapped back by Pi L^-T, re-orthonormalized and refined
                          against A.  NS_MODE_NORMAL only: 2 = inner preconditioning
                          (Sec. 4.4.1), B_L = A^T P_L^-1 A + eps D with P_L = diag(A A^T),
                          applied as the row scaling (S A)^T (S A), S = P_L^-1/2 (0 on a zero
                          row); same null space, refinement against S A.  0 = none
                          (default).  With precond = 1 the post-processing projects in one
                          pass against up to about 3,000 columns (larger N: NS_ERR_INVALID_ARG) */
  double precond_shift;/* diagonal compensation of the factor (Eq. defichol: 0.1, default) */
} ns_opts;

/* Kernel of the thick-restart product Z V_Z (ns_opts.gemm, ns_restart_product). */
typedef enum {
  NS_GEMM_DEFAULT = 0,   /* the library's choice: NS_GEMM_TC3 on the mixed path, NS_GEMM_TC_EXACT
                            on the FP64 path when restart_len <= 208, else CUDA cores          */
  NS_GEMM_CUDA_CORES = 1,/* FP32 / FP64 FMA register-tile kernels                                 */
  NS_GEMM_TC2 = 2,       /* mixed path: tensor cores, operands split into 2 bf16 slices, 3 products
                            (3xBF16)                                                          */
  NS_GEMM_TC3 = 3,       /* mixed path: tensor cores, 3 bf16 slices, 6 products (FP32 accuracy)  */
  NS_GEMM_TC_EXACT = 4   /* FP64 path: tensor cores, each FP64 operand split exactly into eight
                            7-bit integer slices (per-row / per-column exponents), exact FP32
                            slice sums combined in int64: FP64 accuracy; restart_len <= 208  */
} ns_gemm;

typedef struct {
  int64_t nullity;       /* N = number of locked (null) vectors                      */
  int64_t matvecs;       /* B applications counted per column, as in Table tabCH     */
  int64_t restarts;
  int64_t reorth_X;      /* partial reorthogonalizations against the locked set     */
  int64_t reorth_Z;      /* ... against the active basis                            */
  int64_t breakdowns;
  int64_t lock_events;
  int64_t ghosts;        /* lock candidates rejected as copies of locked vectors    */
  int64_t refine_iters_max;
  int64_t kernel_launches; /* library kernels launched by the last ns_solve        */
  double normB;          /* bound on ||B||_2 used in u_d                             */
  double normA;          /* ||A||_2 estimate (largest Ritz value of the last T)      */
  double u_d;            /* Eq. (defmprd)                                            */
  double refine_resid_max; /* max_j ||A x_j||_2 / ||A||_2 after refinement           */
  double orth_before;    /* max |X^T X - I| after refinement, before re-orthonormalizing */
  double orth_after;     /* same after the symmetric correction (predicted remainder)  */
  double t_lanczos_ms;   /* device time of the Lanczos phase                         */
  double t_refine_ms;    /* device time of the refinement phase                      */
  double t_total_ms;
  int64_t d;             /* block size of the solve (the d = dim K / 16 choice for d = 0) */
  int64_t resumed_at;    /* restarts in the checkpoint a resumed solve started from; -1
                            for a solve that did not resume                          */
} ns_stats_t;

typedef struct ns_handle ns_handle;

/* Fill *o with the defaults listed in ns_opts. */
void ns_default_opts(ns_opts* o);

/* ns_create -- copy A (m x n CSR) to the device, build A^T (normal mode) by a
 * stable counting sort, bound ||B|| and draw D (Alg. 2 (its perturbed operator), Eq. defB).  The
 * problem statement of Sec. 1.1: a sparse A is given, its null space is sought.
 *   rowptr  : m+1 int64, rowptr[0] = 0, non-decreasing, rowptr[m] = nnz
 *   colind  : nnz int32 in [0, n)
 *   vals    : nnz values, finite: double when vals_is_fp32 = 0, float when 1
 *   vals_is_fp32 : 1 = FP32 values; they are kept as given for the mixed path and
 *             widened exactly to FP64 on the device (FP64 path, refinement); no
 *             host-side conversion is needed
 *   inputs_on_device : 0 = the three arrays are host memory, 1 = device memory
 *   seed    : Philox-4x32-10 key for D (stream 0) and the start block (stream 1)
 *   mode    : ns_mode; NS_MODE_SPD requires m == n and a symmetric PSD A (not checked)
 *   env     : allocator / stream, may be NULL; copied into the handle
 * Ownership: the arrays are copied; the caller keeps them.
 * Errors: NS_ERR_INVALID_ARG for m < 0, n <= 0, vals_is_fp32 not 0 or 1, broken CSR
 * structure (host inputs are fully checked; device inputs are checked on the
 * device), NaN/Inf values.  m < n in normal mode is allowed but slow (Remark in
 * Sec. 1.1). */
ns_status ns_create(ns_handle** out, int64_t m, int64_t n, const int64_t* rowptr,
                    const int32_t* colind, const void* vals, int vals_is_fp32, int inputs_on_device,
                    uint64_t seed, int mode, const ns_env* env);

/* ns_solve -- Alg. 2 with locking and refinement (Sec. 4).
 *   d           : block size 1, 2, 4 or 8; 0 = the block-size rule of Sec. 5.3.1,
 *                 d = dim K / 16, taken as the largest of 8, 4, 2, 1 that is at most
 *                 max(1, restart_len / 16) and divides restart_len (ns_stats d)
 *   restart_len : maximal Krylov dimension dim K, multiple of d, >= 3d
 *   tol         : lock a Ritz pair when its value is < 3 eps and its residual
 *                 ||Gamma_l V_Z(last block, i)|| <= tol * ||B|| (Remark cormain), with
 *                 ||B|| = min(cheap bound ||A||_1 ||A||_inf + eps (normal) or
 *                 ||A||_inf + eps (SPD), 1.1 x the largest Ritz value seen); the same
 *                 ||B|| scales u_d of the W recurrence
 *   opts        : NULL = defaults
 * Returns NS_OK, NS_ERR_NOT_CONVERGED (max_matvec reached; the basis holds the
 * vectors locked so far), NS_ERR_REFINE (a column missed refine_tol),
 * NS_ERR_NUMERICAL (a reorthogonalized block lost rank), or an error.
 * May be called again on the same handle (new solve, same D and start seed).
 * Checkpoints (opts checkpoint_every, resume, checkpoint_path): at a thick restart
 * (Alg. 2 (the restarted coupling F)) the whole state of the iteration is the retained Ritz vectors
 * and the next block, the projected matrix's arrow part, the W rows, the locked
 * vectors with their Ritz values and residuals, the counters and the SpMM
 * schedules.  A checkpoint holds exactly that (written to checkpoint_path + ".tmp",
 * then renamed over checkpoint_path, so an interrupted write leaves the previous
 * file intact).  A resumed solve restores it and continues as the uninterrupted
 * solve would: with the same opts (max_matvec, stop_factor and the refinement
 * options may differ) its basis and counters are bit-identical to those of a solve
 * that ran straight through with the schedules of the checkpoint.  max_matvec
 * counts B applications since the start of the solve, including those before the
 * checkpoint.  A resumed solve needs a handle made from the same matrix and seed
 * and the same d, restart_len, tol, eps, precision, reorth, gemm and
 * fp64_products, else NS_ERR_INVALID_ARG; an unreadable or corrupt file gives
 * NS_ERR_IO.  A checkpoint stores at most (restart_len + d) n + N n values of the
 * solve's type (N locked vectors) plus O(restart_len^2) doubles. */
ns_status ns_solve(ns_handle* h, int d, int restart_len, double tol, const ns_opts* opts);

/* What a checkpoint file written by ns_solve holds (all fields 8 bytes). */
typedef struct {
  int64_t version;         /* format version, 1                                        */
  int64_t m, n, nnz, mode; /* the matrix of the solve                                  */
  int64_t precision, d, restart_len, reorth, gemm, fp64_products; /* the solve's opts  */
  int64_t spmm_A, spmm_At; /* SpMM schedules in use (A, A^T; A^T is 0 in SPD mode)   */
  uint64_t seed;
  double eps, tol_eff;     /* perturbation strength; lock tolerance in use             */
  double normA1, normAinf; /* ||A||_1, ||A||_inf of the handle (a check of the values) */
  int64_t matvecs, restarts, nullity; /* progress: B applications, restarts, locked   */
  int64_t k0;              /* retained Ritz vectors (the next cycle starts at block k0/d) */
  double precond;          /* precond_shift of an outer-preconditioned solve, -1 inner, 0 none */
} ns_checkpoint_info;

/* ns_read_checkpoint -- read and verify a checkpoint file on the host (no device
 * work): its magic, its length and its FNV-1a checksum.  File layout: 8 bytes
 * "NSCKPT01", the ns_checkpoint_info record, the solver state (host byte order),
 * then the 64-bit checksum of everything before it, computed over little-endian
 * 64-bit words (FNV-1a with the word in place of the byte; a tail shorter than
 * 8 bytes is zero-padded).  NS_ERR_IO for a missing, short or corrupt file. */
ns_status ns_read_checkpoint(const char* path, ns_checkpoint_info* info);

/* Number of null vectors found by the last ns_solve. NS_ERR_STATE before a solve. */
ns_status ns_nullity(const ns_handle* h, int64_t* N);

/* Copy the n x N basis (FP64, column-major, leading dimension ld >= n) to out. */
ns_status ns_basis(const ns_handle* h, double* out, int64_t ld, int out_on_device);

/* Counters and timings of the last ns_solve. */
ns_status ns_stats(const ns_handle* h, ns_stats_t* s);

/* Per-kernel-class measurements of the last ns_solve run with opts.profile > 0.
 * Classes: 0 B-apply (SpMM + recurrence epilogue), 1 recurrence / block QR,
 * 2 CGS2 projections, 3 restart GEMM, 4 projected eigenproblem, 5 locking,
 * 6 refinement, 7 re-orthonormalization.  Bytes and flops are algorithmic
 * (each operand counted once), per launch, averaged over all launches of the
 * class; ms_per_launch is the mean CUDA-event duration of the sampled launches. */
typedef struct {
  char name[24];
  int64_t launches;
  int64_t sampled;
  double ms_per_launch;
  double bytes_per_launch;
  double flops_per_launch;
  double ms_total_est; /* ms_per_launch * launches */
} ns_kernel_prof;

/* Copies min(max, 8) class records to out; returns the number written in *count. */
ns_status ns_profile(const ns_handle* h, ns_kernel_prof* out, int max, int* count);

/* Text of the last error on this handle ("" if none; static string for NULL). */
const char* ns_last_error(const ns_handle* h);

/* Release every device buffer of the handle. NULL is ignored. */
void ns_destroy(ns_handle* h);

/* ---------------------------------------------------------------------------
 * Kernel-level entry points.  They expose single steps of the path on the
 * matrix held by a handle, so that each can be checked on its own.
 * -------------------------------------------------------------------------*/

/* Copy A^T as built on the device (CSR: n+1 rowptr, nnz colind, nnz vals) to
 * host arrays.  Entries of each row of A^T keep the order of the rows of A.
 * NS_ERR_STATE in SPD mode (no transpose is built). */
ns_status ns_get_transpose(const ns_handle* h, int64_t* rowptr, int32_t* colind, double* vals);

/* Copy the diagonal D (n doubles, U[0,1), Philox stream 0) to host memory. */
ns_status ns_get_perturbation(const ns_handle* h, double* D);

/* Draw the n x d start block Omega (row-major, Philox stream 1, Box-Muller) into
 * host memory, exactly as ns_solve draws it (Alg. 2 (its Gaussian start block)). */
ns_status ns_start_block(const ns_handle* h, int d, double* Omega);

/* Y = B X (Eq. defB) for an n x d row-major block, 1 <= d <= 8.
 *   X, Y       : n*d doubles, host or device memory (on_device)
 *   eps        : perturbation strength
 *   precision  : NS_FP64 or NS_MIXED (X rounded to FP32, FP32 arithmetic with
 *                FP32 values of A; Y returned widened to FP64)
 *   schedule   : SpMM schedule: -1 the library's default for this matrix, 1, 2, 4,
 *                8, 16 or 32 threads per CSR row, 64 the TMA-staged schedule
 *                (each CTA bulk-copies a 256-row tile's col/val into shared memory,
 *                a thread per row), or 128 the sliced-ELLPACK copy built by ns_create
 *                (slices of 32 rows, a warp per slice, a lane per row; built when its
 *                padding stays below 30% of nnz, else NS_ERR_INVALID_ARG); anything
 *                else gives NS_ERR_INVALID_ARG.
 * A bounded device wait that expires gives NS_ERR_TIMEOUT (no hang). */
ns_status ns_apply_B(ns_handle* h, int d, const double* X, double* Y, double eps,
                     int precision, int on_device, int schedule);

/* ns_precond_build -- build (or reuse) the outer preconditioner of ns_solve's
 * opts.precond (Sec. 4.4.2, Eq. defichol) on this handle, exposed so that each step
 * can be checked on its own.  NS_MODE_SPD only (else NS_ERR_STATE).
 *   Colouring: Jones-Plassmann rounds on the device; vertex v's priority is the
 *   uniform draw v of Philox stream 0x7FFFFFFF (key: the handle's seed), ties by
 *   index; in each round every uncoloured vertex that beats all its uncoloured
 *   neighbours takes the smallest colour none of its coloured neighbours has.
 *   Renumbering: perm[new] = old, vertices ordered by colour, then by index.
 *   Factor: L, the zero-fill incomplete Cholesky factor of A~ + shift diag(A~),
 *   A~ = Pi^T A Pi, computed on the device one colour at a time.
 *   color   : n int32 (original numbering), may be NULL
 *   perm    : n int64, may be NULL
 *   nnz_L   : entries of L (diagonal included), may be NULL
 *   ncolors : colours used, may be NULL
 * A new shift refactors.  NS_ERR_NUMERICAL when a pivot is not positive (raise the
 * shift); NS_ERR_INVALID_ARG for a negative or non-finite shift. */
ns_status ns_precond_build(ns_handle* h, double shift, int32_t* color, int64_t* perm, int64_t* nnz_L,
                           int32_t* ncolors);

/* The factor L of the last ns_precond_build (or preconditioned ns_solve): CSR of the
 * renumbered matrix, n + 1 rowptr, nnz_L colind (ascending in a row, the diagonal
 * last) and vals, host arrays.  NS_ERR_STATE before a build. */
ns_status ns_precond_factor(const ns_handle* h, int64_t* rowptr, int32_t* colind, double* vals);

/* ns_inner_precond -- build (or reuse) the inner preconditioner of opts.precond = 2
 * (Sec. 4.4.1) on a NS_MODE_NORMAL handle (else NS_ERR_STATE): P_L = diag(A A^T), kept
 * as the row scaling s_i = 1/||a_i||_2 (0 for a zero row) and the scaled copies S A
 * and A^T S.  row_scale: m doubles (host) receiving s, may be NULL. */
ns_status ns_inner_precond(ns_handle* h, double* row_scale);

/* Y = B_R X = L^-1 A~ L^-T X + eps D X in the renumbered space (D indexed there as
 * drawn) on a NS_MODE_SPD handle, or Y = B_L X = A^T P_L^-1 A X + eps D X on a
 * NS_MODE_NORMAL handle; an n x d row-major block, d in {1, 2, 4, 8}; host or device
 * memory (on_device); precision NS_FP64 or NS_MIXED (FP32 values and arithmetic, Y
 * widened).  The triangular solves take one launch per colour.  NS_ERR_STATE
 * before ns_precond_build / ns_inner_precond. */
ns_status ns_apply_precond(ns_handle* h, int d, const double* X, double* Y, double eps, int precision,
                           int on_device);

/* ns_fma_peak -- measured FMA throughput of the current device, in TFLOP/s (two
 * flops per FMA), for precision NS_FP64 (the FP64 pipe) or NS_MIXED (the FP32
 * pipe).  The paper has no counterpart: it is the roofline denominator of the
 * FP64 path, whose dense products are bound by the FP64 pipe.  Runs a grid of 8
 * CTAs of 256 threads per SM, each thread 8 independent FMA chains; the best of
 * three timed launches after one warm-up (about 50 ms each).  Allocates and frees
 * a small device buffer; uses the legacy default stream. */
ns_status ns_fma_peak(int precision, double* tflops);

/* ns_restart_product -- the thick-restart product of Alg. 2 (Sec. 4.1: the retained
 * Ritz vectors Z V_Z(:, keep) and the locked candidates) exactly as ns_solve computes
 * it, exposed so that each kernel can be checked on its own.
 *   Z   : n x R column-major FP64, host (the Lanczos basis; blocks of d columns)
 *   VZ  : R x R column-major FP64, host (eigenvectors of T)
 *   sel : nsel column indices into VZ, host
 *   nl  : the first nl outputs go to the locked-candidate panel, the rest to the
 *         next basis (the two output layouts ns_solve uses); 0 <= nl <= nsel
 *   precision : NS_FP64 (FP64 Z) or NS_MIXED (Z rounded to FP32, FP32 result)
 *   gemm      : ns_gemm; NS_GEMM_TC2 / TC3 need precision NS_MIXED and nsel <= 256,
 *               NS_GEMM_TC_EXACT needs NS_FP64 and R <= 208
 *   out : n x nsel column-major FP64, host
 * d in {1, 2, 4, 8}, R a multiple of d, 1 <= R <= 512.  NS_ERR_TIMEOUT when a bounded
 * device wait gave up.  Allocates its own device buffers. */
ns_status ns_restart_product(int64_t n, int d, int R, const double* Z, const double* VZ, const int32_t* sel,
                             int nsel, int nl, int precision, int gemm, double* out);

/* ns_trace_omega -- the W recurrence of Sec. 4.2 (the bounds w_{k,l} on
 * ||Q_k^T Q_l|| that decide partial reorthogonalization) exactly as ns_solve
 * computes it, exposed so that it can be checked on its own.  Runs the first
 * Lanczos cycle of ns_solve on this handle (start block, steps 1 .. nb-1 with the
 * reorthogonalizations they trigger; no restart, no locking) with the same d,
 * restart_len and opts (checked as ns_solve checks them; a preconditioner named in
 * opts is built and its operator traced; checkpoint options are ignored), and
 * records every new W column.
 *   W : (nb+1) x (nb+1) doubles, column-major, host memory, nb = restart_len / d.
 *       Entry (b, c), b < c, c >= 2, is w_{b,c} as the recurrence produced it,
 *       before the reset to u_d that a reorthogonalization makes; columns 0 and 1
 *       (set to u_d by definition) and entries b >= c are 0.
 * Does not change the handle's last solve result.  Errors as for ns_solve. */
ns_status ns_trace_omega(ns_handle* h, int d, int restart_len, const ns_opts* opts, double* W);

/* Eigen-decomposition of a symmetric k x k matrix (k <= 512) on the device with
 * the library's FP64 solver (Householder tridiagonalization in one CTA, Sturm
 * multisection and inverse iteration spread over the SMs),
 * the solver used for the projected matrix T of Alg. 2 (the projected matrix T).
 *   T     : k*k doubles, column-major, host memory (only the lower triangle is read)
 *   theta : k eigenvalues, ascending;  V : k*k column-major eigenvectors */
ns_status ns_syev(int k, const double* T, double* theta, double* V);

/* Block classical Gram-Schmidt, two passes (CGS2), as used for the partial
 * reorthogonalization (Sec. 4.2): W <- (I - V V^T)^2 W for V (n x K, column-major)
 * and W (n x w, row-major, 1 <= w <= 8).  Host arrays; precision NS_FP64 (FP64
 * FMA), NS_FP64_PAIRS (FP64 data, compensated FP32-pair products, as ns_solve's
 * FP64 path uses by default) or NS_MIXED (FP32).  C (K x w, row-major) receives the
 * summed coefficients of both passes. */
ns_status ns_project(int64_t n, int K, int w, const double* V, double* W, double* C, int precision);

/* ns_project_noalloc -- the same FP64 CGS2 projection as ns_project, for callers
 * that cannot allocate device memory while they run (code inside a CUDA graph
 * being captured, where cudaMalloc is refused; an allocator's own callback, which
 * must not re-enter the allocator; hosts that only hand over pre-allocated
 * buffers).  The paper has no counterpart; this is a service of the library.  It
 * allocates nothing: its scratch is a fixed 4 MiB device array inside the library
 * (held on every GPU that loads the library until exit).
 *   V : n x K column-major FP64, device memory (read)
 *   W : n x w row-major FP64,   device memory (overwritten by W - V V^T W, twice)
 *   C : K x w row-major FP64,   device memory (receives the summed coefficients)
 *   stream : cudaStream_t, NULL = legacy default stream; the call only enqueues work
 * Limits: w in {1, 2, 4, 8}; K*w*(ceil(n/32768)+1) <= 524288 and K*w <= 24320,
 * else NS_ERR_INVALID_ARG (nothing enqueued).
 * Set-up: the first call on a device (and the first after that device's context
 * was reset) looks up the scratch address and raises the projection kernels'
 * shared-memory limit; it must be made outside any stream capture.  Made while
 * `stream` is capturing, it returns NS_ERR_STATE and enqueues nothing.  Later calls
 * only enqueue kernels.
 * Errors: an error already pending on the calling thread gives NS_ERR_CUDA, is left
 * pending for the caller, and nothing is enqueued.  A launch of this call that
 * fails gives NS_ERR_CUDA; W and C are then undefined (partly projected).
 * Sharing: all calls share the one scratch array and every call fully overwrites
 * what it reads, so calls that overlap on the GPU (different streams, no ordering)
 * race and give wrong results. */
ns_status ns_project_noalloc(int64_t n, int K, int w, const double* V, double* W, double* C, void* stream);

/* ------------------------------------------------------------------------
 * Batched form: many independent symmetric PSD matrices (e.g. graph
 * Laplacians), each solved with B_i = A_i + eps D_i (Sec. 5.1 form, d = 1), all
 * in ONE persistent kernel launch replayed from a CUDA graph.  CTAs take
 * instances from an atomic work queue, largest first; each CTA runs the whole
 * method for its instance (Alg. 2 with the W recurrence of Sec. 4.2, locking,
 * thick restart, the stopping rule of Sec. 4.3) with FP32 vectors and an FP64
 * projected problem, then projects every locked vector onto null(A_i) by FP64
 * CG and re-orthonormalizes in FP64.  Instance i draws D_i (Philox stream 0)
 * and its start vector (stream 1) from key seed + i.
 * ------------------------------------------------------------------------ */
typedef struct ns_batch ns_batch;

typedef struct {
  int64_t count;          /* instances                                              */
  int64_t total_nullity;  /* sum of the per-instance nullities                      */
  int64_t failed;         /* instances whose status is not 0                        */
  int64_t matvecs_total;  /* B applications summed over instances                   */
  int64_t matvecs_max;
  int64_t kernel_launches;/* library kernels launched by the last ns_batch_solve    */
  int lanes;              /* threads per CSR row in the SpMV (autotuned: 1, 2 or 4) */
  int grid;               /* CTAs of the persistent launch                          */
  int blocks_per_sm;
  int block;              /* threads per CTA                                        */
  int graph;              /* 1 when the launch was replayed from a CUDA graph       */
  double t_solve_ms;      /* device time of the last solve (graph replay)          */
  double t_tune_ms;       /* device time spent by the autotuner (first solve)       */
} ns_batch_stats_t;

/* ns_batch_create -- copy `count` CSR matrices (host memory) to the device.
 *   n      : count row counts, each in [1, 2^31); every A_i is n_i x n_i
 *   rowptr : the count local row-pointer arrays back to back (n_i + 1 int64 each,
 *            starting at 0, non-decreasing)
 *   colind : the entries' column indices back to back (int32, local to the instance)
 *   vals   : the entries' values back to back, finite: double when vals_is_fp32 =
 *            0 (an FP32 copy is made for the Lanczos phase), float when 1 (kept as
 *            given; an exact FP64 widening is made on the device for the refinement)
 *   vals_is_fp32 : 0 or 1, see vals
 *   seed   : Philox key of instance 0 (instance i uses seed + i)
 *   env    : allocator / stream as for ns_create, may be NULL (the library then
 *            uses its own non-blocking stream)
 * A_i must be symmetric PSD (not checked).  Errors: NS_ERR_INVALID_ARG (bad
 * count, size or row structure, checked on the host before anything is
 * allocated; a column index outside its instance or a non-finite value, checked
 * on the device after the copy, everything freed again), NS_ERR_OOM, NS_ERR_CUDA. */
ns_status ns_batch_create(ns_batch** out, int64_t count, const int64_t* n, const int64_t* rowptr,
                          const int32_t* colind, const void* vals, int vals_is_fp32, uint64_t seed,
                          const ns_env* env);

/* ns_batch_solve -- solve every instance.  d must be 1; restart_len in [8, 64]
 * and every n_i >= restart_len + 34 (the basis, its next vector and up to 32
 * locked vectors must fit); tol > 0 (lock when the Ritz residual is at most
 * max(tol, 1e-5) ||B_i||, FP32 vectors).  From opts (NULL = defaults) it reads
 * eps (> 0: the null test is theta < 3 eps; no unperturbed variant here), max_matvec (<= 0: min(100 n_i + 50 restart_len, 1e6) per instance),
 * stop_factor, refine_tol (||A x|| <= refine_tol * ||A_i||_2), refine_maxit;
 * precision is ignored (the batched form is always the mixed one); use_graphs
 * >= 0 (default) replays the captured graph {queue reset, persistent launch},
 * re-capturing it only when an argument changed, use_graphs < 0 launches
 * directly.  The first
 * solve of a shape class (device, CTA size, restart_len, mean row length, largest
 * instance) autotunes the SpMV lanes on a sample of instances; later handles of
 * the same class in the process reuse that choice (t_tune_ms = 0).  Returns NS_OK when
 * every instance has status 0, else the first non-zero status among
 * NS_ERR_NOT_CONVERGED (max_matvec reached, or more than 32 null vectors) and
 * NS_ERR_REFINE; per-instance results stay readable either way. */
ns_status ns_batch_solve(ns_batch* hb, int d, int restart_len, double tol, const ns_opts* opts);

/* Per-instance results of the last solve (host arrays of `count` entries; any
 * pointer may be NULL): nullity, status (0 ok, 4 max_matvec reached, 7
 * refinement missed its tolerance, 8 more than 32 null vectors) and, in istats
 * (count x 13, row-major), matvecs, restarts, partial reorthogonalizations, the
 * largest refinement iteration count, the SM clock cycles the instance took,
 * those cycles split by phase (Lanczos steps, partial reorthogonalization,
 * projected eigenproblem, locking, thick restart, refinement), and the FP32 and
 * FP64 Jacobi sweeps spent on the projected problems. */
ns_status ns_batch_results(const ns_batch* hb, int32_t* nullity, int32_t* status, int64_t* istats);

/* Null-space basis of instance i: n_i x N_i column-major FP64 into out with
 * leading dimension ld >= n_i (host memory, or device memory if out_on_device). */
ns_status ns_batch_basis(const ns_batch* hb, int64_t i, double* out, int64_t ld, int out_on_device);

/* Every basis of the last solve in one call: instance i's n_i x N_i column-major
 * block starts at offset sum_{j<i} n_j N_j of out (sum_i n_i N_i doubles; N_i
 * from ns_batch_results).  out is host memory, or device memory if out_on_device;
 * a host copy goes through one device staging buffer and one transfer. */
ns_status ns_batch_basis_packed(const ns_batch* hb, double* out, int out_on_device);

ns_status ns_batch_stats(const ns_batch* hb, ns_batch_stats_t* s);
const char* ns_batch_last_error(const ns_batch* hb);
void ns_batch_destroy(ns_batch* hb);

#ifdef __cplusplus
}
#endif

#endif /* NULLSPACE_H */

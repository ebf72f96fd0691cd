// Host driver and C ABI of the null-space library.
//
// Control flow of Alg. 2 (Kressner & Shao) with locking: the device runs every
// arithmetic step (SpMM, recurrence, QR, W recurrence, projections, projected
// eigenproblem, restart GEMM, refinement); the host only sequences kernels and
// takes the per-restart decisions (which Ritz pairs to lock or keep, when to
// stop) from a few scalars it reads back.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nullspace.h"
#include "ns_checkpoint.cuh"
#include "ns_common.cuh"
#include "ns_kernels.cuh"

using namespace ns;

// Sampling profiler: every `every`-th launch of each kernel class is bracketed
// by CUDA events on the library stream; algorithmic bytes / flops of every
// launch are accumulated from the operand sizes.
struct Prof {
  static constexpr int NC = 8;
  int every = 0;
  cudaStream_t s = nullptr;
  long long units[NC] = {}, sampled[NC] = {}, counter[NC] = {};
  double ms[NC] = {}, bytes[NC] = {}, flops[NC] = {};
  struct Pend {
    int c;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Pend> pend;
  void reset(int e, cudaStream_t st) {
    every = e;
    s = st;
    for (int c = 0; c < NC; ++c) units[c] = sampled[c] = counter[c] = 0, ms[c] = bytes[c] = flops[c] = 0.0;
    pend.clear();
    used = 0;
  }
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  int begin(int c, double by, double fl, bool timed = true) {
    units[c] += 1;
    bytes[c] += by;
    flops[c] += fl;
    if (!timed || every <= 0 || (counter[c]++ % every) != 0) return -1;
    Pend p{c, ev(), ev()};
    cudaEventRecord(p.a, s);
    pend.push_back(p);
    return (int)pend.size() - 1;
  }
  void end(int tok) {
    if (tok >= 0) cudaEventRecord(pend[tok].b, s);
  }
  // algorithmic work of a launch of class c that is only known after it was enqueued
  void add(int c, double by, double fl) {
    bytes[c] += by;
    flops[c] += fl;
  }
  void flush() {  // call after the stream was synchronized
    for (auto& p : pend) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.c] += t;
        sampled[p.c] += 1;
      }
    }
    cudaGetLastError();
    pend.clear();
    used = 0;
  }
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct PScope {
  Prof* p;
  int tok;
  PScope(Prof* pp, int c, double by, double fl, bool timed = true) : p(pp), tok(pp->begin(c, by, fl, timed)) {}
  ~PScope() { p->end(tok); }
};

enum { P_APPLY = 0, P_REC = 1, P_PROJ = 2, P_GEMM = 3, P_EIG = 4, P_LOCK = 5, P_REFINE = 6, P_ORTH = 7 };
static const char* kProfNames[Prof::NC] = {"b_apply", "recurrence_qr", "cgs2_project", "restart_gemm",
                                           "projected_eig", "locking", "refine", "reorthonormalize"};

struct ns_handle {
  ns_env env{};
  bool own_alloc = true;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t m = 0, n = 0, nnz = 0;
  int mode = 0;
  uint64_t seed = 0;
  int64_t maxrow_A = 0, maxrow_At = 0;
  // device matrix
  int64_t* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  int64_t* rowptr_t = nullptr;
  int* col_t = nullptr;
  double* val_t = nullptr;
  float* val_t32 = nullptr;
  double* D64 = nullptr;
  float* D32 = nullptr;
  double normA1 = 0.0, normAinf = 0.0;
  // sliced-ELLPACK copies of A and A^T (null when the padding would exceed 30%)
  struct Sell {
    int64_t* sptr = nullptr;
    int* scol = nullptr;
    double* sval = nullptr;
    float* sval32 = nullptr;
    int64_t entries = 0;
  } sell_A, sell_At;
  // outer preconditioner P_R = Pi L of the SPD form (Sec. 4.4.2), built on first use
  struct Pc {
    bool built = false;
    double alpha = -1.0;       // diagonal compensation the factor was computed with
    int ncolors = 0;
    std::vector<int64_t> cstart;  // first renumbered row of each colour (host), ncolors + 1
    std::vector<int> color_h;     // colour of each original vertex (host)
    std::vector<int64_t> perm_h;  // perm[new] = old (host)
    std::vector<double> linit;    // L's initial values: tril(A~) with the uncompensated diagonal
    int64_t nnzL = 0, nnzA = 0;
    int64_t* perm = nullptr;
    int64_t *arp = nullptr, *lrp = nullptr, *urp = nullptr, *umap = nullptr;
    int *acol = nullptr, *lcol = nullptr, *ucol = nullptr;
    double *aval = nullptr, *lval = nullptr, *uval = nullptr;
    float *aval32 = nullptr, *lval32 = nullptr, *uval32 = nullptr;
  } pc;
  // inner preconditioner P_L = diag(A A^T) of the normal form (Sec. 4.4.1), built on first use
  struct Inner {
    bool built = false;
    double* s = nullptr;                       // 1 / ||a_i||_2 per row of A (0 for a zero row)
    double *val = nullptr, *val_t = nullptr;   // S A and A^T S (A's and A^T's CSR order)
    float *val32 = nullptr, *val_t32 = nullptr;
    double normA1 = 0.0, normAinf = 0.0;       // ||S A||_1, ||S A||_inf
  } inner;
  // result
  bool solved = false;
  int64_t N = 0;
  double* basis = nullptr;
  size_t basis_bytes = 0;
  ns_stats_t stats{};
  long long launches = 0;
  Prof prof;
  std::vector<std::pair<void*, size_t>> owned;  // matrix-side arrays and their sizes, freed by ns_destroy
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

struct Fail {
  ns_status st;
  std::string msg;
};

void* dalloc(ns_handle* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (!h->own_alloc) {
    p = h->env.alloc(bytes, h->env.ctx);
    if (!p) throw Fail{NS_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes"};
  } else {
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Fail{NS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    }
  }
  return p;
}

void dfree(ns_handle* h, void* p, size_t bytes) {
  if (!p) return;
  if (!h->own_alloc)
    h->env.free(p, bytes ? bytes : 256, h->env.ctx);
  else
    cudaFree(p);
}

// allocation that lives as long as the handle (its size is kept for the free callback)
void* dalloc_own(ns_handle* h, size_t bytes) {
  void* p = dalloc(h, bytes);
  h->owned.emplace_back(p, bytes ? bytes : 256);
  return p;
}

// CSR col/val arrays end with kCsrPad entries of padding: the TMA-staged SpMM copies
// the 16-byte aligned span around each tile's segment
size_t csr_entries(int64_t nnz) { return (size_t)std::max<int64_t>(nnz, 1) + kCsrPad; }

void ck_at(cudaError_t e, const char* what, int line) {
  if (e != cudaSuccess)
    throw Fail{NS_ERR_CUDA, std::string(what) + " (ns_api.cu:" + std::to_string(line) + "): " + cudaGetErrorString(e)};
}
#define ck(e, what) ck_at((e), (what), __LINE__)

void ck_launch_at(const char* what, int line) { ck_at(cudaGetLastError(), what, line); }
#define ck_launch(what) ck_launch_at((what), __LINE__)

// RAII device buffer through the handle's allocator
struct Buf {
  ns_handle* h = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  Buf() = default;
  Buf(ns_handle* hh, size_t b) : h(hh), p(dalloc(hh, b)), bytes(b) {}
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  Buf(Buf&& o) noexcept : h(o.h), p(o.p), bytes(o.bytes) { o.p = nullptr; }
  Buf& operator=(Buf&& o) noexcept {
    release();
    h = o.h;
    p = o.p;
    bytes = o.bytes;
    o.p = nullptr;
    return *this;
  }
  ~Buf() { release(); }
  void release() {
    if (p) dfree(h, p, bytes);
    p = nullptr;
  }
  template <typename U>
  U* as() const {
    return reinterpret_cast<U*>(p);
  }
};

template <typename T>
struct Prec;
template <>
struct Prec<double> {
  static const double* D(ns_handle* h) { return h->D64; }
  static const double* val(ns_handle* h) { return h->val; }
  static const double* val_t(ns_handle* h) { return h->val_t; }
  static const double* sval(const ns_handle::Sell& s) { return s.sval; }
};
template <>
struct Prec<float> {
  static const float* D(ns_handle* h) { return h->D32; }
  static const float* val(ns_handle* h) { return h->val32; }
  static const float* val_t(ns_handle* h) { return h->val_t32; }
  static const float* sval(const ns_handle::Sell& s) { return s.sval32; }
};

// sliced-ELLPACK copy of a device CSR (slices of kSellC rows, column-major inside a
// slice), kept when its padding stays below 30% of nnz
void build_sell(ns_handle* h, const int64_t* rowptr, const int* col, const double* val, int64_t nrows, int64_t nnz,
                ns_handle::Sell& out) {
  const int64_t nslices = (nrows + kSellC - 1) / kSellC;
  if (nslices == 0) return;
  Buf len(h, sizeof(int) * (size_t)nslices);
  sell_lengths(rowptr, nrows, len.as<int>(), h->stream);
  ck_launch("sell_lengths");
  std::vector<int> lh((size_t)nslices);
  ck(cudaMemcpyAsync(lh.data(), len.p, sizeof(int) * nslices, cudaMemcpyDeviceToHost, h->stream), "d2h");
  ck(cudaStreamSynchronize(h->stream), "sync");
  std::vector<int64_t> ptr((size_t)nslices + 1, 0);
  for (int64_t i = 0; i < nslices; ++i) ptr[i + 1] = ptr[i] + (int64_t)kSellC * lh[i];
  const int64_t entries = ptr[nslices];
  if ((double)entries > 1.3 * (double)std::max<int64_t>(nnz, 1)) return;
  out.sptr = (int64_t*)dalloc_own(h, sizeof(int64_t) * (size_t)(nslices + 1));
  out.scol = (int*)dalloc_own(h, sizeof(int) * (size_t)std::max<int64_t>(entries, 1));
  out.sval = (double*)dalloc_own(h, sizeof(double) * (size_t)std::max<int64_t>(entries, 1));
  out.entries = entries;
  ck(cudaMemcpyAsync(out.sptr, ptr.data(), sizeof(int64_t) * (nslices + 1), cudaMemcpyHostToDevice, h->stream), "h2d");
  sell_fill(rowptr, col, val, nrows, out.sptr, out.scol, out.sval, h->stream);
  ck_launch("sell_fill");
  ck(cudaStreamSynchronize(h->stream), "sync");  // ptr (host) is read by the copy above
}

constexpr uint32_t kPriorityStream = 0x7FFFFFFFu;  // Philox stream of the colouring priorities

// Outer preconditioner of the SPD form (Sec. 4.4.2, Eq. defichol): Jones-Plassmann
// colouring of A's graph on the device (priorities: Philox stream kPriorityStream),
// renumbering colour by colour, the patterns of A~ = Pi^T A Pi, L = tril(A~) and
// L^T on the host, then IC(0) of A~ + alpha diag(A~) on the device, one launch
// per colour.  The structure is built once per handle; a new alpha refactors.
void build_precond(ns_handle* h, double alpha) {
  auto& P = h->pc;
  cudaStream_t s = h->stream;
  const int64_t n = h->n, nnz = h->nnz;
  if (!P.built) {
    // ---- colouring ----
    Buf prio(h, sizeof(double) * n), c0(h, sizeof(int) * n), c1(h, sizeof(int) * n), rem(h, 256);
    rng_uniform<double>(h->seed, kPriorityStream, prio.as<double>(), n, s);
    ck(cudaMemsetAsync(c0.p, 0xFF, sizeof(int) * n, s), "memset");
    unsigned* rem_h = nullptr;
    ck(cudaMallocHost(&rem_h, 64), "cudaMallocHost");
    for (int64_t round = 0; round <= n; ++round) {  // every round colours the largest priority left
      ck(cudaMemcpyAsync(c1.p, c0.p, sizeof(int) * n, cudaMemcpyDeviceToDevice, s), "copy");
      ck(cudaMemsetAsync(rem.p, 0, sizeof(unsigned), s), "memset");
      jp_round(h->rowptr, h->col, n, prio.as<double>(), c0.as<int>(), c1.as<int>(), rem.as<unsigned>(), s);
      h->launches += 1;
      ck(cudaMemcpyAsync(rem_h, rem.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
      ck(cudaStreamSynchronize(s), "sync");
      std::swap(c0, c1);
      if (*rem_h == 0) break;
    }
    cudaFreeHost(rem_h);
    ck_launch("colouring");
    P.color_h.assign(n, 0);
    ck(cudaMemcpyAsync(P.color_h.data(), c0.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "d2h");
    std::vector<int64_t> rp(n + 1);
    std::vector<int> col(nnz);
    std::vector<double> val(nnz);
    ck(cudaMemcpyAsync(rp.data(), h->rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s), "d2h");
    if (nnz) {
      ck(cudaMemcpyAsync(col.data(), h->col, sizeof(int) * nnz, cudaMemcpyDeviceToHost, s), "d2h");
      ck(cudaMemcpyAsync(val.data(), h->val, sizeof(double) * nnz, cudaMemcpyDeviceToHost, s), "d2h");
    }
    ck(cudaStreamSynchronize(s), "sync");
    // ---- renumbering: colour by colour, index order inside a colour ----
    int nc = 0;
    for (int64_t v = 0; v < n; ++v) {
      if (P.color_h[v] < 0) throw Fail{NS_ERR_CUDA, "colouring left a vertex uncoloured"};
      nc = std::max(nc, P.color_h[v] + 1);
    }
    P.ncolors = nc;
    P.cstart.assign(nc + 1, 0);
    for (int64_t v = 0; v < n; ++v) P.cstart[P.color_h[v] + 1] += 1;
    for (int c = 0; c < nc; ++c) P.cstart[c + 1] += P.cstart[c];
    P.perm_h.assign(n, 0);
    std::vector<int64_t> iperm(n), fill(P.cstart.begin(), P.cstart.end() - 1);
    for (int64_t v = 0; v < n; ++v) {
      const int64_t i = fill[P.color_h[v]]++;
      P.perm_h[i] = v;
      iperm[v] = i;
    }
    // ---- A~ = Pi^T A Pi, L = tril(A~) (diagonal last), U = L^T (diagonal first) ----
    std::vector<int64_t> arp(n + 1, 0), lrp(n + 1, 0), urp(n + 1, 0);
    std::vector<int> acol;
    std::vector<double> aval;
    acol.reserve(nnz);
    aval.reserve(nnz);
    std::vector<std::pair<int, double>> row;
    std::vector<int> lcol;
    std::vector<double> lini;
    std::vector<int64_t> diag_pos(n);
    lcol.reserve(nnz / 2 + n);
    lini.reserve(nnz / 2 + n);
    acol.clear();
    aval.clear();
    for (int64_t i = 0; i < n; ++i) {
      const int64_t v = P.perm_h[i];
      row.clear();
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) row.emplace_back((int)iperm[col[e]], val[e]);
      std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
      size_t k = 0;  // repeated columns are summed
      for (size_t t = 0; t < row.size(); ++t) {
        if (k && row[k - 1].first == row[t].first)
          row[k - 1].second += row[t].second;
        else
          row[k++] = row[t];
      }
      row.resize(k);
      double dg = 0.0;
      for (const auto& pr : row) {
        acol.push_back(pr.first);
        aval.push_back(pr.second);
        if (pr.first < i) {
          lcol.push_back(pr.first);
          lini.push_back(pr.second);
        } else if (pr.first == i) {
          dg += pr.second;
        }
      }
      lcol.push_back((int)i);
      lini.push_back(dg);
      diag_pos[i] = (int64_t)lcol.size() - 1;
      lrp[i + 1] = (int64_t)lcol.size();
      arp[i + 1] = (int64_t)acol.size();
    }
    const int64_t nnzA = (int64_t)acol.size();
    const int64_t nnzL = (int64_t)lcol.size();
    // U rows: diagonal, then the L entries (j, i) with j > i in ascending j
    std::vector<int64_t> ucount(n, 1);
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = lrp[j]; p < lrp[j + 1] - 1; ++p) ucount[lcol[p]] += 1;
    for (int64_t i = 0; i < n; ++i) urp[i + 1] = urp[i] + ucount[i];
    std::vector<int> ucol(nnzL);
    std::vector<int64_t> umap(nnzL), ufill(urp.begin(), urp.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
      ucol[ufill[i]] = (int)i;
      umap[ufill[i]++] = diag_pos[i];
    }
    for (int64_t j = 0; j < n; ++j)
      for (int64_t p = lrp[j]; p < lrp[j + 1] - 1; ++p) {
        const int i = lcol[p];
        ucol[ufill[i]] = (int)j;
        umap[ufill[i]++] = p;
      }
    // ---- upload (col / val arrays padded for the TMA-staged SpMM) ----
    auto up = [&](const void* src, size_t bytes, size_t alloc) {
      void* d = dalloc_own(h, alloc);
      ck(cudaMemsetAsync(d, 0, alloc, s), "memset");
      if (bytes) ck(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, s), "h2d");
      return d;
    };
    P.nnzA = nnzA;
    P.nnzL = nnzL;
    P.perm = (int64_t*)up(P.perm_h.data(), sizeof(int64_t) * n, sizeof(int64_t) * n);
    P.arp = (int64_t*)up(arp.data(), sizeof(int64_t) * (n + 1), sizeof(int64_t) * (n + 1));
    P.acol = (int*)up(acol.data(), sizeof(int) * nnzA, sizeof(int) * csr_entries(nnzA));
    P.aval = (double*)up(aval.data(), sizeof(double) * nnzA, sizeof(double) * csr_entries(nnzA));
    P.lrp = (int64_t*)up(lrp.data(), sizeof(int64_t) * (n + 1), sizeof(int64_t) * (n + 1));
    P.lcol = (int*)up(lcol.data(), sizeof(int) * nnzL, sizeof(int) * csr_entries(nnzL));
    P.lval = (double*)up(nullptr, 0, sizeof(double) * csr_entries(nnzL));
    P.urp = (int64_t*)up(urp.data(), sizeof(int64_t) * (n + 1), sizeof(int64_t) * (n + 1));
    P.ucol = (int*)up(ucol.data(), sizeof(int) * nnzL, sizeof(int) * csr_entries(nnzL));
    P.umap = (int64_t*)up(umap.data(), sizeof(int64_t) * nnzL, sizeof(int64_t) * std::max<int64_t>(nnzL, 1));
    P.uval = (double*)up(nullptr, 0, sizeof(double) * csr_entries(nnzL));
    ck(cudaStreamSynchronize(s), "sync");  // the host vectors above are read by the copies
    P.linit = std::move(lini);
    P.built = true;
  }
  if (P.alpha != alpha) {
    // values: tril(A~) with the compensated diagonal, then IC(0) colour by colour
    std::vector<double> v0 = P.linit;
    std::vector<int64_t> lrp(n + 1);
    ck(cudaMemcpyAsync(lrp.data(), P.lrp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s), "d2h");
    ck(cudaStreamSynchronize(s), "sync");
    for (int64_t i = 0; i < n; ++i) v0[lrp[i + 1] - 1] *= (1.0 + alpha);
    Buf fail(h, 256);
    ck(cudaMemsetAsync(fail.p, 0, 256, s), "memset");
    ck(cudaMemcpyAsync(P.lval, v0.data(), sizeof(double) * P.nnzL, cudaMemcpyHostToDevice, s), "h2d");
    for (int c = 0; c < P.ncolors; ++c) {
      ic0_rows(P.lrp, P.lcol, P.lval, P.cstart[c], P.cstart[c + 1], fail.as<unsigned>(), s);
      h->launches += 1;
    }
    gather_vals(P.lval, P.umap, P.uval, P.nnzL, s);
    h->launches += 1;
    unsigned f = 0;
    ck(cudaMemcpyAsync(&f, fail.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
    ck(cudaStreamSynchronize(s), "sync");
    ck_launch("ic0");
    P.alpha = alpha;
    if (P.aval32) {  // FP32 copies follow the new factor
      convert_d2f(P.lval, P.lval32, P.nnzL, s);
      convert_d2f(P.uval, P.uval32, P.nnzL, s);
    }
    if (f) {
      P.alpha = -1.0;
      throw Fail{NS_ERR_NUMERICAL, "IC(0) met a non-positive pivot: raise precond_shift"};
    }
  }
}

// Inner preconditioner of the normal form (Sec. 4.4.1): P_L = diag(A A^T), applied as
// the row scaling S = P_L^-1/2 (the pseudo-inverse for zero rows), so that
// A^T P_L^-1 A = (S A)^T (S A).  Its null space is A's.
void build_inner(ns_handle* h) {
  auto& I = h->inner;
  if (I.built) return;
  cudaStream_t s = h->stream;
  const int64_t m = h->m, n = h->n, nnz = h->nnz;
  I.s = (double*)dalloc_own(h, sizeof(double) * std::max<int64_t>(m, 1));
  I.val = (double*)dalloc_own(h, sizeof(double) * csr_entries(nnz));
  I.val_t = (double*)dalloc_own(h, sizeof(double) * csr_entries(nnz));
  ck(cudaMemsetAsync(I.val, 0, sizeof(double) * csr_entries(nnz), s), "memset");
  ck(cudaMemsetAsync(I.val_t, 0, sizeof(double) * csr_entries(nnz), s), "memset");
  inner_scaling(h->rowptr, h->val, m, h->col_t, h->val_t, nnz, I.s, I.val, I.val_t, s);
  Buf rp(h, sizeof(double) * (size_t)kMaxBlocks * 64 + 256), sm(h, 4096);
  ck(cudaMemsetAsync(sm.p, 0, 4096, s), "memset");
  Red red;
  red.part = rp.as<double>();
  red.ticket = reinterpret_cast<unsigned*>(sm.as<char>() + 1024);
  double* norms = reinterpret_cast<double*>(sm.as<char>() + 2048);
  csr_max_abs_row_sum(h->rowptr, I.val, m, norms, red, s);
  csr_max_abs_row_sum(h->rowptr_t, I.val_t, n, norms + 1, red, s);
  h->launches += 5;
  double nr[2] = {0.0, 0.0};
  ck(cudaMemcpyAsync(nr, norms, sizeof(nr), cudaMemcpyDeviceToHost, s), "d2h");
  ck(cudaStreamSynchronize(s), "sync");
  ck_launch("inner preconditioner");
  I.normAinf = nr[0];
  I.normA1 = nr[1];
  I.built = true;
}

void ensure_fp32(ns_handle* h) {
  // FP32 copies of A's values (already present when A came in as FP32), A^T's values and D
  if (!h->val32) {
    h->val32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(h->nnz));
    convert_d2f(h->val, h->val32, h->nnz, h->stream);
  }
  if (h->mode == NS_MODE_NORMAL && !h->val_t32) {
    h->val_t32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(h->nnz));
    convert_d2f(h->val_t, h->val_t32, h->nnz, h->stream);
  }
  if (!h->D32) {
    h->D32 = (float*)dalloc_own(h, sizeof(float) * (size_t)h->n);
    convert_d2f(h->D64, h->D32, h->n, h->stream);
  }
  auto& I = h->inner;
  if (I.built && !I.val32) {
    I.val32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(h->nnz));
    I.val_t32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(h->nnz));
    convert_d2f(I.val, I.val32, h->nnz, h->stream);
    convert_d2f(I.val_t, I.val_t32, h->nnz, h->stream);
  }
  auto& P = h->pc;
  if (P.built && !P.aval32) {
    P.aval32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(P.nnzA));
    P.lval32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(P.nnzL));
    P.uval32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(P.nnzL));
    convert_d2f(P.aval, P.aval32, P.nnzA, h->stream);
    convert_d2f(P.lval, P.lval32, P.nnzL, h->stream);
    convert_d2f(P.uval, P.uval32, P.nnzL, h->stream);
  }
  for (ns_handle::Sell* sl : {&h->sell_A, &h->sell_At})
    if (sl->sval && !sl->sval32) {
      sl->sval32 = (float*)dalloc_own(h, sizeof(float) * (size_t)sl->entries);
      convert_d2f(sl->sval, sl->sval32, sl->entries, h->stream);
    }
  ck_launch("fp32 copies");
}

template <typename T>
Csr<T> csr_A(ns_handle* h) {
  Csr<T> c;
  c.rowptr = h->rowptr;
  c.col = h->col;
  c.val = Prec<T>::val(h);
  c.nrows = h->m;
  c.ncols = h->n;
  c.nnz = h->nnz;
  c.V = choose_lanes(h->m, h->nnz);
  c.sptr = h->sell_A.sptr;
  c.scol = h->sell_A.scol;
  c.sval = Prec<T>::sval(h->sell_A);
  if (!c.sval) c.sptr = nullptr;
  return c;
}
template <typename T>
Csr<T> csr_At(ns_handle* h) {
  Csr<T> c;
  c.rowptr = h->rowptr_t;
  c.col = h->col_t;
  c.val = Prec<T>::val_t(h);
  c.nrows = h->n;
  c.ncols = h->m;
  c.nnz = h->nnz;
  c.V = choose_lanes(h->n, h->nnz);
  c.sptr = h->sell_At.sptr;
  c.scol = h->sell_At.scol;
  c.sval = Prec<T>::sval(h->sell_At);
  if (!c.sval) c.sptr = nullptr;
  return c;
}

template <typename T>
const T* pc_vals(const double* v64, const float* v32);
template <>
const double* pc_vals<double>(const double* v64, const float*) {
  return v64;
}
template <>
const float* pc_vals<float>(const double*, const float* v32) {
  return v32;
}

// ---------------------------------------------------------------------------
// the solver
// ---------------------------------------------------------------------------
template <typename T, int D>
struct Solver {
  ns_handle* h;
  cudaStream_t s;
  int64_t n, m;
  int R, nb;
  double eps, tol_eff, normB, u, u_d, u_ro, bd_tol;
  double ud_per_normB = 0.0;  // u_d = ud_per_normB * ||B|| (Eq. defmprd with readings M1, M4)
  ns_opts o;
  Csr<T> A, At;  // with the outer preconditioner, A is A~ = Pi^T A Pi
  const T* Dv;
  const ns_handle::Pc* pc = nullptr;  // outer preconditioner (Sec. 4.4.2) or null
  Buf tbuf;                           // L^-T x of the preconditioned product
  // buffers
  Buf zb[2], qp, ybuf, xbuf, lnew, cbuf, dpart, redpart, small, pin, umma_img;
  unsigned* umma_err = nullptr;  // set by the tensor-core restart product when a bounded wait gave up
  T* Z[2];
  int cur = 0;
  int cap = 0, nlock = 0;
  Red red;
  // small device arrays
  double *Xi, *Gam, *nXi, *nGam, *sminGam, *Theta, *F, *nTheta, *nF, *Tm, *theta, *VZ, *resid, *syw, *R1, *R2,
      *Cacc, *gdiag, *wz, *wx, *xtheta, *xrho;
  int* sel;
  unsigned* flags;
  long long* counters;
  unsigned* flags_h;
  double* pin_d;  // pinned host scratch
  std::vector<double> xtheta_h, xrho_h;
  // statistics
  int64_t matvecs = 0, restarts = 0, lock_events = 0, ghosts = 0, breakdowns = 0;
  double theta_max = 0.0;
  std::vector<std::pair<int64_t, int>> events;
  long long& launches;

  // from: the checkpoint a resumed solve continues (its SpMM schedules replace the timing)
  Solver(ns_handle* hh, int R_, double tol, const ns_opts& oo, const ns_checkpoint_info* from = nullptr)
      : h(hh), s(hh->stream), n(hh->n), m(hh->m), R(R_), nb(R_ / D), o(oo), launches(hh->launches) {
    eps = o.eps;
    const bool mixed = std::is_same<T, float>::value;
    tol_eff = mixed ? std::max(tol, o.lock_tol_mixed) : tol;
    normB = (h->mode == NS_MODE_NORMAL ? h->normA1 * h->normAinf : h->normAinf) + eps;
    u = Unit<T>::u;
    if (!mixed) {
      ud_per_normB = D * std::sqrt((double)n) * u;  // Eq. (defmprd)
    } else {
      // FP32 reading M1: the inner-product lengths of one application of B are the row
      // lengths of its stages, not n (sparse B; sqrt(n) u_32 would exceed sqrt(u_32));
      // the two stages of A^T (A x) add their errors
      const double k = (h->mode == NS_MODE_NORMAL)
                           ? std::sqrt((double)std::max<int64_t>(h->maxrow_A, 1)) +
                                 std::sqrt((double)std::max<int64_t>(h->maxrow_At, 1))
                           : std::sqrt((double)std::max<int64_t>(h->maxrow_A, 1));
      ud_per_normB = D * k * u;
    }
    u_d = ud_per_normB * normB;
    u_ro = std::sqrt(u);
    bd_tol = 100.0 * u_d;
    A = csr_A<T>(h);
    if (h->mode == NS_MODE_NORMAL) At = csr_At<T>(h);
    if (o.precond == 2) {  // B_L = (S A)^T (S A) + eps D (Sec. 4.4.1); the CSR schedules only
      const auto& I = h->inner;
      A.val = pc_vals<T>(I.val, I.val32);
      At.val = pc_vals<T>(I.val_t, I.val_t32);
      A.sptr = At.sptr = nullptr;
      normB = I.normA1 * I.normAinf + eps;
      u_d = ud_per_normB * normB;
      bd_tol = 100.0 * u_d;
    }
    if (o.precond == 1) {
      pc = &h->pc;
      A = Csr<T>{};
      A.rowptr = pc->arp;
      A.col = pc->acol;
      A.val = pc_vals<T>(pc->aval, pc->aval32);
      A.nrows = A.ncols = n;
      A.nnz = pc->nnzA;
      A.V = choose_lanes(n, pc->nnzA);
    }
    Dv = Prec<T>::D(h);
    const size_t zbytes = sizeof(T) * (size_t)n * (R + D);
    zb[0] = Buf(h, zbytes);
    zb[1] = Buf(h, zbytes);
    Z[0] = zb[0].as<T>();
    Z[1] = zb[1].as<T>();
    qp = Buf(h, sizeof(T) * (size_t)n * D);
    if (h->mode == NS_MODE_NORMAL || pc) ybuf = Buf(h, sizeof(T) * (size_t)m * D);
    if (pc) tbuf = Buf(h, sizeof(T) * (size_t)n * D);
    lnew = Buf(h, sizeof(T) * (size_t)n * R);
    cap = (int)std::min<int64_t>(n, std::max(64, R));
    xbuf = Buf(h, sizeof(T) * (size_t)n * cap);
    alloc_proj();
    redpart = Buf(h, sizeof(double) * (size_t)kMaxBlocks * 64 + 256);
    red.part = redpart.as<double>();
    // small arena
    const size_t nbp = nb + 1;
    size_t off = 0;
    auto take = [&](size_t cnt) {
      const size_t o2 = off;
      off += (cnt + 7) & ~(size_t)7;
      return o2;
    };
    const size_t oXi = take(nbp * D * D), oGam = take(nbp * D * D), onXi = take(nbp), onGam = take(nbp),
                 osmin = take(nbp), oTheta = take(R), oF = take((size_t)D * R), onTheta = take(nbp), onF = take(nbp),
                 oTm = take((size_t)R * R), otheta = take(R), oVZ = take((size_t)R * R), oresid = take(R),
                 osyw = take(syev_work_doubles(R)), oR1 = take(64), oR2 = take(64), oC = take(64),
                 ogd = take(8), owz = take(3 * nbp), osel = take(R), oflags = take(8), ocnt = take(8);
    small = Buf(h, sizeof(double) * off);
    double* b = small.as<double>();
    Xi = b + oXi;
    Gam = b + oGam;
    nXi = b + onXi;
    nGam = b + onGam;
    sminGam = b + osmin;
    Theta = b + oTheta;
    F = b + oF;
    nTheta = b + onTheta;
    nF = b + onF;
    Tm = b + oTm;
    theta = b + otheta;
    VZ = b + oVZ;
    resid = b + oresid;
    syw = b + osyw;
    R1 = b + oR1;
    R2 = b + oR2;
    Cacc = b + oC;
    gdiag = b + ogd;
    wz = b + owz;
    sel = reinterpret_cast<int*>(b + osel);
    flags = reinterpret_cast<unsigned*>(b + oflags);
    red.ticket = flags + 4;
    umma_err = flags + 8;
    counters = reinterpret_cast<long long*>(b + ocnt);
    ck(cudaMemsetAsync(small.p, 0, sizeof(double) * off, s), "memset");
    alloc_locked_meta();
    if (std::is_same<T, float>::value && gemm_kind() != NS_GEMM_CUDA_CORES)
      umma_img = Buf(h, restart_umma_image_bytes(R, std::min(R, 256), 3));
    if (std::is_same<T, double>::value && gemm_kind() == NS_GEMM_TC_EXACT)
      umma_img = Buf(h, restart_ozaki_scratch_bytes(n, R, R));
    ck(cudaMallocHost(&pin_d, sizeof(double) * (2 * (size_t)R + 64)), "cudaMallocHost");
    flags_h = reinterpret_cast<unsigned*>(pin_d + 2 * R + 32);
    if (from) {  // the schedules the checkpointed iteration ran with
      A.V = checked_schedule(A, from->spmm_A, h->mode == NS_MODE_NORMAL || pc);
      if (h->mode == NS_MODE_NORMAL) At.V = checked_schedule(At, from->spmm_At, false);
    } else if (o.spmm_schedule > 0) {
      A.V = fixed_schedule(A, o.spmm_schedule);
      if (h->mode == NS_MODE_NORMAL) At.V = fixed_schedule(At, o.spmm_schedule);
    } else {
      // SpMM schedule: lanes per row tuned on this matrix (operands: the basis buffers)
      ck(cudaMemsetAsync(Z[1], 0, zbytes, s), "memset");
      if (pc) {  // A~ is applied by the plain SpMM between the two triangular solves
        A.V = tune_lanes<T, D>(A, Z[1], ybuf.as<T>(), s);
      } else if (h->mode == NS_MODE_SPD) {
        A.V = tune_lanczos(A, Z[1]);
      } else {
        A.V = tune_lanes<T, D>(A, Z[1], ybuf.as<T>(), s);
        ck(cudaMemsetAsync(ybuf.p, 0, sizeof(T) * (size_t)m * D, s), "memset");
        At.V = tune_lanczos(At, ybuf.as<T>());
      }
      launches += (h->mode == NS_MODE_SPD ? 15 : 30);
    }
    if (getenv("NS_DEBUG")) fprintf(stderr, "[ns] lanes per row: A %d, A^T %d\n", A.V, At.V);
    ck_launch("tune");
  }
  static int fixed_schedule(const Csr<T>& M, int sched) { return (sched == kSchedSell && !M.sptr) ? 8 : sched; }
  // a schedule read from a checkpoint: one the kernels of this operand support
  static int checked_schedule(const Csr<T>& M, int64_t v, bool plain) {
    const bool ok = v == 1 || v == 2 || v == 4 || v == 8 || v == kSchedTma || (v == kSchedSell && M.sptr) ||
                    (plain && v == 16);
    if (!ok) throw Fail{NS_ERR_INVALID_ARG, "checkpoint SpMM schedule not usable on this handle"};
    return (int)v;
  }
  ~Solver() {
    if (pin_d) cudaFreeHost(pin_d);
  }

  Buf wxbuf;
  // W rows of the locked set (3 rotating columns) + their Ritz values and residuals
  void alloc_locked_meta(int oldcap = 0) {
    Buf nb2(h, sizeof(double) * (size_t)(5 * (size_t)cap + 64));
    ck(cudaMemsetAsync(nb2.p, 0, nb2.bytes, s), "memset");
    if (wxbuf.p && nlock)
      for (int c = 0; c < 3; ++c)
        ck(cudaMemcpyAsync(nb2.as<double>() + (size_t)c * cap, wxbuf.as<double>() + (size_t)c * oldcap,
                           sizeof(double) * nlock, cudaMemcpyDeviceToDevice, s),
           "copy");
    wxbuf = std::move(nb2);
    wx = wxbuf.as<double>();
    xtheta = wx + 3 * (size_t)cap;
    xrho = xtheta + cap;
    if (nlock) {
      ck(cudaMemcpyAsync(xtheta, xtheta_h.data(), sizeof(double) * nlock, cudaMemcpyHostToDevice, s), "h2d");
      ck(cudaMemcpyAsync(xrho, xrho_h.data(), sizeof(double) * nlock, cudaMemcpyHostToDevice, s), "h2d");
    }
  }

  void alloc_proj() {
    // panels up to 2D = 16 wide (the merged [Q_j | Q_j+1] reorthogonalization at d = 8)
    const int K = cap + R + D;
    cbuf = Buf(h, sizeof(double) * (size_t)K * 16);
    const int nch = ceil_div(std::max<int64_t>(n, 1), kDotsMinChunk);  // the auto chunking's smallest chunk
    dpart = Buf(h, sizeof(double) * (size_t)nch * K * 16);
  }

  void grow_locked(int need) {
    if (need <= cap) return;
    int nc = cap;
    while (nc < need) nc *= 2;
    nc = (int)std::min<int64_t>(nc, n);
    Buf nx(h, sizeof(T) * (size_t)n * nc);
    if (nlock) ck(cudaMemcpyAsync(nx.p, xbuf.p, sizeof(T) * (size_t)n * nlock, cudaMemcpyDeviceToDevice, s), "copy");
    ck(cudaStreamSynchronize(s), "sync");
    xbuf = std::move(nx);
    const int oldcap = cap;
    cap = nc;
    alloc_proj();
    alloc_locked_meta(oldcap);
    ck(cudaStreamSynchronize(s), "sync");
  }

  // lanes per row of the fused Lanczos SpMM, timed on this matrix (CUDA events)
  int tune_lanczos(Csr<T> M, const T* v) {
    StepOps<T> op;
    op.x = Z[1];
    op.Dv = Dv;
    op.eps = eps;
    op.out = qp.as<T>();
    op.xi = Xi + (size_t)nb * D * D;  // spare slot
    op.xi_norm = nXi + nb;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = M.V;
    float best_ms = 1e30f;
    for (int V : {kSchedSell, kSchedTma, 1, 2, 4, 8}) {  // sliced ELLPACK, TMA-staged, 1..8 lanes per row
      if (V == kSchedSell && !M.sptr) continue;
      M.V = V;
      spmm_lanczos<T, D>(M, v, op, red, s);
      cudaEventRecord(e0, s);
      spmm_lanczos<T, D>(M, v, op, red, s);
      spmm_lanczos<T, D>(M, v, op, red, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = V;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
  }

  // kernel of the thick-restart product (Sec. 4.1): tensor cores on the mixed path
  int gemm_kind() const {
    if (!std::is_same<T, float>::value) {
      if (o.gemm == NS_GEMM_DEFAULT) return restart_ozaki_supported(R, 1) ? NS_GEMM_TC_EXACT : NS_GEMM_CUDA_CORES;
      return o.gemm;
    }
    return o.gemm == NS_GEMM_DEFAULT ? NS_GEMM_TC3 : o.gemm;
  }
  // [Lnew | Znext] = Z V_Z(:, sel(0:nsel)), the first nl outputs to Lnew
  void restart_product(int nsel, int nl, T* Lnew, T* Znext) {
    const int g = gemm_kind();
    if constexpr (std::is_same<T, float>::value) {
      if ((g == NS_GEMM_TC2 || g == NS_GEMM_TC3) && restart_umma_supported(R, nsel)) {
        ck(restart_gemm_umma(Z[cur], D, R, VZ, sel, nsel, nl, n, Lnew, Znext, umma_img.p, umma_err,
                             g == NS_GEMM_TC2 ? 2 : 3, s),
           "restart_gemm_umma");
        launches += 2;
        return;
      }
    }
    if constexpr (std::is_same<T, double>::value) {
      if (g == NS_GEMM_TC_EXACT && restart_ozaki_supported(R, nsel)) {
        ck(restart_gemm_ozaki(Z[cur], D, R, VZ, sel, nsel, nl, n, Lnew, Znext, umma_img.p, umma_err, s),
           "restart_gemm_ozaki");
        launches += 3;
        return;
      }
    }
    ck(restart_gemm<T>(Z[cur], D, R, VZ, sel, nsel, nl, n, Lnew, Znext, s), "restart_gemm shared-memory limit");
    launches += 1;
  }

  T* X() const { return xbuf.as<T>(); }
  T* blk(int which, int b) const { return Z[which] + (size_t)b * n * D; }

  void sync() {
    ck(cudaStreamSynchronize(s), "stream sync");
    h->prof.flush();
  }

  unsigned read_flags() {
    ck(cudaMemcpyAsync(flags_h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h flags");
    sync();
    return *flags_h;
  }
  void clear_flags() { ck(cudaMemsetAsync(flags, 0, sizeof(unsigned), s), "memset flags"); }

  // ---- B applied to one block with the fused recurrence epilogue ----
  void apply_step(const T* x, const T* qprev, const double* gprev, double* xi, double* xi_norm) {
    StepOps<T> op;
    op.x = x;
    op.Dv = Dv;
    op.eps = eps;
    op.qprev = qprev;
    op.gprev = gprev;
    op.out = qp.as<T>();
    op.xi = xi;
    op.xi_norm = xi_norm;
    const double sv = sizeof(T);
    double by = (double)h->nnz * (4 + sv) + (n + 1) * 8.0 + n * (3.0 * D + 1.0) * sv + (qprev ? n * D * sv : 0.0);
    double fl = 2.0 * h->nnz * D + 2.0 * n * D + 2.0 * n * D * D * (qprev ? 2 : 1);
    if (h->mode == NS_MODE_NORMAL) {
      by += (double)h->nnz * (4 + sv) + (m + 1) * 8.0 + 2.0 * m * D * sv;
      fl += 2.0 * h->nnz * D;
    }
    if (pc) {  // two triangular solves of L, nnz(L) entries and n rows each
      by += 2.0 * pc->nnzL * (4 + sv) + 2.0 * (n + 1) * 8.0 + 4.0 * n * D * sv;
      fl += 4.0 * pc->nnzL * D;
    }
    PScope ps(&h->prof, P_APPLY, by, fl);
    if (pc) {  // B_R x = L^-1 A~ L^-T x + eps D x (Sec. 4.4.2)
      T* t = tbuf.as<T>();
      T* u = ybuf.as<T>();
      const int nc = pc->ncolors;
      trsv_colors<T, D>(pc->urp, pc->ucol, pc_vals<T>(pc->uval, pc->uval32), pc->cstart.data(), nc, false, x, t, s);
      spmm_plain<T, D>(A, t, u, s);
      trsv_colors<T, D>(pc->lrp, pc->lcol, pc_vals<T>(pc->lval, pc->lval32), pc->cstart.data(), nc, true, u, u, s);
      lanczos_epilogue<T, D>(u, n, op, red, s);
      launches += 2 * nc + 2;
    } else if (h->mode == NS_MODE_SPD) {
      spmm_lanczos<T, D>(A, x, op, red, s);
      launches += 1;
    } else {
      spmm_plain<T, D>(A, x, ybuf.as<T>(), s);
      spmm_lanczos<T, D>(At, ybuf.as<T>(), op, red, s);
      launches += 2;
    }
    matvecs += D;
  }

  // ---- CGS2 of a panel of width W against [X(0:kx) | Z blocks 0..nzb-1 of buffer zw] ----
  template <int W>
  void project(T* Wp, int64_t ldw, int kx, int zw, int nzb, bool gram, double* Rout, double* gd) {
    project2<W>(Wp, nullptr, ldw, kx, zw, nzb, gram, Rout, gd, 2);
  }

  // passes = 2: CGS2; passes = 1: one classical Gram-Schmidt pass (enough for the
  // partial reorthogonalization of semi-orthogonal blocks).  Wp2: second panel.
  template <int W>
  void project2(T* Wp, T* Wp2, int64_t ldw, int kx, int zw, int nzb, bool gram, double* Rout, double* gd,
                int passes) {
    VParts<T> V;
    V.X = X();
    V.kx = kx;
    V.Z = Z[zw];
    V.kz = nzb * D;
    V.p = D;
    V.df = (std::is_same<T, double>::value && o.fp64_products == 0) ? 1 : 0;
    if (V.kx + V.kz == 0) {
      if (gram && !Wp2) {
        gram_chol<T, W>(Wp, ldw, W, n, Rout, gd, flags, red, s);
        launches += 1;
      }
      return;
    }
    if ((size_t)(V.kx + V.kz) * W * sizeof(T) > 190 * 1024)
      throw Fail{NS_ERR_INVALID_ARG, "projection basis too wide for one pass"};
    const double K = V.kx + V.kz, sv = sizeof(T);
    PScope ps(&h->prof, P_PROJ, passes * (2.0 * K * n * sv + 3.0 * n * W * sv), 4.0 * passes * K * n * W);
    for (int pass = 0; pass < passes; ++pass) {
      proj_dots<T, W>(V, Wp, Wp2, ldw, n, cbuf.as<double>(), dpart.as<double>(), s, kDotsAutoChunks);
      ck((proj_update<T, W>(V, cbuf.as<double>(), Wp, Wp2, ldw, n, (pass == passes - 1 && gram) ? 1 : 0, Rout, gd,
                            flags, red, s)),
         "proj_update shared-memory limit");
      launches += 3;
    }
  }

  // CholQR2 of a block (in place); pass-1 factor R1 already computed into r1.
  // Leaves the full factor R = R2 R1 in (R1, R2).
  template <int W>
  void cholqr_finish(T* Wp, int64_t ldw, double* r1, double* r2) {
    scale_gram<T, W>(Wp, ldw, Wp, ldw, r1, n, r2, flags, red, s, W);
    scale_gram<T, W>(Wp, ldw, Wp, ldw, r2, n, nullptr, flags, red, s, W);
    launches += 2;
  }

  OmegaArgs omega_args(int j, int r0) {
    OmegaArgs a;
    a.j = j;
    a.r0 = r0;
    a.nb = nb;
    a.d = D;
    a.nlock = nlock;
    a.u_d = u_d;
    a.u_ro = u_ro;
    a.R1 = R1;
    a.R2 = R2;
    a.Gam = Gam;
    a.nGam = nGam;
    a.sminGam = sminGam;
    a.nXi = nXi;
    a.nTheta = nTheta;
    a.nF = nF;
    a.xtheta = xtheta;
    a.xrho = xrho;
    a.wz = wz;
    a.wx = wx;
    a.cap = cap;
    a.bd_tol = bd_tol;
    a.flags = flags;
    a.counters = counters;
    a.trace = trace_dev;
    return a;
  }

  // replacement of a broken-down block (reading R12): random block orthogonalized
  // against [X, Z blocks 0..b-1] of the current buffer
  void replace_block(int which, int b) {
    breakdowns += 1;
    T* q = blk(which, b);
    rng_gauss<T>(h->seed, (uint32_t)(2 + breakdowns - 1), q, n * D, s);
    launches += 1;
    clear_flags();
    project<D>(q, D, nlock, which, b, true, R1, nullptr);
    cholqr_finish<D>(q, D, R1, R2);
    clear_flags();
  }

  void orthonormal_start() {
    T* q0 = blk(cur, 0);
    rng_gauss<T>(h->seed, 1u, q0, n * D, s);  // Alg. 2 (its Gaussian start block)
    launches += 1;
    gram_chol<T, D>(q0, D, D, n, R1, nullptr, flags, red, s);
    launches += 1;
    cholqr_finish<D>(q0, D, R1, R2);  // Alg. 2 (its orthonormalized start block)
    if (read_flags() & 1u) {
      clear_flags();
      replace_block(cur, 0);
    }
  }

  // Alg. 2: the first step of a cycle
  void first_step(int r0) {
    T* q = blk(cur, r0);
    apply_step(q, nullptr, nullptr, Xi + (size_t)r0 * D * D, nXi + r0);
    project<D>(qp.as<T>(), D, nlock, cur, r0 + 1, true, R1, nullptr);
    T* qn = blk(cur, r0 + 1);
    if constexpr (D == 1) {  // a single vector: one normalization (see inner_step)
      scale_gram<T, D>(qp.as<T>(), D, qn, D, R1, n, nullptr, flags, red, s, D);
      OmegaArgs a = omega_args(r0, r0);
      a.R2 = nullptr;
      gamma_store(a, s);
      launches += 2;
    } else {
      scale_gram<T, D>(qp.as<T>(), D, qn, D, R1, n, R2, flags, red, s, D);
      OmegaArgs a = omega_args(r0, r0);
      gamma_store(a, s);
      scale_gram<T, D>(qn, D, qn, D, R2, n, nullptr, flags, red, s, D);
      launches += 3;
    }
    if (read_flags() & 1u) {
      clear_flags();
      replace_block(cur, r0 + 1);
      set_gamma_zero_host(r0);
    }
    omega_init(wz, wx, nb, cap, r0, nlock, u_d, s);
    launches += 2;
  }

  void set_gamma_zero_host(int j) {
    ck(cudaMemsetAsync(Gam + (size_t)j * D * D, 0, sizeof(double) * D * D, s), "memset");
    ck(cudaMemsetAsync(nGam + j, 0, sizeof(double), s), "memset");
    ck(cudaMemsetAsync(sminGam + j, 0, sizeof(double), s), "memset");
  }

  // Alg. 2 (the block recurrence of a cycle) for block j (r0 < j < nb)
  void inner_step(int j, int r0) {
    T* q = blk(cur, j);
    T* qn = blk(cur, j + 1);
    apply_step(q, blk(cur, j - 1), Gam + (size_t)(j - 1) * D * D, Xi + (size_t)j * D * D, nXi + j);
    if constexpr (D == 1) {
      // a single vector: Q_{j+1} = Q' / ||Q'|| in one pass.  The second CholQR pass of a
      // block (below) would re-normalize an already unit vector, an O(u) correction.
      PScope ps(&h->prof, P_REC, 5.0 * n * sizeof(T), 6.0 * n);
      axpy_gram<T, D>(qp.as<T>(), q, Xi + (size_t)j * D * D, n, R1, flags, red, s);
      scale_gram<T, D>(qp.as<T>(), D, qn, D, R1, n, nullptr, flags, red, s, D);
      OmegaArgs a = omega_args(j, r0);
      a.R2 = nullptr;  // Gamma_j = R1 = ||Q'||
      if (o.reorth == NS_REORTH_FULL) a.u_ro = -1.0;  // every column triggers
      step_finalize(a, s);
      launches += 3;
    } else {
      PScope ps(&h->prof, P_REC, 7.0 * n * D * sizeof(T), 8.0 * n * D * D);
      axpy_gram<T, D>(qp.as<T>(), q, Xi + (size_t)j * D * D, n, R1, flags, red, s);
      scale_gram<T, D>(qp.as<T>(), D, qn, D, R1, n, R2, flags, red, s, D);
      OmegaArgs a = omega_args(j, r0);
      if (o.reorth == NS_REORTH_FULL) a.u_ro = -1.0;  // every column triggers
      step_finalize(a, s);
      scale_gram<T, D>(qn, D, qn, D, R2, n, nullptr, flags, red, s, D);
      launches += 4;
    }
    const unsigned f = read_flags();
    if (f) clear_flags();
    if (f & 1u) {  // breakdown: fresh block, coupling set to zero
      replace_block(cur, j + 1);
      omega_column(wz, wx, nb, cap, j + 1, nlock, u_d, s);
      launches += 1;
      return;
    }
    const bool tz = (f & 2u) != 0, tx = (f & 4u) != 0;
    if (tz || tx) {
      // Sec. 4.2: reorthogonalize Q_j and Q_{j+1} against [X, Z_{0..j-1}]; both are
      // semi-orthogonal to that basis, so one classical Gram-Schmidt pass over
      // [Q_j | Q_{j+1}] suffices (Q_{j+1} is locally orthogonal to Q_j already);
      // then each block is re-normalized by CholQR2.
      const int kx = tx ? nlock : 0;
      project2<2 * D>(q, qn, D, kx, cur, tz ? j : 0, false, nullptr, nullptr, 1);
      gram_chol<T, D>(q, D, D, n, R1, nullptr, flags, red, s);
      cholqr_finish<D>(q, D, R1, R2);
      gram_chol<T, D>(qn, D, D, n, R1, nullptr, flags, red, s);
      cholqr_finish<D>(qn, D, R1, R2);
      launches += 2;
      if (read_flags() & 1u) throw Fail{NS_ERR_NUMERICAL, "rank loss in reorthogonalization (numerical)"};
    }
  }

  void project_parts(T* q, int kx, int nzb) {
    project<D>(q, D, kx, cur, nzb, true, R1, nullptr);
    cholqr_finish<D>(q, D, R1, R2);
    if (read_flags() & 1u) throw Fail{NS_ERR_NUMERICAL, "rank loss in reorthogonalization (numerical)"};
  }

  // lock the new Ritz vectors stored in lnew (row-major, width nl); returns ghosts
  int lock_new(int nl, const std::vector<int>& cand, std::vector<char>& is_ghost) {
    T* L = lnew.as<T>();
    int c0 = 0, ng = 0;
    grow_locked(nlock + nl);
    while (c0 < nl) {
      const int left = nl - c0;
      const int w = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
      bool ok = lock_chunk(L + c0, nl, w, cand, c0, is_ghost);
      if (!ok) {  // ghost inside: lock the columns one by one
        for (int c = c0; c < c0 + w; ++c) {
          if (!lock_chunk(L + c, nl, 1, cand, c, is_ghost)) {
            is_ghost[c] = 1;
            ++ng;
          }
        }
      }
      c0 += w;
    }
    return ng;
  }

  template <int W>
  bool lock_chunk_w(T* P, int64_t ld, const std::vector<int>& cand, int c0) {
    clear_flags();
    project<W>(P, ld, nlock, cur, 0, true, R1, gdiag);
    double* gd = pin_d;
    ck(cudaMemcpyAsync(gd, gdiag, sizeof(double) * W, cudaMemcpyDeviceToHost, s), "d2h");
    const unsigned f = read_flags();
    for (int c = 0; c < W; ++c)
      if (!(gd[c] >= 0.25)) return false;  // mostly inside span(X): a ghost
    if (f & 1u) return false;
    cholqr_finish<W>(P, ld, R1, R2);
    if (read_flags() & 1u) return false;
    panel_to_cols<T>(P, ld, W, n, X(), nlock, s);
    launches += 1;
    for (int c = 0; c < W; ++c) {
      xtheta_h.push_back(pin_theta[cand[c0 + c]]);
      xrho_h.push_back(pin_res[cand[c0 + c]]);
    }
    ck(cudaMemcpyAsync(xtheta + nlock, xtheta_h.data() + nlock, sizeof(double) * W, cudaMemcpyHostToDevice, s), "h2d");
    ck(cudaMemcpyAsync(xrho + nlock, xrho_h.data() + nlock, sizeof(double) * W, cudaMemcpyHostToDevice, s), "h2d");
    nlock += W;
    return true;
  }

  bool lock_chunk(T* P, int64_t ld, int w, const std::vector<int>& cand, int c0, std::vector<char>& is_ghost) {
    (void)is_ghost;
    switch (w) {
      case 8: return lock_chunk_w<8>(P, ld, cand, c0);
      case 4: return lock_chunk_w<4>(P, ld, cand, c0);
      case 2: return lock_chunk_w<2>(P, ld, cand, c0);
      default: return lock_chunk_w<1>(P, ld, cand, c0);
    }
  }

  std::vector<double> pin_theta, pin_res;
  double* trace_dev = nullptr;  // optional W-column record (ns_trace_omega)

  // first cycle only (start block, then steps 1..nb-1 with their partial
  // reorthogonalization), for ns_trace_omega
  void run_first_cycle() {
    orthonormal_start();
    first_step(0);
    for (int j = 1; j < nb; ++j) inner_step(j, 0);
    sync();
  }
  bool debug = getenv("NS_DEBUG") != nullptr;
  std::chrono::steady_clock::time_point t_start = std::chrono::steady_clock::now();

  // ---- Alg. 2 (the thick restart) + locking + stopping rule; returns true to stop ----
  bool restart(int& k0) {
    const int r0 = k0 / D;
    {
      PScope ps(&h->prof, P_EIG, 8.0 * 4 * R * R, 9.0 * R * R * R);
      build_T(Theta, F, Xi, Gam, k0, D, R, Tm, s);
      syev(Tm, R, theta, VZ, syw, s);
      ritz_resid(Gam + (size_t)(nb - 1) * D * D, VZ, D, R, resid, s);
    }
    launches += 4;
    (void)r0;
    ck(cudaMemcpyAsync(pin_d, theta, sizeof(double) * R, cudaMemcpyDeviceToHost, s), "d2h");
    ck(cudaMemcpyAsync(pin_d + R, resid, sizeof(double) * R, cudaMemcpyDeviceToHost, s), "d2h");
    sync();
    pin_theta.assign(pin_d, pin_d + R);
    pin_res.assign(pin_d + R, pin_d + 2 * R);
    restarts += 1;
    theta_max = std::max(theta_max, pin_theta[R - 1]);
    // reading M4: once a cycle has run, ||B|| in u_d and in the lock tolerance is
    // min(R9 bound, 1.1 theta_max)
    const double normB_est = std::min(normB, 1.1 * theta_max);
    u_d = ud_per_normB * normB_est;
    bd_tol = 100.0 * u_d;
    // Ritz values counted as null (Remark cormain: below 3 eps); unperturbed (eps = 0, the
    // large-block variant of Sec. 5.3.2) the null Ritz values sit at rounding level: reading L1
    // counts theta <= tol ||B|| instead
    const double small_lim = eps > 0.0 ? 3.0 * eps : tol_eff * normB_est;
    auto small = [&](double th) { return eps > 0.0 ? th < small_lim : th <= small_lim; };
    std::vector<int> cand;
    int nsmall = 0;
    for (int i = 0; i < R; ++i) {
      if (small(pin_theta[i])) {
        ++nsmall;
        if (pin_res[i] <= tol_eff * normB_est) cand.push_back(i);
      }
    }
    std::vector<char> taken(R, 0), is_ghost(cand.size(), 0);
    int nlocked_now = 0;
    if (!cand.empty()) {
      ck(cudaMemcpyAsync(sel, cand.data(), sizeof(int) * cand.size(), cudaMemcpyHostToDevice, s), "h2d");
      {
        const double nc = (double)cand.size();
        PScope ps(&h->prof, P_GEMM, (double)n * (R + nc) * sizeof(T), 2.0 * n * R * nc);
        restart_product((int)cand.size(), (int)cand.size(), lnew.as<T>(), nullptr);
      }
      const int before = nlock;
      int ng = 0;
      {
        const double nc = (double)cand.size();
        PScope ps(&h->prof, P_LOCK, 4.0 * nlock * n * sizeof(T) * ((nc + 7) / 8) + 6.0 * n * nc * sizeof(T),
                  8.0 * nlock * n * nc + 8.0 * n * nc * 8, false);  // spans syncs: counted, not timed
        ng = lock_new((int)cand.size(), cand, is_ghost);
      }
      ghosts += ng;
      nlocked_now = nlock - before;
      if (nlocked_now > 0) {
        events.emplace_back(matvecs, nlocked_now);
        lock_events += 1;
      }
      for (int i : cand) taken[i] = 1;
    }
    const int n_unl = nsmall - (int)cand.size();
    std::vector<int> avail;
    for (int i = 0; i < R; ++i)
      if (!taken[i]) avail.push_back(i);
    int nk = D * ((n_unl + R) / (2 * D));
    nk = std::max(nk, D);
    nk = std::min(nk, R - 2 * D);
    nk = std::min(nk, D * ((int)avail.size() / D));
    // reading R7b: the retained set is capped at the unlocked small pairs (whole
    // blocks) when they fit in 3 dimK/4, else at dimK/2, so every cycle adds new
    // vectors; the most converged small pairs are kept first (any subset of Ritz
    // pairs keeps the Krylov-Schur decomposition exact)
    {
      const int half = std::max(D, D * (R / (2 * D)));
      const int want = D * ((n_unl + D - 1) / D);
      const int cap = (want > half && want <= D * ((3 * R / 4) / D)) ? want : half;
      nk = std::min(nk, std::max(D, cap));
    }
    {
      std::vector<int> sm, rest;
      for (int i : avail) (small(pin_theta[i]) ? sm : rest).push_back(i);
      std::stable_sort(sm.begin(), sm.end(), [&](int a, int b) { return pin_res[a] < pin_res[b]; });
      avail = sm;
      avail.insert(avail.end(), rest.begin(), rest.end());
    }
    const int other = 1 - cur;
    ck(cudaMemcpyAsync(sel, avail.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, s), "h2d");
    {
      PScope ps(&h->prof, P_GEMM, (double)n * (R + nk) * sizeof(T), 2.0 * n * R * nk);
      restart_product(nk, 0, nullptr, Z[other]);
    }
    // Alg. 2 (the re-orthogonalized next block): Q_{l+1} against [X, Z_new], moved to block nk/D of the new buffer
    T* qlast = blk(cur, nb);
    clear_flags();
    project<D>(qlast, D, nlock, other, nk / D, true, R1, nullptr);
    T* qn = blk(other, nk / D);
    scale_gram<T, D>(qlast, D, qn, D, R1, n, R2, flags, red, s, D);
    scale_gram<T, D>(qn, D, qn, D, R2, n, nullptr, flags, red, s, D);
    launches += 2;
    bool bd = (read_flags() & 1u) != 0;
    if (bd) {
      clear_flags();
      replace_block(other, nk / D);
      ck(cudaMemsetAsync(Cacc, 0, sizeof(double) * 64, s), "memset");
    } else {
      mat2(R2, R1, Cacc);  // Rr = R2 R1
    }
    make_F(Cacc, Gam + (size_t)(nb - 1) * D * D, VZ, sel, theta, nk, D, R, F, Theta, nTheta, nF, s);
    launches += 1;
    cur = other;
    k0 = nk;
    // ---- stopping rule (Sec. 4.3, reading R11) ----
    double sv = (double)R;
    if (events.size() >= 2) {
      int later = 0;
      for (size_t e = 1; e < events.size(); ++e) later += events[e].second;
      sv = (double)(events.back().first - events.front().first) / std::max(1.0, (double)later / D);
    }
    sv = std::max(sv, (double)R);
    const int64_t since = matvecs - (events.empty() ? 0 : events.back().first);
    if (debug) {
      long long cnt[4] = {0, 0, 0, 0};
      cudaMemcpy(cnt, counters, sizeof(cnt), cudaMemcpyDeviceToHost);
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      fprintf(stderr,
              "[ns] %.3fs restart %lld matvecs %lld locked %d small %d unlocked %d k0 %d theta0 %.3e res0 %.3e "
              "reorthZ %lld reorthX %lld\n",
              el, (long long)restarts, (long long)matvecs, nlock, nsmall, n_unl, nk, pin_theta[0], pin_res[0], cnt[0],
              cnt[1]);
    }
    // before the first lock there is no speed estimate: the smallest Ritz value must
    // also have converged at or above 3 eps (the direct test of Sec. 4.3)
    const bool settled =
        !events.empty() || (!small(pin_theta[0]) && pin_res[0] <= tol_eff * normB_est);
    if (n_unl == 0 && nlocked_now == 0 && (double)since > o.stop_factor * sv && settled) return true;
    return false;
  }

  void mat2(const double* a, const double* b, double* c) {
    // c = a b for d x d on the device via the finalize helper: reuse a tiny kernel
    mat_small(a, b, c);
  }
  void mat_small(const double* a, const double* b, double* c);

  // ---- checkpoint / resume at a thick restart (the state at the top of the cycle loop) ----
  ns_checkpoint_info checkpoint_record(int k0) const {
    ns_checkpoint_info c{};
    c.version = kCkptVersion;
    c.m = m;
    c.n = n;
    c.nnz = h->nnz;
    c.mode = h->mode;
    c.precision = std::is_same<T, float>::value ? NS_MIXED : NS_FP64;
    c.d = D;
    c.restart_len = R;
    c.reorth = o.reorth;
    c.gemm = o.gemm;
    c.fp64_products = o.fp64_products;
    c.spmm_A = A.V;
    c.spmm_At = h->mode == NS_MODE_NORMAL ? At.V : 0;
    c.seed = h->seed;
    c.eps = eps;
    c.tol_eff = tol_eff;
    c.normA1 = h->normA1;
    c.normAinf = h->normAinf;
    c.matvecs = matvecs;
    c.restarts = restarts;
    c.nullity = nlock;
    c.k0 = k0;
    c.precond = pc ? pc->alpha : (o.precond == 2 ? -1.0 : 0.0);
    return c;
  }
  // host scalars of the iteration, in file order
  struct HostState {
    int64_t cur, cap, nlock, breakdowns, lock_events, ghosts, nevents, small_bytes;
    double theta_max, u_d, bd_tol;
  };
  void save_checkpoint(int k0) {
    sync();
    CkptWriter w;
    if (!w.open(o.checkpoint_path)) throw Fail{NS_ERR_IO, "cannot open checkpoint file for writing"};
    const ns_checkpoint_info c = checkpoint_record(k0);
    w.put(&c, sizeof c);
    const HostState hs{cur, cap, nlock, breakdowns, lock_events, ghosts, (int64_t)events.size(), (int64_t)small.bytes,
                       theta_max, u_d, bd_tol};
    w.put(&hs, sizeof hs);
    for (const auto& e : events) {
      const int64_t ev[2] = {e.first, e.second};
      w.put(ev, sizeof ev);
    }
    w.put(xtheta_h.data(), sizeof(double) * nlock);
    w.put(xrho_h.data(), sizeof(double) * nlock);
    ck(w.put_device(small.p, small.bytes, s), "checkpoint d2h");
    ck(w.put_device(wxbuf.p, wxbuf.bytes, s), "checkpoint d2h");
    ck(w.put_device(Z[cur], sizeof(T) * (size_t)n * (k0 + D), s), "checkpoint d2h");
    ck(w.put_device(X(), sizeof(T) * (size_t)n * nlock, s), "checkpoint d2h");
    if (!w.commit()) throw Fail{NS_ERR_IO, "checkpoint write failed"};
  }
  // restores the state written by save_checkpoint; returns k0
  int restore_checkpoint(CkptReader& r, const ns_checkpoint_info& c) {
    auto bad = [](const char* what) { return Fail{NS_ERR_IO, std::string("checkpoint: ") + what}; };
    HostState hs{};
    if (!r.get(&hs, sizeof hs)) throw bad("short file");
    const int k0 = (int)c.k0;
    if (c.k0 < D || c.k0 > R - 2 * D || c.k0 % D || (hs.cur != 0 && hs.cur != 1) || hs.nlock < 0 ||
        hs.nlock != c.nullity || hs.cap < std::max<int64_t>(hs.nlock, 1) || hs.cap > n || hs.nevents < 0 ||
        hs.nevents > c.restarts || hs.small_bytes != (int64_t)small.bytes || c.matvecs < 0 || c.restarts < 1)
      throw bad("inconsistent state");
    if (hs.cap != cap) {  // the locked store at the checkpoint's capacity (the W rows depend on it)
      xbuf = Buf(h, sizeof(T) * (size_t)n * hs.cap);
      cap = (int)hs.cap;
      alloc_proj();
      alloc_locked_meta(0);
    }
    events.clear();
    for (int64_t i = 0; i < hs.nevents; ++i) {
      int64_t ev[2];
      if (!r.get(ev, sizeof ev)) throw bad("short file");
      events.emplace_back(ev[0], (int)ev[1]);
    }
    nlock = (int)hs.nlock;
    xtheta_h.assign(nlock, 0.0);
    xrho_h.assign(nlock, 0.0);
    if (!r.get(xtheta_h.data(), sizeof(double) * nlock) || !r.get(xrho_h.data(), sizeof(double) * nlock))
      throw bad("short file");
    ck(r.get_device(small.p, small.bytes, s), "checkpoint h2d");
    ck(r.get_device(wxbuf.p, wxbuf.bytes, s), "checkpoint h2d");
    cur = (int)hs.cur;
    ck(r.get_device(Z[cur], sizeof(T) * (size_t)n * (k0 + D), s), "checkpoint h2d");
    ck(r.get_device(X(), sizeof(T) * (size_t)n * nlock, s), "checkpoint h2d");
    if (!r.ok() || !r.finish()) throw bad("short or corrupt file (checksum)");
    // flags, reduction tickets and the tensor-core error word are zero between cycles
    ck(cudaMemsetAsync(flags, 0, 8 * sizeof(double), s), "memset");
    breakdowns = hs.breakdowns;
    lock_events = hs.lock_events;
    ghosts = hs.ghosts;
    theta_max = hs.theta_max;
    u_d = hs.u_d;
    bd_tol = hs.bd_tol;
    matvecs = c.matvecs;
    restarts = c.restarts;
    resumed_at = c.restarts;
    sync();
    return k0;
  }
  int64_t resumed_at = -1;

  // ---- whole Lanczos phase; `from`: a checkpoint to continue instead of a new start ----
  ns_status run(bool& converged, CkptReader* from = nullptr, const ns_checkpoint_info* rec = nullptr) {
    int k0 = 0;
    if (from)
      k0 = restore_checkpoint(*from, *rec);
    else
      orthonormal_start();
    const int64_t maxmv = o.max_matvec > 0 ? o.max_matvec : std::min<int64_t>(100 * n + 50 * R, 1000000);
    converged = false;
    while (true) {
      const int r0 = k0 / D;
      first_step(r0);
      for (int j = r0 + 1; j < nb; ++j) inner_step(j, r0);
      if (restart(k0)) {
        converged = true;
        break;
      }
      const bool stop = matvecs >= maxmv;
      if (o.checkpoint_every > 0 && (stop || restarts % o.checkpoint_every == 0)) save_checkpoint(k0);
      if (stop) break;
    }
    return converged ? NS_OK : NS_ERR_NOT_CONVERGED;
  }
};

__global__ void k_mat_small(const double* a, const double* b, double* c, int d) {
  if (threadIdx.x == 0) matmul_dd(a, b, c, d);
}
template <typename T, int D>
void Solver<T, D>::mat_small(const double* a, const double* b, double* c) {
  k_mat_small<<<1, 32, 0, s>>>(a, b, c, D);
  launches += 1;
}

// ---------------------------------------------------------------------------
// FP64 refinement: project every basis column onto null(A) (CG / CGLS)
// ---------------------------------------------------------------------------
struct RefineOut {
  int64_t iters_max = 0;  // largest number of inner iterations over all chunks
  double resid_max = 0.0; // max_j ||A x_j|| / ||A||_2 after refinement (FP64)
  int failed = 0;
  double bytes = 0.0, flops = 0.0;  // algorithmic work of every kernel enqueued (each operand once)
};

// Projection of every basis column onto null(A) (Remark after Alg. 1 motivates
// removing the perturbation at the end): x <- x - delta with delta the minimum-norm
// solution of A delta = A x (CG, SPD form) or min ||A delta - A x|| (CGLS, normal
// form).  Mixed-precision iterative refinement: the residual r = A x and the update
// x <- x - delta are FP64; each inner solve runs in FP32 and only has to reduce the
// residual of its column by kInner; outer rounds repeat until ||A x|| <= tol ||A||.
RefineOut refine(ns_handle* h, double* X, int64_t N, double normA, const ns_opts& o) {
  RefineOut out;
  constexpr int W = 16;
  constexpr double kInner = 1e-4;
  cudaStream_t s = h->stream;
  const int64_t n = h->n, m = h->m;
  const bool normal = h->mode == NS_MODE_NORMAL;
  const int64_t nr = normal ? m : n;  // rows of the residual
  ensure_fp32(h);
  Csr<double> A64 = csr_A<double>(h);
  Csr<float> A32 = csr_A<float>(h), At32;
  if (normal) At32 = csr_At<float>(h);
  if (o.precond == 2) {  // reading P5: the scaled rows S A (same null space, balanced residual)
    const auto& I = h->inner;
    A64.val = I.val;
    A32.val = I.val32;
    At32.val = I.val_t32;
    A64.sptr = A32.sptr = At32.sptr = nullptr;
    if (A64.V == kSchedSell || A64.V == kSchedTma) A64.V = A32.V = 8;
    if (At32.V == kSchedSell || At32.V == kSchedTma) At32.V = 8;
  }
  if (o.precond == 1) {  // the basis is in the renumbered space: refine against A~
    const auto& P = h->pc;
    A64 = Csr<double>{};
    A64.rowptr = P.arp;
    A64.col = P.acol;
    A64.val = P.aval;
    A64.nrows = A64.ncols = n;
    A64.nnz = P.nnzA;
    A64.V = choose_lanes(n, P.nnzA);
    A32 = Csr<float>{};
    A32.rowptr = P.arp;
    A32.col = P.acol;
    A32.val = P.aval32;
    A32.nrows = A32.ncols = n;
    A32.nnz = P.nnzA;
    A32.V = A64.V;
  }
  Buf bx(h, sizeof(double) * n * W), br64(h, sizeof(double) * nr * W), bd(h, sizeof(float) * n * W),
      bp(h, sizeof(float) * n * W), bq(h, sizeof(float) * nr * W), br(h, sizeof(float) * nr * W),
      bs(h, sizeof(float) * n * W), bred(h, sizeof(double) * (size_t)kMaxBlocks * 64 + 256), bsm(h, 8192);
  Red red;
  red.part = bred.as<double>();
  double* sm = bsm.as<double>();
  double *rr64 = sm, *rr = sm + 32, *rrn = sm + 64, *den = sm + 96, *alpha = sm + 128, *beta = sm + 160,
         *gam = sm + 192, *tin = sm + 224;
  unsigned char* act_out = reinterpret_cast<unsigned char*>(sm + 256);
  unsigned char* act = reinterpret_cast<unsigned char*>(sm + 264);
  int* nact = reinterpret_cast<int*>(sm + 272);
  red.ticket = reinterpret_cast<unsigned*>(sm + 280);
  ck(cudaMemsetAsync(bsm.p, 0, 8192, s), "memset");
  int* nact_h = nullptr;
  ck(cudaMallocHost(&nact_h, 1024), "cudaMallocHost");
  double* rr_h = reinterpret_cast<double*>(nact_h + 8);
  const double tol2 = (o.refine_tol * normA) * (o.refine_tol * normA);
  // algorithmic bytes / flops of the panel kernels (width W, value size sv)
  const double nnz = (double)h->nnz;
  auto spmm_work = [&](double rows, double cols, double sv, bool with_w) {  // y = M v (+ dots)
    out.bytes += nnz * (4.0 + sv) + (rows + 1.0) * 8.0 + cols * W * sv + rows * W * sv * (with_w ? 2.0 : 1.0);
    out.flops += 2.0 * nnz * W + 2.0 * rows * W;
  };
  auto A_work = [&](double sv, bool with_w) { spmm_work((double)nr, (double)n, sv, with_w); };
  auto At_work = [&](double sv) { spmm_work((double)n, (double)m, sv, false); };
  auto stream_work = [&](double rows, double bytes_per, double flops_per) {
    out.bytes += rows * W * bytes_per;
    out.flops += rows * W * flops_per;
  };
  auto read_nact = [&]() {
    ck(cudaMemcpyAsync(nact_h, nact, sizeof(int), cudaMemcpyDeviceToHost, s), "d2h");
    ck(cudaStreamSynchronize(s), "sync");
    return *nact_h;
  };
  const bool dbg = getenv("NS_DEBUG") != nullptr;
  for (int64_t c0 = 0; c0 < N; c0 += W) {
    const int w = (int)std::min<int64_t>(W, N - c0);
    const auto tc0 = std::chrono::steady_clock::now();
    int rounds = 0, inner_total = 0;
    cols_to_panel_w<W>(X, (int)c0, w, n, bx.as<double>(), s);
    stream_work((double)n, 16.0, 0.0);
    std::vector<unsigned char> a0(W, 0);
    for (int c = 0; c < w; ++c) a0[c] = 1;
    ck(cudaMemcpyAsync(act_out, a0.data(), W, cudaMemcpyHostToDevice, s), "h2d");
    h->launches += 1;
    for (int outer = 0; outer < 8; ++outer) {
      // FP64 residual of the current iterate
      spmm_coldot<double, W>(A64, bx.as<double>(), br64.as<double>(), nullptr, 1, rr64, red, s);
      A_work(8.0, false);
      cg_check(rr64, nullptr, tol2, act_out, nact, W, s);
      h->launches += 2;
      if (read_nact() == 0) break;
      // inner solve in FP32: delta with A delta ~ r (CG) or min ||A delta - r|| (CGLS)
      convert_d2f(br64.as<double>(), br.as<float>(), nr * W, s);
      stream_work((double)nr, 12.0, 0.0);
      ck(cudaMemsetAsync(bd.p, 0, bd.bytes, s), "memset");
      ck(cudaMemcpyAsync(act, act_out, W, cudaMemcpyDeviceToDevice, s), "copy");
      scale_vec(rr64, kInner * kInner, tin, W, s);
      h->launches += 2;
      int it = 0;
      if (!normal) {
        ck(cudaMemcpyAsync(bp.p, br.p, sizeof(float) * n * W, cudaMemcpyDeviceToDevice, s), "copy");
        ck(cudaMemcpyAsync(rr, rr64, sizeof(double) * W, cudaMemcpyDeviceToDevice, s), "copy");
        for (; it < o.refine_maxit; ++it) {
          spmm_coldot<float, W>(A32, bp.as<float>(), bq.as<float>(), nullptr, 0, den, red, s);  // p^T A p
          A_work(4.0, false);
          cg_scalars(rr, den, act, alpha, W, s);
          cg_update2<float, W>(bd.as<float>(), bp.as<float>(), n, br.as<float>(), bq.as<float>(), n, alpha, red,
                               rrn, s);
          stream_work(2.0 * n, 12.0, 4.0);
          cg_scalars(rrn, rr, act, beta, W, s);
          cg_direction2<float, W>(bp.as<float>(), br.as<float>(), beta, n, s);
          stream_work((double)n, 12.0, 2.0);
          ck(cudaMemcpyAsync(rr, rrn, sizeof(double) * W, cudaMemcpyDeviceToDevice, s), "copy");
          cg_check(rr, tin, 0.0, act, nact, W, s);
          h->launches += 6;
          if ((it & 3) == 3 && read_nact() == 0) break;
        }
      } else {
        spmm_coldot<float, W>(At32, br.as<float>(), bs.as<float>(), nullptr, 1, gam, red, s);  // s = A^T r
        At_work(4.0);
        ck(cudaMemcpyAsync(bp.p, bs.p, sizeof(float) * n * W, cudaMemcpyDeviceToDevice, s), "copy");
        h->launches += 1;
        for (; it < o.refine_maxit; ++it) {
          spmm_coldot<float, W>(A32, bp.as<float>(), bq.as<float>(), nullptr, 1, den, red, s);  // ||A p||^2
          A_work(4.0, false);
          cg_scalars(gam, den, act, alpha, W, s);
          cg_update2<float, W>(bd.as<float>(), bp.as<float>(), n, br.as<float>(), bq.as<float>(), m, alpha, red,
                               rr, s);
          stream_work((double)(n + m), 12.0, 4.0);
          spmm_coldot<float, W>(At32, br.as<float>(), bs.as<float>(), nullptr, 1, rrn, red, s);  // ||A^T r||^2
          At_work(4.0);
          cg_scalars(rrn, gam, act, beta, W, s);
          cg_direction2<float, W>(bp.as<float>(), bs.as<float>(), beta, n, s);
          stream_work((double)n, 12.0, 2.0);
          ck(cudaMemcpyAsync(gam, rrn, sizeof(double) * W, cudaMemcpyDeviceToDevice, s), "copy");
          cg_check(rr, tin, 0.0, act, nact, W, s);
          h->launches += 7;
          if ((it & 3) == 3 && read_nact() == 0) break;
        }
      }
      out.iters_max = std::max<int64_t>(out.iters_max, it + 1);
      rounds += 1;
      inner_total += it + 1;
      sub_correction<W>(bx.as<double>(), bd.as<float>(), n, s);  // x <- x - delta in FP64
      stream_work((double)n, 20.0, 1.0);
      h->launches += 1;
    }
    // final FP64 residual for the statistics
    spmm_coldot<double, W>(A64, bx.as<double>(), br64.as<double>(), nullptr, 1, rr64, red, s);
    A_work(8.0, false);
    panel_to_cols64<W>(bx.as<double>(), X, (int)c0, w, n, s);
    stream_work((double)n, 16.0, 0.0);
    ck(cudaMemcpyAsync(rr_h, rr64, sizeof(double) * W, cudaMemcpyDeviceToHost, s), "d2h");
    ck(cudaStreamSynchronize(s), "sync");
    ck_launch("refine");
    h->launches += 2;
    if (dbg)
      fprintf(stderr, "[ns] refine chunk %lld: %d rounds, %d inner iterations, %.2f ms\n", (long long)c0, rounds,
              inner_total, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tc0).count());
    for (int c = 0; c < w; ++c) {
      const double rel = std::sqrt(std::max(rr_h[c], 0.0)) / std::max(normA, 1e-300);
      out.resid_max = std::max(out.resid_max, rel);
      if (rr_h[c] > tol2 * 1.0001) out.failed += 1;
    }
  }
  cudaFreeHost(nact_h);
  return out;
}

// Sec. 4.4.2 post-processing: the locked vectors X approximate L^T null(A~), so
// L^-T X spans null(A~).  Panel by panel (W columns): L^-T by colours, CGS2 against
// the columns already done (compensated FP32-pair products), CholQR2; FP64, in the
// renumbered space.  Rank loss is a numerical failure.
template <int W>
void pc_panel(ns_handle* h, const double* Xin, double* Xout, int c0, double* P, double* Q, double* cbuf,
              double* dpart, double* sm, const Red& red, unsigned* flags_h) {
  const auto& pc = h->pc;
  const int64_t n = h->n;
  cudaStream_t s = h->stream;
  double *R1 = sm, *R2 = sm + 64;
  unsigned* flags = reinterpret_cast<unsigned*>(sm + 128);
  if ((size_t)c0 * W * sizeof(double) > 190 * 1024)
    throw Fail{NS_ERR_INVALID_ARG, "too many null vectors for the preconditioned post-processing"};
  cols_to_panel_t<double>(Xin, c0, W, n, Q, s);
  trsv_colors<double, W>(pc.urp, pc.ucol, pc.uval, pc.cstart.data(), pc.ncolors, false, Q, P, s);
  h->launches += 1 + pc.ncolors;
  if (c0 == 0) {
    gram_chol<double, W>(P, W, W, n, R1, nullptr, flags, red, s);
    h->launches += 1;
  } else {
    VParts<double> V;
    V.X = Xout;
    V.kx = c0;
    V.df = 1;
    for (int pass = 0; pass < 2; ++pass) {
      proj_dots<double, W>(V, P, nullptr, W, n, cbuf, dpart, s, kDotsAutoChunks);
      ck((proj_update<double, W>(V, cbuf, P, nullptr, W, n, pass == 1 ? 1 : 0, R1, nullptr, flags, red, s)),
         "proj_update shared-memory limit");
      h->launches += 3;
    }
  }
  scale_gram<double, W>(P, W, P, W, R1, n, R2, flags, red, s, W);
  scale_gram<double, W>(P, W, P, W, R2, n, nullptr, flags, red, s, W);
  panel_to_cols<double>(P, W, W, n, Xout, c0, s);
  h->launches += 3;
  ck(cudaMemcpyAsync(flags_h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  ck(cudaStreamSynchronize(s), "sync");
  if (*flags_h & 1u) throw Fail{NS_ERR_NUMERICAL, "L^-T X lost rank (preconditioned post-processing)"};
}

void pc_postprocess(ns_handle* h, double* X, int64_t N, double* Xout) {
  const int64_t n = h->n;
  Buf P(h, sizeof(double) * n * 8), Q(h, sizeof(double) * n * 8), cbuf(h, sizeof(double) * (size_t)N * 16),
      dpart(h, sizeof(double) * (size_t)ceil_div(std::max<int64_t>(n, 1), kDotsMinChunk) * N * 16),
      red_part(h, sizeof(double) * (size_t)kMaxBlocks * 64 + 256), sm(h, 4096);
  ck(cudaMemsetAsync(sm.p, 0, 4096, h->stream), "memset");
  Red red;
  red.part = red_part.as<double>();
  red.ticket = reinterpret_cast<unsigned*>(sm.as<double>() + 256);
  unsigned* flags_h = nullptr;
  ck(cudaMallocHost(&flags_h, 64), "cudaMallocHost");
  try {
    for (int64_t c0 = 0; c0 < N;) {
      const int64_t left = N - c0;
      const int w = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
      double* a[4] = {P.as<double>(), Q.as<double>(), cbuf.as<double>(), dpart.as<double>()};
      switch (w) {
        case 8: pc_panel<8>(h, X, Xout, (int)c0, a[0], a[1], a[2], a[3], sm.as<double>(), red, flags_h); break;
        case 4: pc_panel<4>(h, X, Xout, (int)c0, a[0], a[1], a[2], a[3], sm.as<double>(), red, flags_h); break;
        case 2: pc_panel<2>(h, X, Xout, (int)c0, a[0], a[1], a[2], a[3], sm.as<double>(), red, flags_h); break;
        default: pc_panel<1>(h, X, Xout, (int)c0, a[0], a[1], a[2], a[3], sm.as<double>(), red, flags_h); break;
      }
      c0 += w;
    }
  } catch (...) {
    cudaFreeHost(flags_h);
    throw;
  }
  cudaFreeHost(flags_h);
  ck_launch("preconditioned post-processing");
}

}  // namespace

// typed bodies of the C entry points
template <typename T, int D>
static ns_status solve_typed(ns_handle* h, int R, double tol, const ns_opts& o) {
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  ns_status st = NS_OK;
  bool conv = false;
  int64_t N = 0;
  h->prof.reset(o.profile, s);
  CkptReader rd;
  ns_checkpoint_info rec{};
  if (o.resume) {
    if (rd.open(o.checkpoint_path, &rec) != NS_OK) throw Fail{NS_ERR_IO, "checkpoint missing or unreadable"};
    if (rec.m != h->m || rec.n != h->n || rec.nnz != h->nnz || rec.mode != h->mode || rec.seed != h->seed ||
        rec.normA1 != h->normA1 || rec.normAinf != h->normAinf)
      throw Fail{NS_ERR_INVALID_ARG, "checkpoint of another matrix or seed"};
    if (rec.precision != (std::is_same<T, float>::value ? NS_MIXED : NS_FP64) || rec.d != D ||
        rec.restart_len != R || rec.reorth != o.reorth || rec.gemm != o.gemm ||
        rec.fp64_products != o.fp64_products || rec.eps != o.eps ||
        rec.precond != (o.precond == 1 ? o.precond_shift : o.precond == 2 ? -1.0 : 0.0))
      throw Fail{NS_ERR_INVALID_ARG, "checkpoint of a solve with other d, restart_len or opts"};
  }
  Solver<T, D> S(h, R, tol, o, o.resume ? &rec : nullptr);
  if (o.resume && rec.tol_eff != S.tol_eff) throw Fail{NS_ERR_INVALID_ARG, "checkpoint of a solve with another tol"};
  cudaEventRecord(e0, s);
  st = S.run(conv, o.resume ? &rd : nullptr, &rec);
  cudaEventRecord(e1, s);
  N = S.nlock;
  // FP64 basis
  if (h->basis) dfree(h, h->basis, h->basis_bytes);
  h->basis_bytes = sizeof(double) * (size_t)std::max<int64_t>(N, 1) * h->n;
  h->basis = (double*)dalloc(h, h->basis_bytes);
  if (N) {
    if (std::is_same<T, double>::value)
      ck(cudaMemcpyAsync(h->basis, S.X(), sizeof(double) * (size_t)N * h->n, cudaMemcpyDeviceToDevice, s), "copy");
    else
      convert_f2d(reinterpret_cast<const float*>(S.X()), h->basis, (int64_t)N * h->n, s);
  }
  double normA = (h->mode == NS_MODE_NORMAL) ? std::sqrt(std::max(S.theta_max, 0.0)) : S.theta_max;
  if (o.precond == 2) normA = std::sqrt(h->inner.normA1 * h->inner.normAinf);  // bound on ||S A||_2
  if (o.precond == 1) {
    // the Ritz values are those of B_R: ||A||_2 is bounded by ||A||_inf instead
    normA = h->normAinf;
    if (N) {
      double* Y = (double*)dalloc(h, h->basis_bytes);
      try {
        pc_postprocess(h, h->basis, N, Y);
      } catch (...) {
        dfree(h, Y, h->basis_bytes);
        throw;
      }
      dfree(h, h->basis, h->basis_bytes);
      h->basis = Y;
    }
  }
  RefineOut ro;
  if (o.refine && N) {
    {
      PScope ps(&h->prof, P_REFINE, 0.0, 0.0);
      ro = refine(h, h->basis, N, normA, o);
    }
    h->prof.add(P_REFINE, ro.bytes, ro.flops);  // one "launch" = the whole refinement phase
    ck(cudaStreamSynchronize(s), "sync");
    h->prof.flush();
    if (ro.failed && st == NS_OK) st = NS_ERR_REFINE;
  }
  // Projecting B-eigenvectors onto null(A) removes an O(eps/sigma) component from
  // each, so the refined basis is orthonormal only to O(eps^2/sigma^2); a
  // symmetric (Loewdin) correction X <- X (I - E/2), E = X^T X - I, restores it.
  double orth0 = 0.0, orth1 = 0.0;
  if (N) {
    Buf G(h, sizeof(double) * (size_t)N * N), part(h, sizeof(double) * gram_part_doubles(h->n, (int)N)),
        mx(h, 256);
    double* X2 = (double*)dalloc(h, h->basis_bytes);
    double* mx_h = nullptr;
    ck(cudaMallocHost(&mx_h, 64), "cudaMallocHost");
    for (int it = 0; it < 4; ++it) {
      {
        PScope ps(&h->prof, P_ORTH, 8.0 * N * h->n, 1.0 * N * N * h->n);
        gram64(h->basis, h->n, (int)N, G.as<double>(), part.as<double>(), s);
        max_offdiag(G.as<double>(), (int)N, mx.as<double>(), s);
      }
      h->launches += 3;
      ck(cudaMemcpyAsync(mx_h, mx.p, sizeof(double), cudaMemcpyDeviceToHost, s), "d2h orth");
      ck(cudaStreamSynchronize(s), "sync");
      h->prof.flush();
      if (it == 0) orth0 = *mx_h;
      orth1 = *mx_h;
      if (*mx_h <= 1e-14) break;
      {
        PScope ps(&h->prof, P_ORTH, 16.0 * N * h->n, 2.0 * N * N * h->n);
        lowdin_update(h->basis, h->n, (int)N, G.as<double>(), X2, s);
      }
      h->launches += 1;
      std::swap(h->basis, X2);
      orth1 = 0.375 * (*mx_h) * (*mx_h) * N;  // predicted second-order remainder
      if (*mx_h <= 1e-6) break;
    }
    if (o.precond == 1) {  // rows back to the original numbering
      unpermute_cols(h->basis, h->pc.perm, h->n, (int)N, X2, s);
      h->launches += 1;
      std::swap(h->basis, X2);
    }
    ck(cudaStreamSynchronize(s), "sync");
    ck_launch("reorthonormalize");
    cudaFreeHost(mx_h);
    dfree(h, X2, h->basis_bytes);
  }
  cudaEventRecord(e2, s);
  ck(cudaEventSynchronize(e2), "sync");
  h->prof.flush();
  float t1 = 0.f, t2 = 0.f;
  cudaEventElapsedTime(&t1, e0, e1);
  cudaEventElapsedTime(&t2, e1, e2);
  long long cnt[4] = {0, 0, 0, 0};
  ck(cudaMemcpy(cnt, S.counters, sizeof(cnt), cudaMemcpyDeviceToHost), "d2h");
  unsigned uerr = 0;
  ck(cudaMemcpy(&uerr, S.umma_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "d2h");
  if (uerr) st = NS_ERR_TIMEOUT;  // a bounded wait of the tensor-core product gave up
  ns_stats_t& x = h->stats;
  x = ns_stats_t{};
  x.nullity = N;
  x.matvecs = S.matvecs;
  x.restarts = S.restarts;
  x.reorth_Z = cnt[0];
  x.reorth_X = cnt[1];
  x.breakdowns = S.breakdowns;
  x.lock_events = S.lock_events;
  x.ghosts = S.ghosts;
  x.refine_iters_max = ro.iters_max;
  x.normB = S.normB;
  x.normA = normA;
  x.u_d = S.u_d;
  x.refine_resid_max = ro.resid_max;
  x.orth_before = orth0;
  x.orth_after = orth1;
  x.t_lanczos_ms = t1;
  x.t_refine_ms = t2;
  x.t_total_ms = t1 + t2;
  x.d = D;
  x.resumed_at = S.resumed_at;
  h->N = N;
  h->solved = true;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  return st;
}

template <typename T, int D>
static void trace_omega_typed(ns_handle* h, int R, const ns_opts& o, double* W) {
  const int nbp = R / D + 1;
  Buf tr(h, sizeof(double) * (size_t)nbp * nbp);
  ck(cudaMemsetAsync(tr.p, 0, tr.bytes, h->stream), "memset");
  h->prof.reset(0, h->stream);
  Solver<T, D> S(h, R, 1.0, o);
  S.trace_dev = tr.as<double>();
  S.run_first_cycle();
  ck(cudaMemcpyAsync(W, tr.p, tr.bytes, cudaMemcpyDeviceToHost, h->stream), "d2h trace");
  ck(cudaStreamSynchronize(h->stream), "sync");
}

template <typename T, int D>
static void apply_B_typed(ns_handle* h, const T* x, T* y, double eps, Red red, int schedule, int pre = 0) {
  StepOps<T> op;
  op.x = x;
  op.Dv = Prec<T>::D(h);
  op.eps = eps;
  op.out = y;
  Buf xi(h, sizeof(double) * 80);
  op.xi = xi.as<double>();
  op.xi_norm = xi.as<double>() + 64;
  Csr<T> A = csr_A<T>(h);
  Csr<T> At = h->mode == NS_MODE_SPD ? A : csr_At<T>(h);
  if (schedule >= 0) A.V = At.V = schedule;
  if (pre == 2) {  // B_L x = (S A)^T (S A) x + eps D x (Sec. 4.4.1)
    A.val = pc_vals<T>(h->inner.val, h->inner.val32);
    At.val = pc_vals<T>(h->inner.val_t, h->inner.val_t32);
    A.sptr = At.sptr = nullptr;
    if (A.V == kSchedSell) A.V = At.V = 8;
  }
  if (pre == 1) {  // B_R x = L^-1 A~ L^-T x + eps D x, renumbered space
    const auto& P = h->pc;
    Csr<T> Ap;
    Ap.rowptr = P.arp;
    Ap.col = P.acol;
    Ap.val = pc_vals<T>(P.aval, P.aval32);
    Ap.nrows = Ap.ncols = h->n;
    Ap.nnz = P.nnzA;
    Ap.V = choose_lanes(h->n, P.nnzA);
    Buf t(h, sizeof(T) * h->n * D), u(h, sizeof(T) * h->n * D);
    trsv_colors<T, D>(P.urp, P.ucol, pc_vals<T>(P.uval, P.uval32), P.cstart.data(), P.ncolors, false, x, t.as<T>(),
                      h->stream);
    spmm_plain<T, D>(Ap, t.as<T>(), u.as<T>(), h->stream);
    trsv_colors<T, D>(P.lrp, P.lcol, pc_vals<T>(P.lval, P.lval32), P.cstart.data(), P.ncolors, true, u.as<T>(),
                      u.as<T>(), h->stream);
    lanczos_epilogue<T, D>(u.as<T>(), h->n, op, red, h->stream);
    ck(cudaStreamSynchronize(h->stream), "sync");
  } else if (h->mode == NS_MODE_SPD) {
    spmm_lanczos<T, D>(A, x, op, red, h->stream);
  } else {
    Buf yb(h, sizeof(T) * h->m * D);
    spmm_plain<T, D>(A, x, yb.as<T>(), h->stream);
    spmm_lanczos<T, D>(At, yb.as<T>(), op, red, h->stream);
    ck(cudaStreamSynchronize(h->stream), "sync");
  }
  ck(cudaStreamSynchronize(h->stream), "sync");
  ck_launch("apply_B");
}

template <typename T, int W>
static void project_typed(ns_handle* h, int64_t n, int K, const double* V, double* Wm, double* C, int df) {
  Buf vb(h, sizeof(T) * n * std::max(K, 1)), wb(h, sizeof(T) * n * W), v64(h, sizeof(double) * n * std::max(K, 1)),
      w64(h, sizeof(double) * n * W), cb(h, sizeof(double) * K * W), cb2(h, sizeof(double) * K * W),
      part(h, sizeof(double) * ((size_t)ceil_div(n, std::min<int64_t>(kThreads * 128, n)) * K * W + 8)),
      rp(h, sizeof(double) * kMaxBlocks * 64 + 256), tk(h, 256);
  ck(cudaMemset(tk.p, 0, 256), "memset");
  Red red;
  red.part = rp.as<double>();
  red.ticket = tk.as<unsigned>();
  ck(cudaMemcpy(v64.p, V, sizeof(double) * n * K, cudaMemcpyHostToDevice), "h2d");
  ck(cudaMemcpy(w64.p, Wm, sizeof(double) * n * W, cudaMemcpyHostToDevice), "h2d");
  T *vp, *wp;
  if (std::is_same<T, double>::value) {
    vp = reinterpret_cast<T*>(v64.p);
    wp = reinterpret_cast<T*>(w64.p);
  } else {
    convert_d2f(v64.as<double>(), vb.as<float>(), n * K, nullptr);
    convert_d2f(w64.as<double>(), wb.as<float>(), n * W, nullptr);
    vp = vb.as<T>();
    wp = wb.as<T>();
  }
  VParts<T> P;
  P.X = vp;
  P.kx = K;
  P.Z = nullptr;
  P.kz = 0;
  P.p = 1;
  P.df = df;
  proj_dots<T, W>(P, wp, nullptr, W, n, cb.as<double>(), part.as<double>(), nullptr);
  ck((proj_update<T, W>(P, cb.as<double>(), wp, nullptr, W, n, 0, nullptr, nullptr, nullptr, red, nullptr)), "limit");
  proj_dots<T, W>(P, wp, nullptr, W, n, cb2.as<double>(), part.as<double>(), nullptr);
  ck((proj_update<T, W>(P, cb2.as<double>(), wp, nullptr, W, n, 0, nullptr, nullptr, nullptr, red, nullptr)),
     "limit");
  ck_launch("project");
  ck(cudaDeviceSynchronize(), "sync");
  if (!std::is_same<T, double>::value) convert_f2d(wb.as<float>(), w64.as<double>(), n * W, nullptr);
  ck(cudaDeviceSynchronize(), "sync");
  ck(cudaMemcpy(Wm, w64.p, sizeof(double) * n * W, cudaMemcpyDeviceToHost), "d2h");
  std::vector<double> c1(K * W), c2(K * W);
  ck(cudaMemcpy(c1.data(), cb.p, sizeof(double) * K * W, cudaMemcpyDeviceToHost), "d2h");
  ck(cudaMemcpy(c2.data(), cb2.p, sizeof(double) * K * W, cudaMemcpyDeviceToHost), "d2h");
  for (int t = 0; t < K * W; ++t) C[t] = c1[t] + c2[t];
}

template <typename T>
static void restart_product_typed(ns_handle* h, int64_t n, int d, int R, const double* Zh, const double* VZh,
                                  const int32_t* selh, int nsel, int nl, int gemm, double* outh) {
  // Z into the solver's panel layout: block b of d columns is an n x d row-major panel
  std::vector<T> zp((size_t)n * R);
  for (int j = 0; j < R; ++j) {
    const int b = j / d, q = j % d;
    for (int64_t i = 0; i < n; ++i) zp[(size_t)b * n * d + (size_t)i * d + q] = (T)Zh[(size_t)j * n + i];
  }
  const int nz = nsel - nl;
  Buf bz(h, sizeof(T) * zp.size()), bv(h, sizeof(double) * (size_t)R * R), bs(h, sizeof(int) * nsel),
      bl(h, sizeof(T) * (size_t)n * std::max(nl, 1)), bn(h, sizeof(T) * (size_t)n * std::max(nz, 1)),
      img(h, std::max(restart_umma_image_bytes(R, std::max(nsel, 1), 3), restart_ozaki_scratch_bytes(n, R, nsel))),
      fl(h, 256);
  cudaStream_t s = h->stream;
  ck(cudaMemcpyAsync(bz.p, zp.data(), bz.bytes, cudaMemcpyHostToDevice, s), "h2d");
  ck(cudaMemcpyAsync(bv.p, VZh, bv.bytes, cudaMemcpyHostToDevice, s), "h2d");
  ck(cudaMemcpyAsync(bs.p, selh, sizeof(int) * nsel, cudaMemcpyHostToDevice, s), "h2d");
  ck(cudaMemsetAsync(fl.p, 0, 256, s), "memset");
  const bool tc = gemm == NS_GEMM_TC2 || gemm == NS_GEMM_TC3 ||
                  (gemm == NS_GEMM_DEFAULT && std::is_same<T, float>::value);
  const bool exact = gemm == NS_GEMM_TC_EXACT ||
                     (gemm == NS_GEMM_DEFAULT && std::is_same<T, double>::value && restart_ozaki_supported(R, nsel));
  if constexpr (std::is_same<T, float>::value) {
    if (tc) {
      if (!restart_umma_supported(R, nsel)) throw Fail{NS_ERR_INVALID_ARG, "tensor-core product needs nsel <= 256"};
      ck(restart_gemm_umma(bz.as<float>(), d, R, bv.as<double>(), bs.as<int>(), nsel, nl, n, bl.as<float>(),
                           bn.as<float>(), img.p, fl.as<unsigned>(), gemm == NS_GEMM_TC2 ? 2 : 3, s),
         "restart_gemm_umma");
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    if (exact) {
      if (!restart_ozaki_supported(R, nsel)) throw Fail{NS_ERR_INVALID_ARG, "exact tensor-core product needs R <= 208"};
      ck(restart_gemm_ozaki(bz.as<double>(), d, R, bv.as<double>(), bs.as<int>(), nsel, nl, n, bl.as<double>(),
                            bn.as<double>(), img.p, fl.as<unsigned>(), s),
         "restart_gemm_ozaki");
    }
  }
  if (!tc && !exact)
    ck(restart_gemm<T>(bz.as<T>(), d, R, bv.as<double>(), bs.as<int>(), nsel, nl, n, bl.as<T>(), bn.as<T>(), s),
       "restart_gemm");
  ck_launch("restart product");
  std::vector<T> L((size_t)n * std::max(nl, 1)), Zn((size_t)n * std::max(nz, 1));
  unsigned err = 0;
  ck(cudaMemcpyAsync(L.data(), bl.p, bl.bytes, cudaMemcpyDeviceToHost, s), "d2h");
  ck(cudaMemcpyAsync(Zn.data(), bn.p, bn.bytes, cudaMemcpyDeviceToHost, s), "d2h");
  ck(cudaMemcpyAsync(&err, fl.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  ck(cudaStreamSynchronize(s), "sync");
  if (err) throw Fail{NS_ERR_TIMEOUT, "a bounded wait of the tensor-core product gave up"};
  for (int c = 0; c < nsel; ++c)
    for (int64_t i = 0; i < n; ++i) {
      double v;
      if (c < nl) {
        v = (double)L[(size_t)i * nl + c];
      } else {
        const int kz = c - nl;
        v = (double)Zn[(size_t)(kz / d) * n * d + (size_t)i * d + kz % d];
      }
      outh[(size_t)c * n + i] = v;
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void ns_default_opts(ns_opts* o) {
  if (!o) return;
  o->eps = 1e-3;
  o->precision = NS_FP64;
  o->reorth = NS_REORTH_PARTIAL;
  o->max_matvec = 0;
  o->stop_factor = 2.0;
  o->lock_tol_mixed = 1e-5;
  o->refine = 1;
  o->refine_tol = 1e-10;
  o->refine_maxit = 500;
  o->refine_chunk = 8;
  o->use_graphs = 0;
  o->batch_block = 0;
  o->profile = 0;
  o->gemm = NS_GEMM_DEFAULT;
  o->fp64_products = 0;
  o->spmm_schedule = 0;
  o->checkpoint_every = 0;
  o->resume = 0;
  o->checkpoint_path = nullptr;
  o->precond = 0;
  o->precond_shift = 0.1;
}

static ns_status set_err(ns_handle* h, ns_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

ns_status ns_create(ns_handle** out, int64_t m, int64_t n, const int64_t* rowptr, const int32_t* colind,
                    const void* vals, int vals_is_fp32, int inputs_on_device, uint64_t seed, int mode,
                    const ns_env* env) {
  if (!out) return NS_ERR_INVALID_ARG;
  *out = nullptr;
  if (m < 0 || n <= 0 || !rowptr || (mode != NS_MODE_NORMAL && mode != NS_MODE_SPD)) return NS_ERR_INVALID_ARG;
  if (vals_is_fp32 != 0 && vals_is_fp32 != 1) return NS_ERR_INVALID_ARG;
  if (mode == NS_MODE_SPD && m != n) return NS_ERR_INVALID_ARG;
  if (n > (int64_t)INT32_MAX || m > (int64_t)INT32_MAX) return NS_ERR_INVALID_ARG;
  const double* vals64 = static_cast<const double*>(vals);
  const float* vals32 = static_cast<const float*>(vals);
  auto value_at = [&](int64_t k) { return vals_is_fp32 ? (double)vals32[k] : vals64[k]; };
  if (!inputs_on_device) {  // host inputs are validated before any device work
    if (rowptr[0] != 0) return NS_ERR_INVALID_ARG;
    for (int64_t r = 0; r < m; ++r)
      if (rowptr[r + 1] < rowptr[r]) return NS_ERR_INVALID_ARG;
    const int64_t nz = rowptr[m];
    if (nz > 0 && (!colind || !vals)) return NS_ERR_INVALID_ARG;
    for (int64_t k = 0; k < nz; ++k)
      if (colind[k] < 0 || (int64_t)colind[k] >= n || !std::isfinite(value_at(k))) return NS_ERR_INVALID_ARG;
  }
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return NS_ERR_CUDA;
  }
  ns_handle* h = new ns_handle();
  h->m = m;
  h->n = n;
  h->mode = mode;
  h->seed = seed;
  if (env) {
    h->env = *env;
    h->own_alloc = (env->alloc == nullptr || env->free == nullptr);
    h->stream = (cudaStream_t)env->stream;
  }
  cudaGetDevice(&dev);
  try {
    int64_t nnz = 0;
    std::vector<int64_t> rp_h;
    if (!inputs_on_device) {
      // full host-side validation
      if (rowptr[0] != 0) throw Fail{NS_ERR_INVALID_ARG, "rowptr[0] != 0"};
      for (int64_t r = 0; r < m; ++r)
        if (rowptr[r + 1] < rowptr[r]) throw Fail{NS_ERR_INVALID_ARG, "rowptr not monotone"};
      nnz = rowptr[m];
      if (nnz > 0 && (!colind || !vals)) throw Fail{NS_ERR_INVALID_ARG, "null colind/vals"};
      if (nnz > (int64_t)INT32_MAX * 2) throw Fail{NS_ERR_INVALID_ARG, "nnz too large"};
      for (int64_t k = 0; k < nnz; ++k) {
        if (colind[k] < 0 || (int64_t)colind[k] >= n) throw Fail{NS_ERR_INVALID_ARG, "column index out of range"};
        if (!std::isfinite(value_at(k))) throw Fail{NS_ERR_INVALID_ARG, "non-finite value"};
      }
      for (int64_t r = 0; r < m; ++r) h->maxrow_A = std::max(h->maxrow_A, rowptr[r + 1] - rowptr[r]);
    } else {
      ck(cudaMemcpy(&nnz, rowptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost), "read nnz");
      rp_h.resize(m + 1);
      ck(cudaMemcpy(rp_h.data(), rowptr, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToHost), "read rowptr");
      for (int64_t r = 0; r < m; ++r) h->maxrow_A = std::max(h->maxrow_A, rp_h[r + 1] - rp_h[r]);
      if (nnz < 0) throw Fail{NS_ERR_INVALID_ARG, "negative nnz"};
    }
    h->nnz = nnz;
    cudaStream_t s = h->stream;
    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    h->rowptr = (int64_t*)dalloc_own(h, sizeof(int64_t) * (m + 1));
    h->col = (int*)dalloc_own(h, sizeof(int) * csr_entries(nnz));
    h->val = (double*)dalloc_own(h, sizeof(double) * csr_entries(nnz));
    ck(cudaMemcpyAsync(h->rowptr, rowptr, sizeof(int64_t) * (m + 1), kind, s), "copy rowptr");
    if (vals_is_fp32) {
      // FP32 values are kept as given (the mixed path's copy) and widened exactly on the
      // device for the FP64 path, the transpose and the refinement
      h->val32 = (float*)dalloc_own(h, sizeof(float) * csr_entries(nnz));
      ck(cudaMemsetAsync(h->val32, 0, sizeof(float) * csr_entries(nnz), s), "memset");
    }
    ck(cudaMemsetAsync(h->val, 0, sizeof(double) * csr_entries(nnz), s), "memset");
    if (nnz) {
      ck(cudaMemcpyAsync(h->col, colind, sizeof(int) * nnz, kind, s), "copy colind");
      if (vals_is_fp32) {
        ck(cudaMemcpyAsync(h->val32, vals, sizeof(float) * nnz, kind, s), "copy vals");
        convert_f2d(h->val32, h->val, nnz, s);
        ck_launch("widen vals");
      } else {
        ck(cudaMemcpyAsync(h->val, vals, sizeof(double) * nnz, kind, s), "copy vals");
      }
    }
    Buf small(h, 4096);
    Red red;
    red.part = nullptr;
    Buf rp(h, sizeof(double) * (size_t)kMaxBlocks * 64 + 256);
    red.part = rp.as<double>();
    ck(cudaMemsetAsync(small.p, 0, 4096, s), "memset");
    red.ticket = reinterpret_cast<unsigned*>(small.as<char>() + 1024);
    unsigned* err = reinterpret_cast<unsigned*>(small.as<char>() + 1032);
    double* norms = reinterpret_cast<double*>(small.as<char>() + 2048);
    if (inputs_on_device) {
      csr_validate(h->rowptr, h->col, h->val, m, n, nnz, err, s);
      unsigned e = 0;
      ck(cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
      ck(cudaStreamSynchronize(s), "sync");
      if (e) throw Fail{NS_ERR_INVALID_ARG, "invalid device CSR (code " + std::to_string(e) + ")"};
    }
    csr_max_abs_row_sum(h->rowptr, h->val, m, norms, red, s);
    h->launches += 1;
    build_sell(h, h->rowptr, h->col, h->val, m, nnz, h->sell_A);
    if (mode == NS_MODE_NORMAL) {
      h->rowptr_t = (int64_t*)dalloc_own(h, sizeof(int64_t) * (n + 1));
      h->col_t = (int*)dalloc_own(h, sizeof(int) * csr_entries(nnz));
      h->val_t = (double*)dalloc_own(h, sizeof(double) * csr_entries(nnz));
      Buf wc(h, sizeof(int) * (n + 1)), wcur(h, sizeof(int64_t) * n), wp(h, sizeof(int64_t) * std::max<int64_t>(nnz, 1)),
          wr(h, sizeof(int) * std::max<int64_t>(nnz, 1)), wb(h, sizeof(int64_t) * (n / 4096 + 2));
      TransposeWork tw{wc.as<int>(), wcur.as<int64_t>(), wp.as<int64_t>(), wr.as<int>(), wb.as<int64_t>()};
      csr_transpose(h->rowptr, h->col, h->val, m, n, nnz, h->rowptr_t, h->col_t, h->val_t, tw, s);
      csr_max_abs_row_sum(h->rowptr_t, h->val_t, n, norms + 1, red, s);
      h->launches += 9;
      build_sell(h, h->rowptr_t, h->col_t, h->val_t, n, nnz, h->sell_At);
      std::vector<int64_t> rpt(n + 1);
      ck(cudaMemcpyAsync(rpt.data(), h->rowptr_t, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s), "d2h");
      ck(cudaStreamSynchronize(s), "sync");
      for (int64_t r = 0; r < n; ++r) h->maxrow_At = std::max(h->maxrow_At, rpt[r + 1] - rpt[r]);
    }
    h->D64 = (double*)dalloc_own(h, sizeof(double) * n);
    rng_uniform<double>(seed, 0u, h->D64, n, s);  // Alg. 2 (its perturbed operator): D ~ U[0,1]
    double nr[2] = {0.0, 0.0};
    ck(cudaMemcpyAsync(nr, norms, sizeof(double) * 2, cudaMemcpyDeviceToHost, s), "d2h");
    ck(cudaStreamSynchronize(s), "sync");
    ck_launch("ns_create");
    h->normAinf = nr[0];
    h->normA1 = (mode == NS_MODE_NORMAL) ? nr[1] : nr[0];
  } catch (const Fail& f) {
    const ns_status st = f.st;
    fprintf(stderr, "ns_create: %s\n", f.msg.c_str());
    ns_destroy(h);
    return st;
  }
  *out = h;
  return NS_OK;
}

// Sec. 5.3.1: block size dim K / 16, as the largest supported d that divides dim K
static int block_size_rule(int restart_len) {
  for (int d : {8, 4, 2})
    if (d <= std::max(1, restart_len / 16) && restart_len % d == 0 && restart_len >= 3 * d) return d;
  return 1;
}

// option checks shared by ns_solve and ns_trace_omega (everything the Solver reads)
static ns_status validate_opts(ns_handle* h, const ns_opts& o, int restart_len) {
  if (!(o.eps >= 0.0) || o.stop_factor <= 0.0) return set_err(h, NS_ERR_INVALID_ARG, "bad opts");
  if (!(o.precision == NS_FP64 || o.precision == NS_MIXED) || !(o.fp64_products == 0 || o.fp64_products == 1))
    return set_err(h, NS_ERR_INVALID_ARG, "precision must be NS_FP64 or NS_MIXED; fp64_products 0 or 1");
  if (o.gemm < NS_GEMM_DEFAULT || o.gemm > NS_GEMM_TC_EXACT ||
      (o.precision != NS_MIXED && (o.gemm == NS_GEMM_TC2 || o.gemm == NS_GEMM_TC3)) ||
      (o.precision == NS_MIXED && o.gemm == NS_GEMM_TC_EXACT) ||
      (o.gemm == NS_GEMM_TC_EXACT && !restart_ozaki_supported(restart_len, 1)))
    return set_err(h, NS_ERR_INVALID_ARG,
                   "gemm: 0..4; TC2/TC3 on the mixed path, TC_EXACT on the FP64 path with restart_len <= 208");
  {
    const int sc = o.spmm_schedule;
    if (!(sc == 0 || sc == 1 || sc == 2 || sc == 4 || sc == 8 || sc == kSchedTma || sc == kSchedSell))
      return set_err(h, NS_ERR_INVALID_ARG, "spmm_schedule must be 0, 1, 2, 4, 8, 64 or 128");
    if (o.checkpoint_every < 0 || !(o.resume == 0 || o.resume == 1) ||
        ((o.checkpoint_every > 0 || o.resume) && (!o.checkpoint_path || !*o.checkpoint_path)))
      return set_err(h, NS_ERR_INVALID_ARG, "checkpoint_every >= 0, resume 0 or 1, both need checkpoint_path");
    if (!(o.precond >= 0 && o.precond <= 2) || (o.precond == 1 && h->mode != NS_MODE_SPD) ||
        (o.precond == 2 && h->mode != NS_MODE_NORMAL) ||
        (o.precond == 1 && !(o.precond_shift >= 0.0 && std::isfinite(o.precond_shift))))
      return set_err(h, NS_ERR_INVALID_ARG,
                     "precond: 0, 1 (outer, NS_MODE_SPD, precond_shift >= 0) or 2 (inner, NS_MODE_NORMAL)");
  }
  return NS_OK;
}

ns_status ns_solve(ns_handle* h, int d, int restart_len, double tol, const ns_opts* opts) {
  if (!h) return NS_ERR_INVALID_ARG;
  if (d == 0) d = block_size_rule(restart_len);
  if (!(d == 1 || d == 2 || d == 4 || d == 8)) return set_err(h, NS_ERR_INVALID_ARG, "d must be 0, 1, 2, 4 or 8");
  if (restart_len % d || restart_len < 3 * d || restart_len > 512)
    return set_err(h, NS_ERR_INVALID_ARG, "restart_len must be a multiple of d in [3d, 512]");
  if (!(tol > 0.0)) return set_err(h, NS_ERR_INVALID_ARG, "tol must be positive");
  ns_opts o;
  ns_default_opts(&o);
  if (opts) o = *opts;
  {
    const ns_status vs = validate_opts(h, o, restart_len);
    if (vs != NS_OK) return vs;
  }
  h->err.clear();
  h->solved = false;
  h->launches = 0;
  try {
    ns_status st;
    if (o.precond == 1) build_precond(h, o.precond_shift);
    if (o.precond == 2) build_inner(h);
    if (o.precision == NS_MIXED) {
      ensure_fp32(h);
      switch (d) {
        case 1: st = solve_typed<float, 1>(h, restart_len, tol, o); break;
        case 2: st = solve_typed<float, 2>(h, restart_len, tol, o); break;
        case 4: st = solve_typed<float, 4>(h, restart_len, tol, o); break;
        default: st = solve_typed<float, 8>(h, restart_len, tol, o); break;
      }
    } else {
      switch (d) {
        case 1: st = solve_typed<double, 1>(h, restart_len, tol, o); break;
        case 2: st = solve_typed<double, 2>(h, restart_len, tol, o); break;
        case 4: st = solve_typed<double, 4>(h, restart_len, tol, o); break;
        default: st = solve_typed<double, 8>(h, restart_len, tol, o); break;
      }
    }
    h->stats.kernel_launches = h->launches;
    if (spmm_wait_timeouts(true)) {
      h->solved = false;
      return set_err(h, NS_ERR_TIMEOUT, "a bounded device wait of the SpMM expired; results discarded");
    }
    return st;
  } catch (const Fail& f) {
    cudaGetLastError();
    return set_err(h, f.st, f.msg);
  }
}

ns_status ns_read_checkpoint(const char* path, ns_checkpoint_info* info) {
  if (!path || !info) return NS_ERR_INVALID_ARG;
  CkptReader r;
  ns_checkpoint_info c{};
  const ns_status st = r.open(path, &c);
  if (st != NS_OK) return st;
  if (!r.skip_rest() || !r.finish()) return NS_ERR_IO;
  *info = c;
  return NS_OK;
}

ns_status ns_nullity(const ns_handle* h, int64_t* N) {
  if (!h || !N) return NS_ERR_INVALID_ARG;
  if (!h->solved) return NS_ERR_STATE;
  *N = h->N;
  return NS_OK;
}

ns_status ns_basis(const ns_handle* hc, double* out, int64_t ld, int out_on_device) {
  ns_handle* h = const_cast<ns_handle*>(hc);
  if (!h || (!out && h->N)) return NS_ERR_INVALID_ARG;
  if (!h->solved) return NS_ERR_STATE;
  if (ld < h->n) return set_err(h, NS_ERR_INVALID_ARG, "ld < n");
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  try {
    if (h->N)
      ck(cudaMemcpy2DAsync(out, sizeof(double) * ld, h->basis, sizeof(double) * h->n, sizeof(double) * h->n, h->N,
                           kind, h->stream),
         "copy basis");
    ck(cudaStreamSynchronize(h->stream), "sync");
  } catch (const Fail& f) {
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_stats(const ns_handle* h, ns_stats_t* s) {
  if (!h || !s) return NS_ERR_INVALID_ARG;
  if (!h->solved) return NS_ERR_STATE;
  *s = h->stats;
  return NS_OK;
}

ns_status ns_profile(const ns_handle* h, ns_kernel_prof* out, int max, int* count) {
  if (!h || !out || !count) return NS_ERR_INVALID_ARG;
  if (!h->solved) return NS_ERR_STATE;
  const Prof& p = h->prof;
  int k = 0;
  for (int c = 0; c < Prof::NC && k < max; ++c, ++k) {
    ns_kernel_prof& r = out[k];
    std::memset(&r, 0, sizeof(r));
    std::snprintf(r.name, sizeof(r.name), "%s", kProfNames[c]);
    r.launches = p.units[c];
    r.sampled = p.sampled[c];
    r.ms_per_launch = p.sampled[c] ? p.ms[c] / (double)p.sampled[c] : 0.0;
    r.bytes_per_launch = p.units[c] ? p.bytes[c] / (double)p.units[c] : 0.0;
    r.flops_per_launch = p.units[c] ? p.flops[c] / (double)p.units[c] : 0.0;
    r.ms_total_est = r.ms_per_launch * (double)p.units[c];
  }
  *count = k;
  return NS_OK;
}

const char* ns_last_error(const ns_handle* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

void ns_destroy(ns_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& pr : h->owned) dfree(h, pr.first, pr.second);
  h->owned.clear();
  dfree(h, h->basis, h->basis_bytes);
  delete h;
}

// ---------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------
ns_status ns_get_transpose(const ns_handle* h, int64_t* rowptr, int32_t* colind, double* vals) {
  if (!h || !rowptr) return NS_ERR_INVALID_ARG;
  if (h->mode != NS_MODE_NORMAL) return NS_ERR_STATE;
  cudaStream_t s = h->stream;
  if (cudaMemcpyAsync(rowptr, h->rowptr_t, sizeof(int64_t) * (h->n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return NS_ERR_CUDA;
  if (h->nnz) {
    if (!colind || !vals) return NS_ERR_INVALID_ARG;
    cudaMemcpyAsync(colind, h->col_t, sizeof(int) * h->nnz, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(vals, h->val_t, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost, s);
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

ns_status ns_get_perturbation(const ns_handle* h, double* D) {
  if (!h || !D) return NS_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(D, h->D64, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return NS_ERR_CUDA;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

ns_status ns_start_block(const ns_handle* hc, int d, double* Omega) {
  ns_handle* h = const_cast<ns_handle*>(hc);
  if (!h || !Omega || d < 1 || d > 8) return NS_ERR_INVALID_ARG;
  try {
    Buf b(h, sizeof(double) * h->n * d);
    rng_gauss<double>(h->seed, 1u, b.as<double>(), h->n * d, h->stream);
    ck_launch("rng");
    ck(cudaMemcpyAsync(Omega, b.p, sizeof(double) * h->n * d, cudaMemcpyDeviceToHost, h->stream), "d2h");
    ck(cudaStreamSynchronize(h->stream), "sync");
  } catch (const Fail& f) {
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_apply_B(ns_handle* h, int d, const double* X, double* Y, double eps, int precision, int on_device,
                     int schedule) {
  if (!h || !X || !Y || !(d == 1 || d == 2 || d == 4 || d == 8)) return NS_ERR_INVALID_ARG;
  if (!(schedule == -1 || schedule == kSchedTma || schedule == kSchedSell || schedule == 1 || schedule == 2 ||
        schedule == 4 || schedule == 8 || schedule == 16 || schedule == 32))
    return set_err(h, NS_ERR_INVALID_ARG, "schedule must be -1, 64, 128 or a power of two up to 32");
  if (schedule == kSchedSell && (!h->sell_A.sptr || (h->mode == NS_MODE_NORMAL && !h->sell_At.sptr)))
    return set_err(h, NS_ERR_INVALID_ARG, "no sliced-ELLPACK copy for this matrix (padding above 30%)");
  try {
    const size_t cnt = (size_t)h->n * d;
    Buf xb(h, sizeof(double) * cnt), yb(h, sizeof(double) * cnt), rp(h, sizeof(double) * kMaxBlocks * 64 + 256),
        tk(h, 256);
    ck(cudaMemsetAsync(tk.p, 0, 256, h->stream), "memset");
    Red red;
    red.part = rp.as<double>();
    red.ticket = tk.as<unsigned>();
    ck(cudaMemcpyAsync(xb.p, X, sizeof(double) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream),
       "copy X");
    if (precision == NS_MIXED) {
      ensure_fp32(h);
      Buf xf(h, sizeof(float) * cnt), yf(h, sizeof(float) * cnt);
      convert_d2f(xb.as<double>(), xf.as<float>(), (int64_t)cnt, h->stream);
      switch (d) {
        case 1: apply_B_typed<float, 1>(h, xf.as<float>(), yf.as<float>(), eps, red, schedule); break;
        case 2: apply_B_typed<float, 2>(h, xf.as<float>(), yf.as<float>(), eps, red, schedule); break;
        case 4: apply_B_typed<float, 4>(h, xf.as<float>(), yf.as<float>(), eps, red, schedule); break;
        default: apply_B_typed<float, 8>(h, xf.as<float>(), yf.as<float>(), eps, red, schedule); break;
      }
      convert_f2d(yf.as<float>(), yb.as<double>(), (int64_t)cnt, h->stream);
      ck(cudaStreamSynchronize(h->stream), "sync");
    } else {
      switch (d) {
        case 1: apply_B_typed<double, 1>(h, xb.as<double>(), yb.as<double>(), eps, red, schedule); break;
        case 2: apply_B_typed<double, 2>(h, xb.as<double>(), yb.as<double>(), eps, red, schedule); break;
        case 4: apply_B_typed<double, 4>(h, xb.as<double>(), yb.as<double>(), eps, red, schedule); break;
        default: apply_B_typed<double, 8>(h, xb.as<double>(), yb.as<double>(), eps, red, schedule); break;
      }
    }
    ck(cudaMemcpyAsync(Y, yb.p, sizeof(double) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream),
       "copy Y");
    ck(cudaStreamSynchronize(h->stream), "sync");
    if (spmm_wait_timeouts(true)) throw Fail{NS_ERR_TIMEOUT, "a bounded device wait of the SpMM expired"};
  } catch (const Fail& f) {
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_precond_build(ns_handle* h, double shift, int32_t* color, int64_t* perm, int64_t* nnz_L,
                           int32_t* ncolors) {
  if (!h) return NS_ERR_INVALID_ARG;
  if (h->mode != NS_MODE_SPD) return set_err(h, NS_ERR_STATE, "outer preconditioning needs NS_MODE_SPD");
  if (!(shift >= 0.0 && std::isfinite(shift))) return set_err(h, NS_ERR_INVALID_ARG, "shift must be >= 0");
  try {
    build_precond(h, shift);
    const auto& P = h->pc;
    if (color) std::copy(P.color_h.begin(), P.color_h.end(), color);
    if (perm) std::copy(P.perm_h.begin(), P.perm_h.end(), perm);
    if (nnz_L) *nnz_L = P.nnzL;
    if (ncolors) *ncolors = P.ncolors;
  } catch (const Fail& f) {
    cudaGetLastError();
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_inner_precond(ns_handle* h, double* row_scale) {
  if (!h) return NS_ERR_INVALID_ARG;
  if (h->mode != NS_MODE_NORMAL) return set_err(h, NS_ERR_STATE, "inner preconditioning needs NS_MODE_NORMAL");
  try {
    build_inner(h);
    if (row_scale && h->m)
      ck(cudaMemcpy(row_scale, h->inner.s, sizeof(double) * h->m, cudaMemcpyDeviceToHost), "d2h");
  } catch (const Fail& f) {
    cudaGetLastError();
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_precond_factor(const ns_handle* h, int64_t* rowptr, int32_t* colind, double* vals) {
  if (!h || !rowptr) return NS_ERR_INVALID_ARG;
  const auto& P = h->pc;
  if (!P.built || P.alpha < 0.0) return NS_ERR_STATE;
  cudaStream_t s = h->stream;
  if (cudaMemcpyAsync(rowptr, P.lrp, sizeof(int64_t) * (h->n + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return NS_ERR_CUDA;
  if (P.nnzL) {
    if (!colind || !vals) return NS_ERR_INVALID_ARG;
    cudaMemcpyAsync(colind, P.lcol, sizeof(int) * P.nnzL, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(vals, P.lval, sizeof(double) * P.nnzL, cudaMemcpyDeviceToHost, s);
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

ns_status ns_apply_precond(ns_handle* h, int d, const double* X, double* Y, double eps, int precision,
                           int on_device) {
  if (!h || !X || !Y || !(d == 1 || d == 2 || d == 4 || d == 8)) return NS_ERR_INVALID_ARG;
  if (!(precision == NS_FP64 || precision == NS_MIXED)) return set_err(h, NS_ERR_INVALID_ARG, "precision");
  const int kind = h->mode == NS_MODE_SPD ? 1 : 2;
  if (kind == 1 && (!h->pc.built || h->pc.alpha < 0.0))
    return set_err(h, NS_ERR_STATE, "no preconditioner: ns_precond_build first");
  if (kind == 2 && !h->inner.built) return set_err(h, NS_ERR_STATE, "no preconditioner: ns_inner_precond first");
  try {
    const size_t cnt = (size_t)h->n * d;
    Buf xb(h, sizeof(double) * cnt), yb(h, sizeof(double) * cnt), rp(h, sizeof(double) * kMaxBlocks * 64 + 256),
        tk(h, 256);
    ck(cudaMemsetAsync(tk.p, 0, 256, h->stream), "memset");
    Red red;
    red.part = rp.as<double>();
    red.ticket = tk.as<unsigned>();
    ck(cudaMemcpyAsync(xb.p, X, sizeof(double) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream),
       "copy X");
    if (precision == NS_MIXED) {
      ensure_fp32(h);
      Buf xf(h, sizeof(float) * cnt), yf(h, sizeof(float) * cnt);
      convert_d2f(xb.as<double>(), xf.as<float>(), (int64_t)cnt, h->stream);
      switch (d) {
        case 1: apply_B_typed<float, 1>(h, xf.as<float>(), yf.as<float>(), eps, red, -1, kind); break;
        case 2: apply_B_typed<float, 2>(h, xf.as<float>(), yf.as<float>(), eps, red, -1, kind); break;
        case 4: apply_B_typed<float, 4>(h, xf.as<float>(), yf.as<float>(), eps, red, -1, kind); break;
        default: apply_B_typed<float, 8>(h, xf.as<float>(), yf.as<float>(), eps, red, -1, kind); break;
      }
      convert_f2d(yf.as<float>(), yb.as<double>(), (int64_t)cnt, h->stream);
    } else {
      switch (d) {
        case 1: apply_B_typed<double, 1>(h, xb.as<double>(), yb.as<double>(), eps, red, -1, kind); break;
        case 2: apply_B_typed<double, 2>(h, xb.as<double>(), yb.as<double>(), eps, red, -1, kind); break;
        case 4: apply_B_typed<double, 4>(h, xb.as<double>(), yb.as<double>(), eps, red, -1, kind); break;
        default: apply_B_typed<double, 8>(h, xb.as<double>(), yb.as<double>(), eps, red, -1, kind); break;
      }
    }
    ck(cudaMemcpyAsync(Y, yb.p, sizeof(double) * cnt, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream),
       "copy Y");
    ck(cudaStreamSynchronize(h->stream), "sync");
  } catch (const Fail& f) {
    cudaGetLastError();
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_restart_product(int64_t n, int d, int R, const double* Z, const double* VZ, const int32_t* sel, int nsel,
                             int nl, int precision, int gemm, double* out) {
  if (n < 1 || !(d == 1 || d == 2 || d == 4 || d == 8) || R < 1 || R > 512 || R % d || nsel < 1 || nl < 0 ||
      nl > nsel || (nsel - nl) % d || !Z || !VZ || !sel || !out || gemm < 0 || gemm > NS_GEMM_TC_EXACT ||
      (precision != NS_FP64 && precision != NS_MIXED))
    return NS_ERR_INVALID_ARG;
  if (precision == NS_FP64 && (gemm == NS_GEMM_TC2 || gemm == NS_GEMM_TC3)) return NS_ERR_INVALID_ARG;
  if (precision == NS_MIXED && gemm == NS_GEMM_TC_EXACT) return NS_ERR_INVALID_ARG;
  for (int c = 0; c < nsel; ++c)
    if (sel[c] < 0 || sel[c] >= R) return NS_ERR_INVALID_ARG;
  ns_handle tmp;
  try {
    if (precision == NS_MIXED)
      restart_product_typed<float>(&tmp, n, d, R, Z, VZ, sel, nsel, nl, gemm, out);
    else
      restart_product_typed<double>(&tmp, n, d, R, Z, VZ, sel, nsel, nl, gemm, out);
  } catch (const Fail& f) {
    cudaGetLastError();
    fprintf(stderr, "ns_restart_product: %s\n", f.msg.c_str());
    return f.st;
  }
  return NS_OK;
}

ns_status ns_trace_omega(ns_handle* h, int d, int restart_len, const ns_opts* opts, double* W) {
  if (!h || !W) return NS_ERR_INVALID_ARG;
  if (!(d == 1 || d == 2 || d == 4 || d == 8)) return set_err(h, NS_ERR_INVALID_ARG, "d must be 1, 2, 4 or 8");
  if (restart_len % d || restart_len < 3 * d || restart_len > 512)
    return set_err(h, NS_ERR_INVALID_ARG, "restart_len must be a multiple of d in [3d, 512]");
  ns_opts o;
  ns_default_opts(&o);
  if (opts) o = *opts;
  {
    const ns_status vs = validate_opts(h, o, restart_len);
    if (vs != NS_OK) return vs;
  }
  o.checkpoint_every = 0;  // the first cycle only: no restart, nothing to save or resume
  o.resume = 0;
  try {
    if (o.precond == 1) build_precond(h, o.precond_shift);
    if (o.precond == 2) build_inner(h);
    if (o.precision == NS_MIXED) {
      ensure_fp32(h);
      switch (d) {
        case 1: trace_omega_typed<float, 1>(h, restart_len, o, W); break;
        case 2: trace_omega_typed<float, 2>(h, restart_len, o, W); break;
        case 4: trace_omega_typed<float, 4>(h, restart_len, o, W); break;
        default: trace_omega_typed<float, 8>(h, restart_len, o, W); break;
      }
    } else {
      switch (d) {
        case 1: trace_omega_typed<double, 1>(h, restart_len, o, W); break;
        case 2: trace_omega_typed<double, 2>(h, restart_len, o, W); break;
        case 4: trace_omega_typed<double, 4>(h, restart_len, o, W); break;
        default: trace_omega_typed<double, 8>(h, restart_len, o, W); break;
      }
    }
    if (spmm_wait_timeouts(true)) throw Fail{NS_ERR_TIMEOUT, "a bounded device wait of the SpMM expired"};
  } catch (const Fail& f) {
    cudaGetLastError();
    return set_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_syev(int k, const double* T, double* theta, double* V) {
  if (k < 1 || k > 512 || !T || !theta || !V) return NS_ERR_INVALID_ARG;
  ns_handle tmp;
  try {
    Buf bt(&tmp, sizeof(double) * k * k), bth(&tmp, sizeof(double) * k), bv(&tmp, sizeof(double) * k * k),
        bw(&tmp, sizeof(double) * syev_work_doubles(k));
    ck(cudaMemcpy(bt.p, T, sizeof(double) * k * k, cudaMemcpyHostToDevice), "h2d");
    syev(bt.as<double>(), k, bth.as<double>(), bv.as<double>(), bw.as<double>(), nullptr);
    ck_launch("syev");
    ck(cudaDeviceSynchronize(), "sync");
    ck(cudaMemcpy(theta, bth.p, sizeof(double) * k, cudaMemcpyDeviceToHost), "d2h");
    ck(cudaMemcpy(V, bv.p, sizeof(double) * k * k, cudaMemcpyDeviceToHost), "d2h");
  } catch (const Fail& f) {
    return f.st;
  }
  return NS_OK;
}

ns_status ns_project(int64_t n, int K, int w, const double* V, double* Wm, double* C, int precision) {
  if (n < 1 || K < 1 || !(w == 1 || w == 2 || w == 4 || w == 8) || !V || !Wm || !C) return NS_ERR_INVALID_ARG;
  if (precision != NS_FP64 && precision != NS_MIXED && precision != NS_FP64_PAIRS) return NS_ERR_INVALID_ARG;
  const int df = precision == NS_FP64_PAIRS ? 1 : 0;
  ns_handle tmp;
  tmp.n = n;
  try {
    if (precision == NS_MIXED) {
      switch (w) {
        case 1: project_typed<float, 1>(&tmp, n, K, V, Wm, C, 0); break;
        case 2: project_typed<float, 2>(&tmp, n, K, V, Wm, C, 0); break;
        case 4: project_typed<float, 4>(&tmp, n, K, V, Wm, C, 0); break;
        default: project_typed<float, 8>(&tmp, n, K, V, Wm, C, 0); break;
      }
    } else {
      switch (w) {
        case 1: project_typed<double, 1>(&tmp, n, K, V, Wm, C, df); break;
        case 2: project_typed<double, 2>(&tmp, n, K, V, Wm, C, df); break;
        case 4: project_typed<double, 4>(&tmp, n, K, V, Wm, C, df); break;
        default: project_typed<double, 8>(&tmp, n, K, V, Wm, C, df); break;
      }
    }
  } catch (const Fail& f) {
    return f.st;
  }
  return NS_OK;
}

}  // extern "C"

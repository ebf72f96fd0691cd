// Host driver of the batched persistent form: ingest of many CSR matrices into
// one concatenated device layout, the per-CTA workspace, the SpMV-lane
// autotuner, the CUDA graph holding {queue reset, persistent launch}, and the
// ns_batch_* C entry points.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <map>
#include <mutex>
#include <tuple>

#include "../../include/nullspace.h"
#include "ns_batch.cuh"
#include "ns_kernels.cuh"

struct ns_batch {
  ns_env env{};
  bool own_alloc = true;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int64_t count = 0;
  int nmax = 0;
  uint64_t seed = 0;
  std::vector<int64_t> n_h, nnz_h, out_off_h;
  std::vector<std::pair<void*, size_t>> allocs;  // freed by ns_batch_destroy
  // device arrays
  int64_t* rowptr = nullptr;
  int* col = nullptr;
  float* val = nullptr;
  double* val64 = nullptr;
  int64_t *rp_off = nullptr, *nz_off = nullptr, *out_off = nullptr;
  int *nrows = nullptr, *order = nullptr, *order_sample = nullptr;
  int sample_count = 0;
  double* basis = nullptr;
  int *nullity = nullptr, *status = nullptr;
  long long* istats = nullptr;
  unsigned* queue = nullptr;
  // workspace (per CTA slot), grown on demand
  float* ws32 = nullptr;
  double* ws64 = nullptr;
  size_t ws32_bytes = 0, ws64_bytes = 0;
  // schedule
  int lanes = 0, bps = 0, grid = 0, tuned_block = 0;
  double t_tune_ms = 0.0;
  // graph of the last solve
  cudaGraphExec_t gexec = nullptr;
  ns::BatchArgs gargs{};
  int glanes = 0, ggrid = 0, gblock = 0;
  // results
  bool solved = false;
  std::vector<int> nullity_h, status_h;
  std::vector<long long> istats_h;
  ns_batch_stats_t stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

struct BFail {
  ns_status st;
  std::string msg;
};

void bck_at(cudaError_t e, const char* what, int line) {
  if (e != cudaSuccess)
    throw BFail{NS_ERR_CUDA, std::string(what) + " (ns_batch.cu:" + std::to_string(line) + "): " + cudaGetErrorString(e)};
}
#define bck(e, what) bck_at((e), (what), __LINE__)

void* balloc(ns_batch* h, size_t bytes) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (!h->own_alloc) {
    p = h->env.alloc(bytes, h->env.ctx);
    if (!p) throw BFail{NS_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes"};
  } else {
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw BFail{NS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    }
  }
  h->allocs.emplace_back(p, bytes);
  return p;
}

void bfree(ns_batch* h, void* p) {
  if (!p) return;
  for (size_t k = 0; k < h->allocs.size(); ++k)
    if (h->allocs[k].first == p) {
      if (!h->own_alloc)
        h->env.free(p, h->allocs[k].second, h->env.ctx);
      else
        cudaFree(p);
      h->allocs.erase(h->allocs.begin() + (long)k);
      return;
    }
}

template <typename T>
T* bput(ns_batch* h, const T* src, size_t cnt) {
  T* d = static_cast<T*>(balloc(h, cnt * sizeof(T)));
  if (cnt) bck(cudaMemcpyAsync(d, src, cnt * sizeof(T), cudaMemcpyHostToDevice, h->stream), "H2D copy");
  return d;
}

ns_status bset_err(ns_batch* h, ns_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

void drop_graph(ns_batch* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
}

bool same_args(const ns::BatchArgs& a, const ns::BatchArgs& b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

// Autotuner results shared by every handle of the process, per shape class: device,
// CTA size, restart length, mean row length (quarter steps) and the largest
// instance (powers of two).  A new batch of the same class skips the tuning runs.
using TuneKey = std::tuple<int, int, int, int64_t, int>;
std::mutex g_tune_mutex;
std::map<TuneKey, int> g_tune_cache;

TuneKey tune_key(const ns_batch* h, int dev, int block, int R) {
  int64_t rows = 0, nz = 0;
  for (int64_t i = 0; i < h->count; ++i) {
    rows += h->n_h[i];
    nz += h->nnz_h[i];
  }
  const int64_t len4 = rows ? (4 * nz + rows / 2) / rows : 0;
  int lg = 0;
  while ((1 << lg) < h->nmax) ++lg;
  return TuneKey(dev, block, R, len4, lg);
}

}  // namespace

extern "C" {

ns_status ns_batch_create(ns_batch** out, int64_t count, const int64_t* n, const int64_t* rowptr,
                          const int32_t* colind, const void* vals, int vals_is_fp32, uint64_t seed,
                          const ns_env* env) {
  if (!out) return NS_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || count > (int64_t)0x7fffffff || !n || !rowptr) return NS_ERR_INVALID_ARG;
  if (vals_is_fp32 != 0 && vals_is_fp32 != 1) return NS_ERR_INVALID_ARG;
  // host-side structure checks (nothing is allocated before they pass)
  std::vector<int64_t> nnz(count), rp_off(count), nz_off(count), out_off(count);
  int64_t rp_tot = 0, nz_tot = 0, nmax = 0, basis_tot = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > (int64_t)0x7fffffff) return NS_ERR_INVALID_ARG;
    const int64_t* rp = rowptr + rp_tot;
    if (rp[0] != 0) return NS_ERR_INVALID_ARG;
    for (int64_t r = 0; r < n[i]; ++r)
      if (rp[r + 1] < rp[r]) return NS_ERR_INVALID_ARG;
    nnz[i] = rp[n[i]];
    rp_off[i] = rp_tot;
    nz_off[i] = nz_tot;
    out_off[i] = basis_tot;
    rp_tot += n[i] + 1;
    nz_tot += nnz[i];
    basis_tot += n[i] * ns::kBMaxLock;
    nmax = std::max(nmax, n[i]);
  }
  if (nz_tot > 0 && (!colind || !vals)) return NS_ERR_INVALID_ARG;
  // the row structure is checked above on the host; the entries (columns, values)
  // are checked on the device right after the copy
  ns_batch* h = new ns_batch();
  if (env && env->alloc) {
    h->env = *env;
    h->own_alloc = false;
  }
  try {
    if (env && env->stream) {
      h->stream = static_cast<cudaStream_t>(env->stream);
    } else {
      bck(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "cudaStreamCreate");
      h->own_stream = true;
    }
    bck(cudaEventCreate(&h->ev0), "cudaEventCreate");
    bck(cudaEventCreate(&h->ev1), "cudaEventCreate");
    h->count = count;
    h->nmax = (int)nmax;
    h->seed = seed;
    h->n_h.assign(n, n + count);
    h->nnz_h = nnz;
    h->out_off_h = out_off;
    std::vector<int> nrows(count);
    for (int64_t i = 0; i < count; ++i) nrows[i] = (int)n[i];
    // largest instances first, so the tail of the queue holds the short ones
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nnz[a] + n[a] > nnz[b] + n[b]; });
    h->rowptr = bput(h, rowptr, (size_t)rp_tot);
    h->col = bput(h, reinterpret_cast<const int*>(colind), (size_t)nz_tot);
    if (vals_is_fp32) {  // FP32 values as given; an exact FP64 widening for the refinement
      h->val = bput(h, static_cast<const float*>(vals), (size_t)nz_tot);
      h->val64 = static_cast<double*>(balloc(h, sizeof(double) * (size_t)std::max<int64_t>(nz_tot, 1)));
      ns::convert_f2d(h->val, h->val64, nz_tot, h->stream);
    } else {
      h->val64 = bput(h, static_cast<const double*>(vals), (size_t)nz_tot);
      h->val = static_cast<float*>(balloc(h, sizeof(float) * (size_t)std::max<int64_t>(nz_tot, 1)));
      ns::convert_d2f(h->val64, h->val, nz_tot, h->stream);
    }
    h->rp_off = bput(h, rp_off.data(), (size_t)count);
    h->nz_off = bput(h, nz_off.data(), (size_t)count);
    h->out_off = bput(h, out_off.data(), (size_t)count);
    h->nrows = bput(h, nrows.data(), (size_t)count);
    h->order = bput(h, order.data(), (size_t)count);
    // autotuner sample: instances evenly spaced through the size order
    const int S = (int)std::min<int64_t>(count, 256);
    std::vector<int> smp(S);
    for (int k = 0; k < S; ++k) smp[k] = order[(size_t)((int64_t)k * count / S)];
    h->order_sample = bput(h, smp.data(), (size_t)S);
    h->sample_count = S;
    h->basis = static_cast<double*>(balloc(h, sizeof(double) * (size_t)basis_tot));
    h->nullity = static_cast<int*>(balloc(h, sizeof(int) * (size_t)count));
    h->status = static_cast<int*>(balloc(h, sizeof(int) * (size_t)count));
    h->istats = static_cast<long long*>(balloc(h, sizeof(long long) * ns::kBStats * (size_t)count));
    h->queue = static_cast<unsigned*>(balloc(h, 256));
    {  // entry checks on the device
      ns::BatchArgs va;
      std::memset(&va, 0, sizeof(va));
      va.rowptr = h->rowptr;
      va.rp_off = h->rp_off;
      va.nz_off = h->nz_off;
      va.nrows = h->nrows;
      va.col = h->col;
      va.val64 = h->val64;
      va.count = (int)count;
      unsigned* err = h->queue + 32;  // spare word of the queue's 256-byte block
      bck(cudaMemsetAsync(err, 0, sizeof(unsigned), h->stream), "memset");
      ns::batch_validate(va, err, h->stream);
      bck(cudaGetLastError(), "k_batch_validate");
      unsigned e = 0;
      bck(cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream), "d2h");
      bck(cudaStreamSynchronize(h->stream), "ingest");
      if (e) throw BFail{NS_ERR_INVALID_ARG, "column index out of range or non-finite value"};
    }
  } catch (const BFail& f) {
    ns_batch_destroy(h);
    return f.st;
  }
  *out = h;
  return NS_OK;
}

ns_status ns_batch_solve(ns_batch* h, int d, int restart_len, double tol, const ns_opts* opts) {
  if (!h) return NS_ERR_INVALID_ARG;
  if (d != 1) return bset_err(h, NS_ERR_INVALID_ARG, "the batched form takes d = 1");
  if (restart_len < 8 || restart_len > ns::kBMaxR)
    return bset_err(h, NS_ERR_INVALID_ARG, "restart_len must be in [8, 64]");
  if (!(tol > 0.0)) return bset_err(h, NS_ERR_INVALID_ARG, "tol must be positive");
  const int64_t nmin = *std::min_element(h->n_h.begin(), h->n_h.end());
  if (nmin < restart_len + ns::kBMaxLock + 2)
    return bset_err(h, NS_ERR_INVALID_ARG, "every instance needs n >= restart_len + 34");
  ns_opts o;
  ns_default_opts(&o);
  if (opts) o = *opts;
  // eps > 0: the batched kernel counts Ritz values below 3 eps as null (no unperturbed variant)
  if (!(o.eps > 0.0) || !(o.stop_factor > 0.0) || !(o.refine_tol > 0.0) || o.refine_maxit < 0)
    return bset_err(h, NS_ERR_INVALID_ARG, "bad opts");
  if (!(o.batch_block == 0 || o.batch_block == 128 || o.batch_block == 256))
    return bset_err(h, NS_ERR_INVALID_ARG, "batch_block must be 0, 128 or 256");
  const int block = o.batch_block ? o.batch_block : 128;
  const int R = restart_len;
  try {
    int dev = 0, sms = 0;
    bck(cudaGetDevice(&dev), "cudaGetDevice");
    bck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    int bps[5] = {0, 0, 0, 0, 0};
    for (int L : {1, 2, 4}) {
      bck(ns::batched_prepare(L, block, R, &bps[L]), "batched_prepare");
      if (bps[L] < 1) throw BFail{NS_ERR_CUDA, "batched kernel does not fit on an SM"};
    }
    const int bps_max = std::max(bps[1], std::max(bps[2], bps[4]));
    const int slots = (int)std::min<int64_t>(h->count, (int64_t)bps_max * sms);
    const int64_t s32 = (int64_t)((ns::batched_ws32_per_slot(h->nmax, R) + 63) / 64 * 64);
    const int64_t s64 = (int64_t)((ns::batched_ws64_per_slot(h->nmax) + 31) / 32 * 32);
    const size_t need32 = sizeof(float) * (size_t)s32 * slots, need64 = sizeof(double) * (size_t)s64 * slots;
    if (need32 > h->ws32_bytes) {
      bfree(h, h->ws32);
      h->ws32 = nullptr;
      h->ws32 = static_cast<float*>(balloc(h, need32));
      h->ws32_bytes = need32;
    }
    if (need64 > h->ws64_bytes) {
      bfree(h, h->ws64);
      h->ws64 = nullptr;
      h->ws64 = static_cast<double*>(balloc(h, need64));
      h->ws64_bytes = need64;
    }
    ns::BatchArgs a;
    std::memset(&a, 0, sizeof(a));  // padding too: the graph cache compares bytes
    a.rowptr = h->rowptr;
    a.col = h->col;
    a.val = h->val;
    a.val64 = h->val64;
    a.rp_off = h->rp_off;
    a.nz_off = h->nz_off;
    a.nrows = h->nrows;
    a.out_off = h->out_off;
    a.order = h->order;
    a.count = (int)h->count;
    a.seed = h->seed;
    a.eps = o.eps;
    a.tol = tol;
    a.R = R;
    a.max_matvec = o.max_matvec;
    a.stop_factor = o.stop_factor;
    a.refine_tol = o.refine_tol;
    a.refine_maxit = o.refine_maxit;
    a.ws32 = h->ws32;
    a.ws64 = h->ws64;
    a.ws32_stride = s32;
    a.ws64_stride = s64;
    a.nmax = h->nmax;
    a.basis = h->basis;
    a.nullity = h->nullity;
    a.status = h->status;
    a.istats = h->istats;
    a.queue = h->queue;
    int64_t launches = 0;
    // ---- autotuner: SpMV lanes per row, ranked by the SM cycles the sampled
    // instances take while running side by side (first solve only) ----
    if (h->lanes == 0 || h->tuned_block != block) {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(tune_key(h, dev, block, R));
      if (it != g_tune_cache.end()) {
        h->lanes = it->second;
        h->tuned_block = block;
        h->t_tune_ms = 0.0;
      }
    }
    if (h->lanes == 0 || h->tuned_block != block) {
      ns::BatchArgs t = a;
      t.order = h->order_sample;
      t.count = h->sample_count;
      std::vector<long long> st((size_t)ns::kBStats * h->count);
      std::vector<int> smp(h->sample_count);
      bck(cudaMemcpy(smp.data(), h->order_sample, sizeof(int) * smp.size(), cudaMemcpyDeviceToHost), "sample");
      double best = 0.0;
      int best_l = 1;
      bck(cudaEventRecord(h->ev0, h->stream), "event");
      for (int L : {1, 2, 4}) {
        const int g = (int)std::min<int64_t>(t.count, (int64_t)bps[L] * sms);
        bck(cudaMemsetAsync(h->queue, 0, sizeof(unsigned), h->stream), "queue reset");
        ns::batched_launch(t, L, block, g, h->stream);
        bck(cudaGetLastError(), "k_batched (tuning)");
        launches += 1;
        bck(cudaMemcpyAsync(st.data(), h->istats, sizeof(long long) * st.size(), cudaMemcpyDeviceToHost, h->stream),
            "tuning stats");
        bck(cudaStreamSynchronize(h->stream), "tuning run");
        double cyc = 0.0;
        for (int i : smp) cyc += (double)st[(size_t)ns::kBStats * i + 4];
        if (L == 1 || cyc < best) {
          best = cyc;
          best_l = L;
        }
      }
      bck(cudaEventRecord(h->ev1, h->stream), "event");
      bck(cudaEventSynchronize(h->ev1), "event");
      float ms = 0.f;
      bck(cudaEventElapsedTime(&ms, h->ev0, h->ev1), "event");
      h->t_tune_ms = ms;
      h->lanes = best_l;
      h->tuned_block = block;
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[tune_key(h, dev, block, R)] = best_l;
    }
    h->bps = bps[h->lanes];
    h->grid = (int)std::min<int64_t>(h->count, (int64_t)h->bps * sms);
    // ---- the solve: graph {queue reset, persistent launch}, re-captured only
    // when an argument changed ----
    const bool want_graph = o.use_graphs >= 0;
    bool replayed = false;
    if (want_graph) {
      if (!h->gexec || !same_args(h->gargs, a) || h->glanes != h->lanes || h->ggrid != h->grid ||
          h->gblock != block) {
        drop_graph(h);
        cudaGraph_t g = nullptr;
        bck(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaMemsetAsync(h->queue, 0, sizeof(unsigned), h->stream);
        ns::batched_launch(a, h->lanes, block, h->grid, h->stream);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
        bck(le, "k_batched (capture)");
        bck(ce, "end capture");
        const cudaError_t ie = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        bck(ie, "graph instantiate");
        h->gargs = a;
        h->glanes = h->lanes;
        h->ggrid = h->grid;
        h->gblock = block;
      }
      bck(cudaEventRecord(h->ev0, h->stream), "event");
      bck(cudaGraphLaunch(h->gexec, h->stream), "graph launch");
      replayed = true;
    } else {
      bck(cudaEventRecord(h->ev0, h->stream), "event");
      bck(cudaMemsetAsync(h->queue, 0, sizeof(unsigned), h->stream), "queue reset");
      ns::batched_launch(a, h->lanes, block, h->grid, h->stream);
      bck(cudaGetLastError(), "k_batched");
    }
    launches += 1;
    bck(cudaEventRecord(h->ev1, h->stream), "event");
    h->nullity_h.resize(h->count);
    h->status_h.resize(h->count);
    h->istats_h.resize((size_t)ns::kBStats * h->count);
    bck(cudaMemcpyAsync(h->nullity_h.data(), h->nullity, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->stream),
        "results");
    bck(cudaMemcpyAsync(h->status_h.data(), h->status, sizeof(int) * h->count, cudaMemcpyDeviceToHost, h->stream),
        "results");
    bck(cudaMemcpyAsync(h->istats_h.data(), h->istats, sizeof(long long) * h->istats_h.size(), cudaMemcpyDeviceToHost,
                        h->stream),
        "results");
    bck(cudaStreamSynchronize(h->stream), "batched solve");
    float ms = 0.f;
    bck(cudaEventElapsedTime(&ms, h->ev0, h->ev1), "event");
    ns_batch_stats_t& S = h->stats;
    S = ns_batch_stats_t{};
    S.count = h->count;
    ns_status ret = NS_OK;
    for (int64_t i = 0; i < h->count; ++i) {
      S.total_nullity += h->nullity_h[i];
      const long long mv = h->istats_h[(size_t)ns::kBStats * i];
      S.matvecs_total += mv;
      S.matvecs_max = std::max<int64_t>(S.matvecs_max, mv);
      const int st = h->status_h[i];
      if (st != 0) {
        ++S.failed;
        if (ret == NS_OK) ret = (st == 7) ? NS_ERR_REFINE : NS_ERR_NOT_CONVERGED;
      }
    }
    S.kernel_launches = launches;
    S.lanes = h->lanes;
    S.grid = h->grid;
    S.blocks_per_sm = h->bps;
    S.block = block;
    S.graph = replayed ? 1 : 0;
    S.t_solve_ms = ms;
    S.t_tune_ms = h->t_tune_ms;
    h->solved = true;
    if (ret != NS_OK) h->err = std::to_string(S.failed) + " instance(s) with a non-zero status";
    return ret;
  } catch (const BFail& f) {
    if (f.st == NS_ERR_CUDA) {
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(h->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(h->stream, &g);
        if (g) cudaGraphDestroy(g);
      }
    }
    return bset_err(h, f.st, f.msg);
  }
}

ns_status ns_batch_results(const ns_batch* h, int32_t* nullity, int32_t* status, int64_t* istats) {
  if (!h) return NS_ERR_INVALID_ARG;
  if (!h->solved) return NS_ERR_STATE;
  for (int64_t i = 0; i < h->count; ++i) {
    if (nullity) nullity[i] = h->nullity_h[i];
    if (status) status[i] = h->status_h[i];
  }
  if (istats)
    for (size_t k = 0; k < h->istats_h.size(); ++k) istats[k] = h->istats_h[k];
  return NS_OK;
}

ns_status ns_batch_basis(const ns_batch* hc, int64_t i, double* out, int64_t ld, int out_on_device) {
  ns_batch* h = const_cast<ns_batch*>(hc);
  if (!h || !out || i < 0 || i >= h->count) return NS_ERR_INVALID_ARG;
  if (!h->solved) return bset_err(h, NS_ERR_STATE, "ns_batch_basis before ns_batch_solve");
  const int64_t n = h->n_h[i];
  if (ld < n) return bset_err(h, NS_ERR_INVALID_ARG, "ld < n_i");
  const int N = h->nullity_h[i];
  if (N == 0) return NS_OK;
  try {
    bck(cudaMemcpy2DAsync(out, sizeof(double) * ld, h->basis + h->out_off_h[i], sizeof(double) * n,
                          sizeof(double) * n, N, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream),
        "basis copy");
    bck(cudaStreamSynchronize(h->stream), "basis copy");
  } catch (const BFail& f) {
    return bset_err(h, f.st, f.msg);
  }
  return NS_OK;
}

ns_status ns_batch_basis_packed(const ns_batch* hc, double* out, int out_on_device) {
  ns_batch* h = const_cast<ns_batch*>(hc);
  if (!h || !out) return NS_ERR_INVALID_ARG;
  if (!h->solved) return bset_err(h, NS_ERR_STATE, "ns_batch_basis_packed before ns_batch_solve");
  std::vector<int64_t> poff(h->count), plen(h->count);
  int64_t tot = 0;
  for (int64_t i = 0; i < h->count; ++i) {
    poff[i] = tot;
    plen[i] = h->n_h[i] * (int64_t)h->nullity_h[i];
    tot += plen[i];
  }
  if (tot == 0) return NS_OK;
  void* dpo = nullptr;
  void* dpl = nullptr;
  void* stage = nullptr;
  try {
    dpo = balloc(h, sizeof(int64_t) * (size_t)h->count);
    dpl = balloc(h, sizeof(int64_t) * (size_t)h->count);
    bck(cudaMemcpyAsync(dpo, poff.data(), sizeof(int64_t) * poff.size(), cudaMemcpyHostToDevice, h->stream), "h2d");
    bck(cudaMemcpyAsync(dpl, plen.data(), sizeof(int64_t) * plen.size(), cudaMemcpyHostToDevice, h->stream), "h2d");
    double* dst = out;
    if (!out_on_device) {
      stage = balloc(h, sizeof(double) * (size_t)tot);
      dst = static_cast<double*>(stage);
    }
    ns::batch_pack(h->basis, h->out_off, static_cast<int64_t*>(dpo), static_cast<int64_t*>(dpl), (int)h->count, dst,
                   h->stream);
    bck(cudaGetLastError(), "k_batch_pack");
    if (!out_on_device)
      bck(cudaMemcpyAsync(out, stage, sizeof(double) * (size_t)tot, cudaMemcpyDeviceToHost, h->stream), "d2h");
    bck(cudaStreamSynchronize(h->stream), "basis pack");
  } catch (const BFail& f) {
    bfree(h, stage);
    bfree(h, dpl);
    bfree(h, dpo);
    return bset_err(h, f.st, f.msg);
  }
  bfree(h, stage);
  bfree(h, dpl);
  bfree(h, dpo);
  return NS_OK;
}

ns_status ns_batch_stats(const ns_batch* h, ns_batch_stats_t* s) {
  if (!h || !s) return NS_ERR_INVALID_ARG;
  if (!h->solved) return NS_ERR_STATE;
  *s = h->stats;
  return NS_OK;
}

const char* ns_batch_last_error(const ns_batch* h) { return h ? h->err.c_str() : "null batch handle"; }

void ns_batch_destroy(ns_batch* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  while (!h->allocs.empty()) bfree(h, h->allocs.back().first);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"

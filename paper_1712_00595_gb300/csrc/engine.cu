// Host engine behind the C ABI of include/osp.h: device memory, the graph
// loader, the per-batch launch sequence and the queries.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <thread>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace osp;

namespace {

constexpr int kIngestSmem = kMaxBatch * 8;
// pinned staging: host ops of a batch first, then the batch size for graph
// replays, then the ||x(i)||_1 history read back with the control block
constexpr size_t kPinnedBytes = 256 * 1024;
constexpr size_t kPinnedBatchSize = sizeof(osp_update) * kMaxBatch;
constexpr size_t kPinnedHist = kPinnedBatchSize + 64;
constexpr size_t kPinnedRes = kPinnedHist + sizeof(double) * kMaxHist;  // per-seed residual bounds
static_assert(kPinnedRes + sizeof(double) * kMaxSeeds <= kPinnedBytes, "pinned staging too small");

struct HostCtlView {  // the leading fields of Ctl, read back after every call
  Ctl c;
};

constexpr int kMaxQuerySlots = 64;
// host-mapped result block of a query slot: scores, ids, count
constexpr size_t kSlotHostBytes = (sizeof(double) + sizeof(int)) * kTopkMaxK + 64;

// Device scratch of one top-k query.
struct TopkScratch {
  TopkState* st;
  unsigned* hist;
  int* blk_a;
  int* blk_b;
  unsigned long long* keys;
  int* ids;
  int* out_ids;
  double* out_sc;
  int* out_k;
  double* dsum;
};

// A query slot: its own scratch and column buffer, so that queries in flight on
// the query stream do not share memory with each other or with the engine.
struct QuerySlot {
  TopkScratch t{};       // out_* point into host_out (host-mapped pinned memory)
  void* host_out = nullptr;
  double* col = nullptr;
  cudaEvent_t done = nullptr;
  int busy = 0;
  int k = 0;
};

}  // namespace

struct osp_ctx {
  osp_options opt{};
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bool broken = false;

  // sizes mirrored on the host
  int64_t n = 0, m = 0, nc = 0;
  unsigned long long cap_r = 0, cap_c = 0, top_r = 0, top_c = 0;
  bool loaded = false, seeded = false, scored = false;
  int seed = -1;
  int S = 1;                   // seeds tracked (S > 1: the seed block d.mu)
  int64_t pagerank_n = 0;      // > 0: uniform restart vector over nodes 0..pagerank_n-1
  double c = 0.15;
  int grid_multi = 0;
  int grid_multi_init = 0;
  int seed_force_max = 0;      // largest per-seed step count set by osp_set_seed_iterations
  // pull-step schedule: task size, long-list threshold and piece, node weight
  // (defaults by seed count until osp_init_scores autotunes them)
  int sched[4] = {0, 0, 0, 0};
  // CUDA graphs of the batch path, by (ingest shared-memory bucket, eps, fixed
  // step counts); dropped whenever device buffers move
  struct GraphPair {
    cudaGraphExec_t update = nullptr, propagate = nullptr;
    int launches = 0;
  };
  std::map<std::tuple<int, double, int, int>, GraphPair> graphs;
  // query slots (osp_query_slots): queries run on qstream after the scores of
  // ev_scores; the next propagation waits for ev_queries
  std::vector<QuerySlot> qslots;
  std::vector<void*> qallocs;
  cudaStream_t qstream = nullptr;
  cudaEvent_t ev_scores = nullptr, ev_queries = nullptr;
  std::vector<void*> mallocs;  // buffers of the seed block, freed when the seeds change
  int fixed_iters = 0;
  int grid_prop = 0;
  int last_iters = 0;
  std::vector<int32_t> col_of;  // several seeds: seed j -> its column of the seed block
  double res_bound = 0.0;       // one seed: bound on ||rho||_1 of the stored scores
  int64_t hbm_used = 0;         // bytes of device memory held by the context
  std::map<void*, size_t> dsizes;

  Dev d{};
  std::vector<void*> allocs;
  osp_update* ops_stage = nullptr;  // device staging for host batches
  void* pinned = nullptr;           // pinned host staging (ops in, control block out)
  double* dsum = nullptr;
  double* dtmp = nullptr;  // n doubles for normalised queries
  unsigned* scan_off = nullptr;
  unsigned* scan_bsum = nullptr;
  int* pool_spare = nullptr;  // compaction target
  unsigned long long spare_cap = 0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // call start, propagation start, end
  int launches = 0;  // kernels launched by the current call
  std::vector<int32_t> e2i, i2e;  // caller id <-> internal id (identity above the loaded ids)
  // top-k scratch
  TopkState* tk_state = nullptr;
  unsigned* tk_hist = nullptr;
  int* tk_blk_a = nullptr;
  int* tk_blk_b = nullptr;
  unsigned long long* tk_keys = nullptr;
  int* tk_ids = nullptr;
  int* tk_out_ids = nullptr;
  double* tk_out_sc = nullptr;
  int* tk_out_k = nullptr;
};

namespace {

osp_status fail(osp_ctx* ctx, osp_status s, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return s;
}

osp_status cuda_fail(osp_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, OSP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                    \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);        \
  } while (0)

template <typename T>
osp_status dalloc(osp_ctx* ctx, T** p, size_t count, int fill = 0,
                  std::vector<void*>* list = nullptr) {
  void* q = nullptr;
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (ctx->opt.hbm_budget_bytes > 0 && ctx->hbm_used + (int64_t)bytes > ctx->opt.hbm_budget_bytes)
    return fail(ctx, OSP_ENOMEM, "HBM budget of " + std::to_string(ctx->opt.hbm_budget_bytes) +
                                     " bytes would be exceeded (" + std::to_string(ctx->hbm_used) +
                                     " held, " + std::to_string(bytes) + " asked)");
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, OSP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  ctx->hbm_used += (int64_t)bytes;
  ctx->dsizes[q] = bytes;
  e = cudaMemsetAsync(q, fill, bytes, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
  (list ? list : &ctx->allocs)->push_back(q);
  *p = (T*)q;
  return OSP_OK;
}

void dfree(osp_ctx* ctx, void* p) {
  auto it = ctx->dsizes.find(p);
  if (it != ctx->dsizes.end()) {
    ctx->hbm_used -= (int64_t)it->second;
    ctx->dsizes.erase(it);
  }
  cudaFree(p);
}

void drop_graphs(osp_ctx* ctx) {
  for (auto& kv : ctx->graphs) {
    if (kv.second.update) cudaGraphExecDestroy(kv.second.update);
    if (kv.second.propagate) cudaGraphExecDestroy(kv.second.propagate);
  }
  ctx->graphs.clear();
}

void free_slots(osp_ctx* ctx) {
  if (ctx->qstream) cudaStreamSynchronize(ctx->qstream);
  for (auto& q : ctx->qslots) {
    if (q.done) cudaEventDestroy(q.done);
    if (q.host_out) cudaFreeHost(q.host_out);
  }
  ctx->qslots.clear();
  for (void* p : ctx->qallocs) dfree(ctx, p);
  ctx->qallocs.clear();
}

void free_multi(osp_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_graphs(ctx);
  for (void* p : ctx->mallocs) dfree(ctx, p);
  ctx->mallocs.clear();
  ctx->d.mu = Multi{};
  ctx->S = 1;
  ctx->seed_force_max = 0;
  ctx->col_of.clear();
}

void free_all(osp_ctx* ctx) {
  free_slots(ctx);
  free_multi(ctx);
  for (void* p : ctx->allocs) dfree(ctx, p);
  ctx->allocs.clear();
  ctx->d = Dev{};
  ctx->ops_stage = nullptr;
  ctx->dsum = nullptr;
  ctx->dtmp = nullptr;
  ctx->scan_off = nullptr;
  ctx->scan_bsum = nullptr;
  ctx->pool_spare = nullptr;
  ctx->tk_state = nullptr;
  ctx->tk_hist = nullptr;
  ctx->tk_blk_a = ctx->tk_blk_b = nullptr;
  ctx->tk_keys = nullptr;
  ctx->tk_ids = ctx->tk_out_ids = ctx->tk_out_k = nullptr;
  ctx->tk_out_sc = nullptr;
}

// Sorted, de-duplicated adjacency lists of one direction from (key, val) pairs.
void build_lists(int64_t n, const std::vector<int32_t>& key, const std::vector<int32_t>& val,
                 std::vector<unsigned>& off, std::vector<int>& len, std::vector<int>& pool) {
  std::vector<int64_t> start(n + 1, 0);
  for (int32_t k : key) start[k + 1]++;
  for (int64_t i = 0; i < n; ++i) start[i + 1] += start[i];
  std::vector<int> tmp(key.size());
  {
    std::vector<int64_t> pos(start.begin(), start.end() - 1);
    for (size_t e = 0; e < key.size(); ++e) tmp[pos[key[e]]++] = val[e];
  }
  len.assign(n, 0);
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    th.emplace_back([&, t]() {
      for (int64_t u = t; u < n; u += nt) {
        int* b = tmp.data() + start[u];
        int* e = tmp.data() + start[u + 1];
        std::sort(b, e);
        len[u] = (int)(std::unique(b, e) - b);
      }
    });
  }
  for (auto& x : th) x.join();
  off.assign(n, 0);
  int64_t tot = 0;
  for (int64_t u = 0; u < n; ++u) {
    off[u] = (unsigned)tot;
    tot += len[u];
  }
  pool.resize(tot);
  for (int64_t u = 0; u < n; ++u)
    std::memcpy(pool.data() + off[u], tmp.data() + start[u], sizeof(int) * len[u]);
}

// The same adjacency under the internal ids: list of internal node i is the
// list of caller node i2e[i], each entry mapped by e2i and re-sorted.
void relabel_lists(int64_t n, const std::vector<int32_t>& e2i, const std::vector<int32_t>& i2e,
                   const std::vector<unsigned>& off, const std::vector<int>& len,
                   const std::vector<int>& pool, std::vector<unsigned>& off2, std::vector<int>& len2,
                   std::vector<int>& pool2) {
  off2.assign(n, 0);
  len2.assign(n, 0);
  int64_t tot = 0;
  for (int64_t i = 0; i < n; ++i) {
    off2[i] = (unsigned)tot;
    len2[i] = len[i2e[i]];
    tot += len2[i];
  }
  pool2.resize(tot);
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    th.emplace_back([&, t]() {
      for (int64_t i = t; i < n; i += nt) {
        const int u = i2e[i];
        int* dst = pool2.data() + off2[i];
        for (int k = 0; k < len[u]; ++k) dst[k] = e2i[pool[off[u] + k]];
        std::sort(dst, dst + len[u]);
      }
    });
  }
  for (auto& x : th) x.join();
}

osp_status read_ctl(osp_ctx* ctx, Ctl* out) {
  CK(cudaMemcpyAsync(ctx->pinned, ctx->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, ctx->pinned, sizeof(Ctl));
  return OSP_OK;
}

osp_status write_ctl(osp_ctx* ctx, const Ctl& in) {
  std::memcpy(ctx->pinned, &in, sizeof(Ctl));
  CK(cudaMemcpyAsync(ctx->d.ctl, ctx->pinned, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return OSP_OK;
}

int default_max_iter(const osp_ctx* ctx, double eps) {
  if (ctx->opt.max_iter > 0) return ctx->opt.max_iter;
  double k = std::ceil(std::log(eps / 2.0) / std::log(1.0 - ctx->c));
  if (!(k > 0)) k = 1;
  return (int)std::min(k + 8.0, (double)kMaxHist - 1);
}

// Reclaim stale pool space: lists are copied in node order to the spare pool,
// which then becomes the live one.
osp_status compact(osp_ctx* ctx, bool rows) {
  Dev& d = ctx->d;
  const int n = (int)ctx->n;
  unsigned* off = rows ? d.off_r : d.off_c;
  int* len = rows ? d.len_r : d.len_c;
  int*& pool = rows ? d.pool_r : d.pool_c;
  unsigned long long& cap = rows ? ctx->cap_r : ctx->cap_c;
  const int nb = (n + 4095) / 4096;
  if (n > 0) {
    k_scan_local<<<nb, 1024, 0, ctx->stream>>>(len, ctx->scan_off, ctx->scan_bsum, n);
    ++ctx->launches;
    k_scan_top<<<1, 1024, 0, ctx->stream>>>(ctx->scan_bsum, nb);
    ++ctx->launches;
    k_scan_add<<<(n + 255) / 256, 256, 0, ctx->stream>>>(ctx->scan_off, ctx->scan_bsum, n);
    ++ctx->launches;
    k_compact_copy<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(off, len, pool, ctx->scan_off,
                                                               ctx->pool_spare, n);
    ++ctx->launches;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(off, ctx->scan_off, sizeof(unsigned) * n, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  }
  std::swap(pool, ctx->pool_spare);
  std::swap(cap, ctx->spare_cap);
  drop_graphs(ctx);  // captured kernels hold the old pool pointers
  Ctl h;
  osp_status s = read_ctl(ctx, &h);
  if (s != OSP_OK) return s;
  // live entries: sum of list lengths = m for either direction
  if (rows) {
    h.pool_top_r = (unsigned long long)ctx->m;
    h.pool_cap_r = cap;
    ctx->top_r = h.pool_top_r;
  } else {
    h.pool_top_c = (unsigned long long)ctx->m;
    h.pool_cap_c = cap;
    ctx->top_c = h.pool_top_c;
  }
  return write_ctl(ctx, h);
}

// Make sure the next batch of U ops cannot run out of node slots or pool space.
osp_status reserve_for_batch(osp_ctx* ctx, int64_t U) {
  if (ctx->n + U > ctx->nc)
    return fail(ctx, OSP_ENOMEM, "node capacity exhausted; create the context with a larger max_nodes");
  // a batch writes at most m + U entries per direction (the new lists)
  const unsigned long long need = (unsigned long long)(ctx->m + U) + 64;
  if (ctx->cap_r - ctx->top_r < need) {
    osp_status s = compact(ctx, true);
    if (s != OSP_OK) return s;
  }
  if (ctx->cap_c - ctx->top_c < need) {
    osp_status s = compact(ctx, false);
    if (s != OSP_OK) return s;
  }
  if (ctx->cap_r - ctx->top_r < need || ctx->cap_c - ctx->top_c < need)
    return fail(ctx, OSP_ENOMEM, "graph pool too small for this batch");
  return OSP_OK;
}

// hist: host copy of the ||x(i)||_1 history (kMaxHist entries)
void fill_stats(osp_ctx* ctx, const Ctl& h, osp_batch_stats* st, int64_t m_before,
                const double* hist) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->iterations = h.iter;
  st->push_iterations = h.push_iters;
  st->visited_edges = h.visited;
  st->n_nodes = h.n;
  st->m_edges = h.m;
  st->net_inserts = h.net_ins;
  st->net_deletes = h.net_ins - (h.m - m_before);
  st->changed_rows = h.n_rec_r;
  st->bad_op = h.status == OSP_EINVAL ? h.bad_op : -1;
  st->qoff_l1 = hist[0];
  st->last_x_l1 = hist[std::max(0, std::min(h.iter, kMaxHist - 1))];
  st->kernel_launches = ctx->launches;
  st->push_frontier = h.push_f;
  st->push_reached = h.push_r;
  st->pull_dst_nodes = h.n_dst_nz;
  st->pull_src_nodes = h.n_src_nz;
  if (ctx->S > 1) {
    const double* rb = (const double*)((const char*)ctx->pinned + kPinnedRes);
    for (int j = 0; j < ctx->S; ++j) st->residual_bound = std::max(st->residual_bound, rb[j]);
  } else {
    st->residual_bound = ctx->res_bound;
  }
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]) == cudaSuccess) st->ms_update = a;
  if (cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]) == cudaSuccess) st->ms_propagate = b;
  cudaGetLastError();
}

osp_status finish_call(osp_ctx* ctx, int64_t m_before, osp_batch_stats* st) {
  // the history (and the seed block's residual bounds) come back with the
  // control block: one synchronisation per call
  const double* hist = (const double*)((const char*)ctx->pinned + kPinnedHist);
  CK(cudaMemcpyAsync((char*)ctx->pinned + kPinnedHist, ctx->d.l1_hist, sizeof(double) * kMaxHist,
                     cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->S > 1 && st)
    CK(cudaMemcpyAsync((char*)ctx->pinned + kPinnedRes, ctx->d.mu.res_bound,
                       sizeof(double) * ctx->S, cudaMemcpyDeviceToHost, ctx->stream));
  Ctl h;
  osp_status s = read_ctl(ctx, &h);
  if (s != OSP_OK) return s;
  ctx->last_iters = h.iter;
  if (ctx->S == 1 && h.status == 0)  // the untaken tail: ||x(k+1)||_1 <= (1-c) ||x(k)||_1
    ctx->res_bound += (1.0 - ctx->c) * hist[std::max(0, std::min(h.iter, kMaxHist - 1))];
  if (h.status == OSP_EINVAL) {
    fill_stats(ctx, h, st, m_before, hist);
    return fail(ctx, OSP_EINVAL, "invalid update batch (first invalid op " +
                                     std::to_string(h.bad_op) + ")");
  }
  if (h.status != 0) {
    ctx->broken = true;
    fill_stats(ctx, h, st, m_before, hist);
    return fail(ctx, (osp_status)h.status,
                std::string("device error: ") + osp_status_string((osp_status)h.status));
  }
  ctx->n = h.n;
  ctx->m = h.m;
  ctx->top_r = h.pool_top_r;
  ctx->top_c = h.pool_top_c;
  fill_stats(ctx, h, st, m_before, hist);
  if (h.noconv) return fail(ctx, OSP_ENOCONV, "iteration cap reached before ||x||_1 <= eps");
  ctx->err.clear();
  return OSP_OK;
}

// The pull-step schedule in force: {task items, long-list threshold, piece,
// node weight}; unset entries take the defaults of the seed count.
const int* schedule(osp_ctx* ctx) {
  static const int single[4] = {kTaskItems, kHubThreshold, kHubPiece, 1};
  static const int multi[4] = {kTaskItems, kMultiHub, kMultiHub, kMultiNodeItems};
  if (ctx->sched[0] > 0) return ctx->sched;
  return ctx->S > 1 ? multi : single;
}

// Pull-step plan for the graph as it is after the merge: in-list length prefix
// over the first n_bound + 1 ids (ids at or above n have empty lists) and the
// merge-path tile starts.
osp_status plan_pull(osp_ctx* ctx, int64_t n_bound, int64_t m_bound) {
  (void)m_bound;
  const int ns = (int)std::min<int64_t>(n_bound + 1, ctx->nc);
  const int nb = (ns + 4095) / 4096;
  cudaStream_t st = ctx->stream;
  k_merge_finish<<<1, 1, 0, st>>>(ctx->d);
  ++ctx->launches;
  k_scan_local<<<nb, 1024, 0, st>>>(ctx->d.len_c, ctx->d.pc, ctx->scan_bsum, ns);
  ++ctx->launches;
  k_scan_top<<<1, 1024, 0, st>>>(ctx->scan_bsum, nb);
  ++ctx->launches;
  k_scan_add<<<(ns + 255) / 256, 256, 0, st>>>(ctx->d.pc, ctx->scan_bsum, ns);
  ++ctx->launches;
  const int* sc = schedule(ctx);
  k_pull_plan<<<ctx->num_sms * 4, 256, 0, st>>>(ctx->d, sc[1], sc[3], sc[0]);
  ++ctx->launches;
  k_hub_prefix<<<1, 1024, 0, st>>>(ctx->d, sc[2], ctx->opt.deterministic != 0);
  ++ctx->launches;
  CK(cudaGetLastError());
  return OSP_OK;
}

// CTAs of the L1-norm reduction: two per SM, at most kAbsParts partials.
int abs_grid(const osp_ctx* ctx) { return std::min(ctx->num_sms * 2, kAbsParts); }

PropParams prop_params(osp_ctx* ctx, double eps) {
  PropParams pp;
  pp.eps = eps;
  pp.max_iter = default_max_iter(ctx, eps);
  pp.force_iters = ctx->fixed_iters;
  if (pp.force_iters > pp.max_iter) pp.max_iter = std::min(pp.force_iters, kMaxHist - 1);
  if (ctx->S > 1 && ctx->seed_force_max > pp.max_iter)
    pp.max_iter = std::min(ctx->seed_force_max, kMaxHist - 1);
  pp.alpha = ctx->opt.push_alpha > 0 ? ctx->opt.push_alpha : kPushAlpha;
  pp.beta = ctx->opt.push_beta > 0 ? ctx->opt.push_beta : kPushBeta;
  pp.fp32 = ctx->opt.precision == OSP_PREC_FP32_ACC64;
  pp.hot_n = 0;
  pp.det = ctx->opt.deterministic != 0;
  return pp;
}

// Seed block: gather rows of internal ids below hot_n get L2 priority. With
// the degree node order those are the most-read rows; the budget is
// osp_options.l2_hot_bytes (default 60% of L2) over the bytes of one group's
// row slice.
int hot_rows(const osp_ctx* ctx, int precision, int KG) {
  if (ctx->opt.node_order != 1 || ctx->opt.l2_hot_bytes < 0) return 0;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  const int64_t budget = ctx->opt.l2_hot_bytes > 0 ? ctx->opt.l2_hot_bytes : (int64_t)l2 * 6 / 10;
  const int elem = precision == OSP_PREC_FP64 ? 8 : precision == OSP_PREC_FP32_ACC64 ? 4 : 2;
  const int64_t rows = budget / (32LL * KG * elem);
  return (int)std::min<int64_t>(rows, ctx->nc);
}

// Seed block of K column groups computed in `precision`: stage source rows by
// bulk copies? By default only for rows of at most 256 bytes, where it was
// measured faster (Chung-Lu 2^22, 64 FP32 seeds: 4.16 vs 6.08 ms per pull
// step); rows of 512 bytes (R-MAT 2^24, 256 bf16 seeds) ran slower (30.7 vs
// 26.3 ms) and keep register gathers.
bool seed_bulk(const osp_ctx* ctx, int precision, int KG) {
  if (ctx->opt.seed_gather != 0) return ctx->opt.seed_gather == 2;
  const int elem = precision == OSP_PREC_FP64 ? 8 : precision == OSP_PREC_FP32_ACC64 ? 4 : 2;
  const int row = 32 * KG * elem;
  return row >= 128 && row <= 256;
}

// The persistent propagation kernel of one call.
osp_status enqueue_propagate(osp_ctx* ctx, const PropParams& pp, bool init) {
  if (ctx->S > 1) {
    // bf16 gather vectors carry the small offsets of batches; the initial CPI
    // (total mass 1) runs with float gather vectors
    const bool as_init = init && ctx->opt.precision == OSP_PREC_BF16_ACC64;
    const int prec = as_init ? (int)OSP_PREC_FP32_ACC64 : ctx->opt.precision;
    const int KG = as_init ? ctx->d.mu.KG_init : ctx->d.mu.KG;
    PropParams p = pp;
    p.hot_n = hot_rows(ctx, prec, KG);
    const bool bulk = seed_bulk(ctx, prec, KG);
    Dev d = ctx->d;
    // bf16 32-column groups gathered by teams: the columns are packed into
    // groups per call, largest offsets first, so that the columns still running
    // after the first steps share few groups
    d.mu.pack = prec == OSP_PREC_BF16_ACC64 && KG == 1 && !bulk && d.mu.Sp > 32;
    CK(launch_propagate_multi(d, p, prec, KG, as_init ? ctx->grid_multi_init : ctx->grid_multi,
                              bulk, ctx->stream));
  }
  else
    CK(launch_propagate(ctx->d, pp, ctx->grid_prop, ctx->stream));
  ++ctx->launches;
  return OSP_OK;
}

osp_status run_propagation(osp_ctx* ctx, double eps, int64_t n_bound, int64_t m_bound,
                           bool init = false) {
  const PropParams pp = prop_params(ctx, eps);
  osp_status s = plan_pull(ctx, n_bound, m_bound);
  if (s != OSP_OK) return s;
  // queries in flight read the scores this kernel changes
  if (!ctx->qslots.empty()) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_queries, 0));
  CK(cudaEventRecord(ctx->ev[1], ctx->stream));
  s = enqueue_propagate(ctx, pp, init);
  if (s != OSP_OK) return s;
  CK(cudaEventRecord(ctx->ev[2], ctx->stream));
  if (!ctx->qslots.empty()) CK(cudaEventRecord(ctx->ev_scores, ctx->stream));
  return OSP_OK;
}

osp_status check_ready(osp_ctx* ctx, bool need_scores) {
  if (!ctx) return OSP_EINVAL;
  if (ctx->broken) return fail(ctx, OSP_ESTATE, "context is broken by an earlier device error");
  if (!ctx->loaded) return fail(ctx, OSP_ESTATE, "no graph loaded");
  if (!ctx->seeded) return fail(ctx, OSP_ESTATE, "no seed set");
  if (need_scores && !ctx->scored) return fail(ctx, OSP_ESTATE, "scores not initialised");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return OSP_OK;
}

// Ingest, merge and offset of one batch (U < 0: k_ingest reads the size from
// the control block, as a graph replay does).
osp_status enqueue_update(osp_ctx* ctx, const osp_update* ops_dev, int U, int Np,
                          bool cont = false) {
  const int g = ctx->num_sms * 4;
  k_reset_batch<<<1, 1, 0, ctx->stream>>>(ctx->d, cont ? 1 : 0);
  ++ctx->launches;
  k_ingest<<<1, 1024, (size_t)Np * 8, ctx->stream>>>(ctx->d, ops_dev, U);
  ++ctx->launches;
  k_expand<<<g, 256, 0, ctx->stream>>>(ctx->d);
  ++ctx->launches;
  k_merge_pieces<<<1, 1024, 0, ctx->stream>>>(
      ctx->d, ctx->opt.push_beta > 0 ? ctx->opt.push_beta : kPushBeta);
  ++ctx->launches;
  k_merge_count<<<g, 256, 0, ctx->stream>>>(ctx->d);
  ++ctx->launches;
  k_merge_plan<<<g, 256, 0, ctx->stream>>>(ctx->d);
  ++ctx->launches;
  k_merge_write<<<g, 256, 0, ctx->stream>>>(ctx->d);
  ++ctx->launches;
  if (ctx->S > 1) {  // the seed block's offset, from the old and new out-lists
    k_offset_multi_plan<<<1, 1024, 0, ctx->stream>>>(ctx->d);
    ++ctx->launches;
    CK(launch_offset_multi(ctx->d, g, ctx->stream));
    ++ctx->launches;
  }
  CK(cudaGetLastError());
  return OSP_OK;
}

// Capture the batch path for this bucket, eps and step settings.
osp_status capture_graphs(osp_ctx* ctx, int Np, double eps, osp_ctx::GraphPair* out) {
  cudaStream_t st = ctx->stream;
  const int before = ctx->launches;
  ctx->launches = 0;
  const PropParams pp = prop_params(ctx, eps);
  for (int part = 0; part < 2; ++part) {
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    osp_status s = OSP_OK;
    if (part == 0) {
      s = enqueue_update(ctx, ctx->ops_stage, -1, Np);
      if (s == OSP_OK) s = plan_pull(ctx, ctx->nc - 1, 0);  // every node slot: fixed grids
    } else {
      s = enqueue_propagate(ctx, pp, false);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != OSP_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    cudaGraphExec_t x = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(ctx, ie, "cudaGraphInstantiate");
    (part == 0 ? out->update : out->propagate) = x;
  }
  out->launches = ctx->launches;
  ctx->launches = before;
  return OSP_OK;
}

// A batch of more than kMaxBatch ops: consecutive sub-batches of kMaxBatch ops
// are ingested and merged one after the other, all against the same r_old, so
// their offsets add up to the offset of the whole batch; one propagation
// follows. ops is a device pointer, or a host one when host != 0 (staged per
// sub-batch through pinned memory). An invalid op stops the sequence: the
// sub-batches before it stay applied and are propagated.
// Sub-batches of a large host batch of edge ops only (ids in [0, n)): the ops
// stably ordered by source row, whole rows packed into each sub-batch (a row
// with more than kMaxBatch ops is cut), so that every changed row's offset is
// formed once instead of once per sub-batch that edits it. Ops on one row keep
// their order, and ops on different rows commute, so the final edge set is the
// one of the batch in its own order. Returns false (and leaves perm empty) when
// the batch holds another kind of op or an id out of range.
bool group_by_row(const osp_update* ops, int64_t U, int64_t n, std::vector<int32_t>& perm,
                  std::vector<int64_t>& cuts) {
  perm.clear();
  cuts.clear();
  for (int64_t i = 0; i < U; ++i) {
    const osp_update& o = ops[i];
    if ((o.op != OSP_OP_INSERT_EDGE && o.op != OSP_OP_DELETE_EDGE) || o.u < 0 || o.u >= n ||
        o.v < 0 || o.v >= n)
      return false;
  }
  // LSD radix sort of the op indices by source row (stable), 11 bits a pass
  std::vector<int32_t> a(U), b(U);
  for (int64_t i = 0; i < U; ++i) a[i] = (int32_t)i;
  int bits = 1;
  while ((int64_t(1) << bits) < n) ++bits;
  std::vector<int64_t> cnt(1 << 11);
  for (int sh = 0; sh < bits; sh += 11) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t i = 0; i < U; ++i) ++cnt[(ops[a[i]].u >> sh) & 2047];
    int64_t t = 0;
    for (auto& c : cnt) {
      const int64_t x = c;
      c = t;
      t += x;
    }
    for (int64_t i = 0; i < U; ++i) b[cnt[(ops[a[i]].u >> sh) & 2047]++] = a[i];
    a.swap(b);
  }
  perm.swap(a);
  cuts.push_back(0);
  int64_t start = 0;  // of the open sub-batch
  for (int64_t i = 0; i < U;) {
    int64_t j = i;
    while (j < U && ops[perm[j]].u == ops[perm[i]].u) ++j;
    if (j - i > kMaxBatch) {  // a row alone above the limit: cut it
      if (i > start) cuts.push_back(i);
      for (int64_t c = i + kMaxBatch; c < j; c += kMaxBatch) cuts.push_back(c);
      start = cuts.back();
    } else if (j - start > kMaxBatch) {
      cuts.push_back(i);
      start = i;
    }
    i = j;
  }
  cuts.push_back(U);
  return true;
}

osp_status apply_large(osp_ctx* ctx, const osp_update* ops, bool host, int64_t U, double eps,
                       osp_batch_stats* st) {
  if (!(eps > 0)) return fail(ctx, OSP_EINVAL, "eps must be > 0");
  ctx->launches = 0;
  const int64_t m_before = ctx->m;
  int64_t bad = -1;
  osp_status err = OSP_OK;
  std::vector<int32_t> perm;
  std::vector<int64_t> cuts;
  if (!(host && group_by_row(ops, U, ctx->n, perm, cuts))) {
    perm.clear();
    cuts.clear();
    for (int64_t s0 = 0; s0 < U; s0 += kMaxBatch) cuts.push_back(s0);
    cuts.push_back(U);
  }
  CK(cudaEventRecord(ctx->ev[0], ctx->stream));
  for (size_t ci = 0; ci + 1 < cuts.size(); ++ci) {
    const int64_t s0 = cuts[ci];
    const int u = (int)(cuts[ci + 1] - s0);
    osp_status s = reserve_for_batch(ctx, u);
    if (s != OSP_OK) {
      err = s;
      break;
    }
    const osp_update* p = ops + s0;
    if (host) {
      osp_update* pin = (osp_update*)ctx->pinned;
      if (perm.empty()) {
        std::memcpy(pin, p, sizeof(osp_update) * (size_t)u);
      } else {
        for (int i = 0; i < u; ++i) pin[i] = ops[perm[s0 + i]];
      }
      CK(cudaMemcpyAsync(ctx->ops_stage, ctx->pinned, sizeof(osp_update) * (size_t)u,
                         cudaMemcpyHostToDevice, ctx->stream));
      p = ctx->ops_stage;
    }
    int Np = 2;
    while (Np < u) Np <<= 1;
    s = enqueue_update(ctx, p, u, Np, s0 > 0);
    if (s != OSP_OK) return s;
    Ctl h;
    s = read_ctl(ctx, &h);  // also orders the pinned buffer's reuse
    if (s != OSP_OK) return s;
    if (h.status == OSP_EINVAL) {
      bad = perm.empty() ? s0 + h.bad_op : (int64_t)perm[s0 + h.bad_op];
      h.status = 0;
      s = write_ctl(ctx, h);
      if (s != OSP_OK) return s;
      break;
    }
    if (h.status != 0) {
      ctx->broken = true;
      return fail(ctx, (osp_status)h.status, "device error in a sub-batch");
    }
    ctx->n = h.n;
    ctx->m = h.m + h.m_delta;  // live entries so far (the change is folded in at the end)
    ctx->top_r = h.pool_top_r;
    ctx->top_c = h.pool_top_c;
  }
  osp_status s = run_propagation(ctx, eps, ctx->nc - 1, ctx->m);
  if (s != OSP_OK) return s;
  s = finish_call(ctx, m_before, st);
  if (bad >= 0) {
    if (st) st->bad_op = bad;
    return fail(ctx, OSP_EINVAL, "invalid op " + std::to_string(bad) +
                                     "; the sub-batches before it were applied");
  }
  if (err != OSP_OK) return fail(ctx, err, ctx->err + " (the sub-batches before it were applied)");
  return s;
}

osp_status apply_common(osp_ctx* ctx, const osp_update* ops_dev, int64_t U, double eps,
                        osp_batch_stats* st) {
  if (!(eps > 0)) return fail(ctx, OSP_EINVAL, "eps must be > 0");
  ctx->launches = 0;
  osp_status s = reserve_for_batch(ctx, U);
  if (s != OSP_OK) return s;
  const int64_t m_before = ctx->m;
  const int N = (int)std::max<int64_t>(2, U);
  int Np = 2;
  while (Np < N) Np <<= 1;
  if (ctx->opt.use_graphs) {
    if (U > 0 && ops_dev != ctx->ops_stage)
      CK(cudaMemcpyAsync(ctx->ops_stage, ops_dev, sizeof(osp_update) * (size_t)U,
                         cudaMemcpyDeviceToDevice, ctx->stream));
    int* pu = (int*)((char*)ctx->pinned + kPinnedBatchSize);
    *pu = (int)U;
    CK(cudaMemcpyAsync(&ctx->d.ctl->batch_U, pu, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    const auto key = std::make_tuple(Np, eps, ctx->fixed_iters, ctx->seed_force_max);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
      osp_ctx::GraphPair gp;
      s = capture_graphs(ctx, Np, eps, &gp);
      if (s != OSP_OK) {
        if (gp.update) cudaGraphExecDestroy(gp.update);
        return s;
      }
      it = ctx->graphs.emplace(key, gp).first;
    }
    CK(cudaEventRecord(ctx->ev[0], ctx->stream));
    CK(cudaGraphLaunch(it->second.update, ctx->stream));
    if (!ctx->qslots.empty()) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_queries, 0));
    CK(cudaEventRecord(ctx->ev[1], ctx->stream));
    CK(cudaGraphLaunch(it->second.propagate, ctx->stream));
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    if (!ctx->qslots.empty()) CK(cudaEventRecord(ctx->ev_scores, ctx->stream));
    ctx->launches = it->second.launches;
    return finish_call(ctx, m_before, st);
  }
  CK(cudaEventRecord(ctx->ev[0], ctx->stream));
  s = enqueue_update(ctx, ops_dev, (int)U, Np);
  if (s != OSP_OK) return s;
  s = run_propagation(ctx, eps, std::min<int64_t>(ctx->n + U, ctx->nc - 1), ctx->m + U);
  if (s != OSP_OK) return s;
  return finish_call(ctx, m_before, st);
}

// Seed j's column of the seed block (the seed itself with one seed).
int col_for(const osp_ctx* ctx, int j) { return ctx->S > 1 ? ctx->col_of[j] : j; }

// Column col of the scores in caller order into dst, on stream st.
// Score columns in caller order into dsts[i] (device, n doubles each).
osp_status enqueue_gather(osp_ctx* ctx, cudaStream_t st, const int* cols, double* const* dsts, int m) {
  const int n = (int)ctx->n;
  if (ctx->S > 1) {
    GatherJobs G{};
    for (int i = 0; i < m; ++i) {
      G.col[i] = cols[i];
      G.dst[i] = dsts[i];
    }
    k_gather_cols<<<dim3(ctx->num_sms * 4, m), 256, 0, st>>>(ctx->d.mu.r, ctx->d.mu.Sp,
                                                            ctx->d.int2ext, n, G);
    ++ctx->launches;
  } else {
    for (int i = 0; i < m; ++i) {
      k_gather_ext<<<ctx->num_sms * 4, 256, 0, st>>>(ctx->d.r, ctx->d.ext2int, n, dsts[i]);
      ++ctx->launches;
    }
  }
  CK(cudaGetLastError());
  return OSP_OK;
}

TopkJob topk_job(const double* src, const TopkScratch& t, bool normalize) {
  TopkJob j{};
  j.src = src;
  j.st = t.st;
  j.hist = t.hist;
  j.blk_a = t.blk_a;
  j.blk_b = t.blk_b;
  j.keys = t.keys;
  j.ids = t.ids;
  j.norm = normalize ? t.dsum : nullptr;
  j.out_ids = t.out_ids;
  j.out_sc = t.out_sc;
  j.out_k = t.out_k;
  return j;
}

// Top-k of every job of J on stream st: the norms asked for, the radix
// select and ordered compaction, the sort (results in each job's out_*).
osp_status enqueue_topk(osp_ctx* ctx, cudaStream_t st, const TopkJobs& J) {
  for (int i = 0; i < J.m; ++i)
    if (J.j[i].norm) {
      double* sum = const_cast<double*>(J.j[i].norm);
      k_abs_sum<<<abs_grid(ctx), 256, 0, st>>>(J.j[i].src, J.n, sum, sum + 1);
      ++ctx->launches;
    }
  ctx->launches += enqueue_topk_select(J, ctx->num_sms, st);
  ctx->launches += enqueue_topk_sort(J, st);
  CK(cudaGetLastError());
  return OSP_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void osp_default_options(osp_options* opt) {
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = OSP_PREC_FP32_ACC64;
}

const char* osp_status_string(osp_status s) {
  switch (s) {
    case OSP_OK: return "OSP_OK";
    case OSP_EINVAL: return "OSP_EINVAL";
    case OSP_ENOMEM: return "OSP_ENOMEM";
    case OSP_ECUDA: return "OSP_ECUDA";
    case OSP_ETIMEOUT: return "OSP_ETIMEOUT";
    case OSP_ENOCONV: return "OSP_ENOCONV";
    case OSP_ESTATE: return "OSP_ESTATE";
    case OSP_ENOTSUP: return "OSP_ENOTSUP";
  }
  return "OSP_UNKNOWN";
}

const char* osp_last_error(const osp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t osp_max_batch(void) { return kMaxBatch; }

osp_status osp_selftest_wait(int32_t device, int32_t which, int32_t lose) {
  if (which != 0 && which != 1) return OSP_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return OSP_ECUDA;
  Ctl* ctl = nullptr;
  float* src = nullptr;
  cudaStream_t st = nullptr;
  osp_status r = OSP_ECUDA;
  std::vector<float> h(64);
  for (int i = 0; i < 64; ++i) h[i] = 1.0f + (float)i;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
      cudaMalloc(&ctl, sizeof(Ctl)) == cudaSuccess &&
      cudaMalloc(&src, sizeof(float) * 64) == cudaSuccess &&
      cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) == cudaSuccess &&
      cudaMemcpyAsync(src, h.data(), sizeof(float) * 64, cudaMemcpyHostToDevice, st) == cudaSuccess &&
      launch_selftest(ctl, src, which, lose ? 1 : 0, st) == cudaSuccess &&
      cudaStreamSynchronize(st) == cudaSuccess) {
    Ctl c;
    if (cudaMemcpy(&c, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) == cudaSuccess) {
      if (c.status != 0) r = (osp_status)c.status;
      else r = c.iter == 1 ? OSP_OK : OSP_ECUDA;  // completed, and (staging) the rows intact
    }
  }
  cudaGetLastError();
  if (src) cudaFree(src);
  if (ctl) cudaFree(ctl);
  if (st) cudaStreamDestroy(st);
  return r;
}

osp_status osp_create(osp_ctx** out, const osp_options* opt) {
  if (!out) return OSP_EINVAL;
  *out = nullptr;
  osp_ctx* ctx = new osp_ctx();
  if (opt) ctx->opt = *opt;
  else osp_default_options(&ctx->opt);
  if (ctx->opt.precision != OSP_PREC_FP64 && ctx->opt.precision != OSP_PREC_FP32_ACC64 &&
      ctx->opt.precision != OSP_PREC_BF16_ACC64) {
    delete ctx;
    return OSP_EINVAL;
  }
  if (ctx->opt.seed_gather < 0 || ctx->opt.seed_gather > 2) {
    delete ctx;
    return OSP_EINVAL;
  }
  {
    const int g = ctx->opt.seed_group;
    if (g != 0 && g != 32 && g != 64 && g != 128 && g != 256) {
      delete ctx;
      return OSP_EINVAL;
    }
  }
  ctx->device = ctx->opt.device;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) {
    if (ctx->opt.stream) {
      ctx->stream = (cudaStream_t)ctx->opt.stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->pinned, kPinnedBytes);
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_ingest, cudaFuncAttributeMaxDynamicSharedMemorySize, kIngestSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_topk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTopkSortSmem);
  if (e != cudaSuccess) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
    cudaGetLastError();
    return OSP_ECUDA;
  }
  ctx->grid_prop = propagate_grid(ctx->opt.precision != OSP_PREC_FP64, ctx->num_sms);
  if (ctx->grid_prop <= 0) {
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    cudaFreeHost(ctx->pinned);
    delete ctx;
    return OSP_ECUDA;
  }
  *out = ctx;
  return OSP_OK;
}

void osp_destroy(osp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  free_all(ctx);
  for (cudaEvent_t ev : ctx->ev)
    if (ev) cudaEventDestroy(ev);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->qstream) cudaStreamDestroy(ctx->qstream);
  if (ctx->ev_scores) cudaEventDestroy(ctx->ev_scores);
  if (ctx->ev_queries) cudaEventDestroy(ctx->ev_queries);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

osp_status osp_load_graph(osp_ctx* ctx, int64_t n, int64_t m, const int32_t* src,
                          const int32_t* dst, int undirected) {
  if (!ctx) return OSP_EINVAL;
  if (n <= 0 || n >= kMaxNodes || m < 0 || (m > 0 && (!src || !dst)))
    return fail(ctx, OSP_EINVAL, "bad graph size");
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
      return fail(ctx, OSP_EINVAL, "edge " + std::to_string(e) + " has an id outside [0, n)");
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaSetDevice");
  free_all(ctx);
  ctx->loaded = ctx->seeded = ctx->scored = false;
  ctx->broken = false;

  // sorted, de-duplicated out- and in-lists
  const int64_t k = undirected ? 2 * m : m;
  std::vector<int32_t> a(k), b(k);
  for (int64_t e = 0; e < m; ++e) {
    a[e] = src[e];
    b[e] = dst[e];
    if (undirected) {
      a[m + e] = dst[e];
      b[m + e] = src[e];
    }
  }
  std::vector<unsigned> off_r, off_c;
  std::vector<int> len_r, len_c, pool_r, pool_c;
  build_lists(n, a, b, off_r, len_r, pool_r);
  build_lists(n, b, a, off_c, len_c, pool_c);
  const int64_t mm = (int64_t)pool_r.size();
  // internal order: the caller's ids, or descending out-degree (ties by id)
  std::vector<int32_t> i2e(n), e2i(n);
  for (int64_t i = 0; i < n; ++i) i2e[i] = (int32_t)i;
  if (ctx->opt.node_order == 1)
    std::stable_sort(i2e.begin(), i2e.end(),
                     [&](int32_t x, int32_t y) { return len_r[x] > len_r[y]; });
  for (int64_t i = 0; i < n; ++i) e2i[i2e[i]] = (int32_t)i;
  {
    std::vector<unsigned> o2;
    std::vector<int> l2, p2;
    relabel_lists(n, e2i, i2e, off_r, len_r, pool_r, o2, l2, p2);
    off_r.swap(o2);
    len_r.swap(l2);
    pool_r.swap(p2);
    relabel_lists(n, e2i, i2e, off_c, len_c, pool_c, o2, l2, p2);
    off_c.swap(o2);
    len_c.swap(l2);
    pool_c.swap(p2);
  }

  int64_t nc = ctx->opt.max_nodes > 0 ? ctx->opt.max_nodes : n + n / 4 + 4096;
  nc = std::max<int64_t>(nc, n + kMaxBatch);
  nc = std::min<int64_t>(nc, kMaxNodes);
  if (nc < n + 1) return fail(ctx, OSP_EINVAL, "graph too large");
  const unsigned long long cap = 4ull * (unsigned long long)mm + 4ull * kMaxBatch + 65536;
  if (cap >= 0xFFFFFFFFull) return fail(ctx, OSP_EINVAL, "graph too large for 32-bit pool offsets");
  ctx->nc = nc;
  ctx->n = n;
  ctx->m = mm;
  ctx->e2i = e2i;
  ctx->i2e = i2e;
  ctx->e2i.resize(nc);
  ctx->i2e.resize(nc);
  for (int64_t x = n; x < nc; ++x) ctx->e2i[x] = ctx->i2e[x] = (int32_t)x;
  ctx->cap_r = ctx->cap_c = ctx->spare_cap = cap;
  ctx->top_r = ctx->top_c = (unsigned long long)mm;

  Dev& d = ctx->d;
  d.nc = (int)nc;
  osp_status s = OSP_OK;
#define AL(p, cnt, fill)                          \
  do {                                            \
    s = dalloc(ctx, &(p), (size_t)(cnt), (fill)); \
    if (s != OSP_OK) {                            \
      free_all(ctx);                              \
      return s;                                   \
    }                                             \
  } while (0)
  AL(d.ext2int, nc, 0);
  AL(d.int2ext, nc, 0);
  AL(d.off_r, nc, 0);
  AL(d.len_r, nc, 0);
  AL(d.off_c, nc, 0);
  AL(d.len_c, nc, 0);
  AL(d.pool_r, cap, 0);
  AL(d.pool_c, cap, 0);
  AL(ctx->pool_spare, cap, 0);
  AL(d.r, nc, 0);
  double* y0;
  double* y1;
  AL(y0, nc, 0);
  AL(y1, nc, 0);
  d.y0 = y0;
  d.y1 = y1;
  AL(d.xacc, nc, 0);
  if (ctx->opt.deterministic) AL(d.xfix, nc, 0);
  AL(d.scale_d, nc, 0);
  AL(d.scale_f, nc, 0);
  AL(d.mark, nc, 0);
  AL(d.q0, nc, 0);
  AL(d.q1, nc, 0);
  AL(d.dead, nc, 0);
  AL(d.seedflag, nc, 0);
  AL(d.del_pos, nc, 0x7F);
  AL(d.clr_pos, nc, 0xFF);
  AL(d.rflag, nc, 0);
  AL(d.cflag, nc, 0);
  AL(d.ins_r, kMaxBatch, 0);
  AL(d.del_r, kMaxBatch, 0);
  AL(d.ins_c, kMaxBatch, 0);
  AL(d.del_c, kMaxBatch, 0);
  AL(d.gi, kMaxBatch + 1, 0);
  AL(d.gd, kMaxBatch + 1, 0);
  AL(d.rec_r_node, nc, 0);
  AL(d.rec_r_is, nc, 0);
  AL(d.rec_r_ic, nc, 0);
  AL(d.rec_r_ds, nc, 0);
  AL(d.rec_r_dc, nc, 0);
  AL(d.rec_c_node, nc, 0);
  AL(d.rec_c_is, nc, 0);
  AL(d.rec_c_ic, nc, 0);
  AL(d.rec_c_ds, nc, 0);
  AL(d.rec_c_dc, nc, 0);
  AL(d.del_nodes, kMaxBatch, 0);
  AL(d.clr_nodes, kMaxBatch, 0);
  AL(d.rec_old_off, 2 * nc + 1, 0);
  AL(d.rec_old_len, 2 * nc + 1, 0);
  AL(d.rec_pstart, 2 * nc + 1, 0);
  AL(d.rec_fbase, 2 * nc, 0);
  AL(d.rec_dp, 2 * nc, 0);
  {
    // pieces: at most one per changed list plus one per kPiece old entries
    const int64_t npc = 2 * nc + 2 * (int64_t)(cap / kPiece) + 2;
    AL(d.piece_rec, npc, 0);
    AL(d.piece_cnt, npc, 0);
    AL(d.piece_base, npc, 0);
  }
  AL(d.pc, nc + 1, 0);
  AL(d.task_first, (int64_t)(kMultiNodeItems * nc + (int64_t)cap) / kMinTaskItems + 2, 0);
  {
    // lists longer than a threshold t number at most (live edges) / t <= cap / t;
    // the pull plan uses t = kMultiHub for the seed block, kHubThreshold otherwise
    const int64_t nh = (int64_t)(cap / kMultiHub) + 2;
    AL(d.hubs, nh, 0);
    AL(d.hub_pstart, nh + 1, 0);
    // pieces: at most m / piece + (lists) <= 2 cap / kMultiHub, pieces never shorter than kMultiHub
    AL(d.piece_hub, 2 * nh + 4, 0);
    AL(d.piece_part, 2 * nh + 4, 0);
    AL(d.hub_l1, nh, 0);
    AL(d.hub_acc, nh, 0);
    AL(d.hub_cnt, nh, 0);
    const int64_t nb = (int64_t)(cap / kHubThreshold) + 2;  // push: rows above kHubThreshold
    AL(d.big_u, nb, 0);
    AL(d.big_y, nb, 0);
  }
  AL(d.part_l1, kMaxGrid, 0);
  AL(d.part_ef, kMaxGrid, 0);
  AL(d.l1_hist, kMaxHist, 0);
  AL(d.step_ns, kMaxHist + 1, 0);
  AL(d.ctl, 1, 0);
  AL(ctx->ops_stage, kMaxBatch, 0);
  AL(ctx->dsum, kAbsParts + 2, 0);  // the norm, its per-CTA partials, the CTA count
  AL(ctx->dtmp, nc, 0);
  AL(ctx->scan_off, nc, 0);
  AL(ctx->scan_bsum, nc / 4096 + 2, 0);
  AL(ctx->tk_state, 1, 0);
  AL(ctx->tk_hist, 4096, 0);
  AL(ctx->tk_blk_a, nc / kTopkChunk + 2, 0);
  AL(ctx->tk_blk_b, nc / kTopkChunk + 2, 0);
  AL(ctx->tk_keys, kTopkMaxK + kTopkCand, 0);
  AL(ctx->tk_ids, kTopkMaxK + kTopkCand, 0);
  AL(ctx->tk_out_ids, kTopkMaxK, 0);
  AL(ctx->tk_out_sc, kTopkMaxK, 0);
  AL(ctx->tk_out_k, 1, 0);
#undef AL
  CK(cudaMemcpyAsync(d.ext2int, ctx->e2i.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d.int2ext, ctx->i2e.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d.off_r, off_r.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d.len_r, len_r.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d.off_c, off_c.data(), sizeof(unsigned) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d.len_c, len_c.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  if (mm > 0) {
    CK(cudaMemcpyAsync(d.pool_r, pool_r.data(), sizeof(int) * mm, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d.pool_c, pool_c.data(), sizeof(int) * mm, cudaMemcpyHostToDevice, ctx->stream));
  }
  Ctl h;
  std::memset(&h, 0, sizeof(h));
  h.n = (int)n;
  h.m = mm;
  h.pool_top_r = h.pool_top_c = (unsigned long long)mm;
  h.pool_cap_r = h.pool_cap_c = cap;
  h.epoch = 1;
  h.seed = 0;
  h.c = ctx->c;
  s = write_ctl(ctx, h);
  if (s != OSP_OK) return s;
  ctx->loaded = true;
  ctx->err.clear();
  return OSP_OK;
}

osp_status osp_set_seeds(osp_ctx* ctx, const int32_t* seeds, int32_t S, double c) {
  if (!ctx) return OSP_EINVAL;
  if (!ctx->loaded) return fail(ctx, OSP_ESTATE, "no graph loaded");
  if (ctx->broken) return fail(ctx, OSP_ESTATE, "context is broken by an earlier device error");
  if (!seeds || S < 1 || S > kMaxSeeds)
    return fail(ctx, OSP_EINVAL, "need between 1 and 256 seeds");
  if (!(c > 0.0 && c < 1.0)) return fail(ctx, OSP_EINVAL, "c must lie in (0, 1)");
  const bool pagerank = S == 1 && seeds[0] == OSP_PAGERANK;
  std::vector<int32_t> sorted(seeds, seeds + S);
  std::sort(sorted.begin(), sorted.end());
  for (int i = 0; i < S && !pagerank; ++i) {
    if (sorted[i] < 0 || sorted[i] >= ctx->n) return fail(ctx, OSP_EINVAL, "seed id out of range");
    if (i > 0 && sorted[i] == sorted[i - 1]) return fail(ctx, OSP_EINVAL, "duplicate seed");
  }
  if (S == 1 && ctx->opt.precision == OSP_PREC_BF16_ACC64)
    return fail(ctx, OSP_ENOTSUP, "bf16 gather vectors are built for two or more seeds");
  if (S > 1 && ctx->opt.deterministic)
    return fail(ctx, OSP_ENOTSUP, "the deterministic mode covers the one-seed path");
  CK(cudaSetDevice(ctx->device));
  std::vector<int32_t> s_int(S, 0);
  for (int i = 0; i < S && !pagerank; ++i) {
    s_int[i] = ctx->e2i[seeds[i]];
    unsigned char dead = 0;
    CK(cudaMemcpy(&dead, ctx->d.dead + s_int[i], 1, cudaMemcpyDeviceToHost));
    if (dead) return fail(ctx, OSP_EINVAL, "seed is a deleted node");
  }
  if (ctx->qstream) CK(cudaStreamSynchronize(ctx->qstream));  // no query reads the old scores
  free_multi(ctx);
  ctx->seeded = ctx->scored = false;
  Ctl h;
  osp_status s = read_ctl(ctx, &h);
  if (s != OSP_OK) return s;
  h.seed = pagerank ? -1 : s_int[0];
  h.c = c;
  h.multi = S > 1;
  ctx->pagerank_n = pagerank ? ctx->n : 0;
  s = write_ctl(ctx, h);
  if (s != OSP_OK) return s;
  ctx->seed = seeds[0];
  ctx->c = c;
  CK(cudaMemsetAsync(ctx->d.seedflag, 0, ctx->nc, ctx->stream));
  for (int i = 0; i < S && !pagerank; ++i)
    CK(cudaMemsetAsync(ctx->d.seedflag + s_int[i], 1, 1, ctx->stream));
  k_set_scale<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->d, (int)ctx->n, c);
  ++ctx->launches;
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(ctx->d.r, 0, sizeof(double) * ctx->nc, ctx->stream));
  if (S > 1) {
    // the seed block: n x Sp per vector, Sp = 32 K with K in {1, 2, 4, 8}
    Multi& M = ctx->d.mu;
    const int K = S <= 32 ? 1 : S <= 64 ? 2 : S <= 128 ? 4 : 8;
    const size_t cells = (size_t)ctx->nc * 32 * K;
    // bf16 batches keep float-sized gather blocks: the initial CPI runs in float
    const size_t ybytes = ctx->opt.precision == OSP_PREC_FP64 ? 8 : 4;
    const size_t nh = (size_t)(ctx->cap_c / kMultiHub) + 2;
    unsigned char* y0 = nullptr;
    unsigned char* y1 = nullptr;
    unsigned char* ebuf = nullptr;
    unsigned char* yn0 = nullptr;
    unsigned char* yn1 = nullptr;
    double* hub = nullptr;
    // columns: seeds with out-edges first, then dead-end seeds (whose column
    // has a zero offset unless a batch gives the seed out-edges), each part in
    // the caller's order, so that column groups of dead-end seeds mostly skip
    std::vector<int32_t> deg(S, 0);
    for (int i = 0; i < S; ++i)
      CK(cudaMemcpy(&deg[i], ctx->d.len_r + s_int[i], sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int32_t> order;
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i < S; ++i)
        if ((deg[i] > 0) == (pass == 0)) order.push_back(i);
    ctx->col_of.assign(S, 0);
    std::vector<int32_t> by_col(S);
    for (int c = 0; c < S; ++c) {
      ctx->col_of[order[c]] = c;
      by_col[c] = s_int[order[c]];
    }
#define ML(p, cnt)                                                    \
  do {                                                                \
    s = dalloc(ctx, &(p), (size_t)(cnt), 0, &ctx->mallocs);           \
    if (s != OSP_OK) {                                                \
      free_multi(ctx);                                                \
      return s;                                                       \
    }                                                                 \
  } while (0)
    ML(M.seeds, S);
    ML(M.r, cells);
    ML(M.xacc, cells);
    ML(y0, cells * ybytes);
    ML(y1, cells * ybytes);
    if (ctx->opt.precision == OSP_PREC_BF16_ACC64) ML(ebuf, cells * 2);
    if (ctx->opt.precision == OSP_PREC_BF16_ACC64 && K > 1) {  // narrow steps (up to 8 bf16 per node)
      ML(yn0, (size_t)ctx->nc * 16);
      ML(yn1, (size_t)ctx->nc * 16);
    }
    ML(M.part, (size_t)kMaxGrid * 32 * K);
    ML(M.active, 32 * K);
    ML(M.touched, 32 * K);
    ML(M.col_iters, 32 * K);
    ML(M.col_q, 32 * K);
    ML(M.col_last, 32 * K);
    ML(M.res_bound, 32 * K);
    ML(M.force, 32 * K);
    ML(M.slot_col, 32 * K);
    ML(M.col_slot, 32 * K);
    ML(hub, nh * 32 * K);
    ML(M.hub_cnt, nh * 8);
#undef ML
    M.S = S;
    M.K = K;
    M.Sp = 32 * K;
    M.y0 = y0;
    M.y1 = y1;
    M.e = ebuf;
    M.yn0 = yn0;
    M.yn1 = yn1;
    M.hub_acc = hub;
    // column groups: 32 columns for bf16 gather rows (64-byte slices; measured
    // 8 ms per pass at R-MAT 2^24 against 28.7 ms for one masked 256-column
    // pass), else one group of all Sp columns, unless the options say
    const int g = ctx->opt.seed_group > 0 ? ctx->opt.seed_group
                  : ctx->opt.precision == OSP_PREC_BF16_ACC64 ? 32 : 32 * K;
    M.KG = std::max(1, std::min(K, g / 32));
    M.KG_init = ctx->opt.seed_group > 0 ? M.KG : K;
    CK(cudaMemcpyAsync(M.seeds, by_col.data(), sizeof(int32_t) * S, cudaMemcpyHostToDevice, ctx->stream));
    const int prec_init =
        ctx->opt.precision == OSP_PREC_FP64 ? OSP_PREC_FP64 : OSP_PREC_FP32_ACC64;
    ctx->grid_multi = propagate_multi_grid(ctx->opt.precision, M.KG, ctx->num_sms,
                                           seed_bulk(ctx, ctx->opt.precision, M.KG));
    ctx->grid_multi_init = propagate_multi_grid(prec_init, M.KG_init, ctx->num_sms,
                                                seed_bulk(ctx, prec_init, M.KG_init));
    if (ctx->grid_multi <= 0 || ctx->grid_multi_init <= 0) {
      free_multi(ctx);
      return fail(ctx, OSP_ECUDA, "no resident grid for the seed-block kernel");
    }
    ctx->S = S;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->seeded = true;
  ctx->err.clear();
  return OSP_OK;
}

// x(0) = c e_s per seed, with the scores cleared.
osp_status enqueue_cpi_start(osp_ctx* ctx) {
  k_reset_batch<<<1, 1, 0, ctx->stream>>>(ctx->d, 0);
  ++ctx->launches;
  if (ctx->S > 1) {
    const Multi& M = ctx->d.mu;
    CK(cudaMemsetAsync(M.r, 0, sizeof(double) * (size_t)ctx->nc * M.Sp, ctx->stream));
    CK(cudaMemsetAsync(M.res_bound, 0, sizeof(double) * M.Sp, ctx->stream));
    k_multi_cpi_begin<<<1, kMaxSeeds, 0, ctx->stream>>>(ctx->d);
  } else {
    CK(cudaMemsetAsync(ctx->d.r, 0, sizeof(double) * ctx->nc, ctx->stream));
    if (ctx->pagerank_n > 0)
      k_cpi_begin_uniform<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(ctx->d, (int)ctx->pagerank_n);
    else
      k_cpi_begin<<<1, 1, 0, ctx->stream>>>(ctx->d);
  }
  ++ctx->launches;
  CK(cudaGetLastError());
  return OSP_OK;
}

// Time the first CPI steps under each candidate pull schedule and keep the
// fastest: three steps with several seeds (every step is a pull step), twelve
// with one (the first steps from a single seed are push steps).
osp_status autotune(osp_ctx* ctx, double eps) {
  const bool multi = ctx->S > 1;
  const int tis[3] = {512, 1024, 2048};
  const int hubs_single[3] = {512, 1024, 4096};
  const int hubs_multi[3] = {kMultiHub, 2 * kMultiHub, 4 * kMultiHub};
  const int nws_multi[3] = {2, 4, 8};
  std::vector<std::array<int, 4>> cands;
  for (int ti : tis)
    for (int h = 0; h < 3; ++h)
      for (int w = 0; w < (multi ? 3 : 1); ++w) {
        const int hub = multi ? hubs_multi[h] : hubs_single[h];
        cands.push_back({ti, hub, hub, multi ? nws_multi[w] : 1});
      }
  PropParams pp = prop_params(ctx, eps);
  pp.force_iters = multi ? 3 : 12;
  pp.max_iter = std::max(pp.max_iter, pp.force_iters);
  float best = 1e30f;
  std::array<int, 4> pick = cands[0];
  for (int trial = -1; trial < (int)cands.size(); ++trial) {  // trial -1 warms up
    const auto& cd = cands[trial < 0 ? 0 : trial];
    for (int i = 0; i < 4; ++i) ctx->sched[i] = cd[i];
    osp_status s = enqueue_cpi_start(ctx);
    if (s == OSP_OK) s = plan_pull(ctx, ctx->n, ctx->m);
    if (s != OSP_OK) return s;
    CK(cudaEventRecord(ctx->ev[1], ctx->stream));
    // time the kernel the batches will run (bf16 gather rows included; the
    // scores of these trial steps are discarded)
    s = enqueue_propagate(ctx, pp, false);
    if (s != OSP_OK) return s;
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    CK(cudaEventSynchronize(ctx->ev[2]));
    Ctl h;
    s = read_ctl(ctx, &h);
    if (s != OSP_OK) return s;
    if (h.status != 0) {
      ctx->broken = true;
      return fail(ctx, (osp_status)h.status, "device error while tuning the pull schedule");
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]));
    if (trial >= 0 && ms < best) {
      best = ms;
      pick = cd;
    }
  }
  for (int i = 0; i < 4; ++i) ctx->sched[i] = pick[i];
  drop_graphs(ctx);  // captured plans hold the previous schedule
  return OSP_OK;
}

osp_status osp_init_scores(osp_ctx* ctx, double eps, osp_batch_stats* stats) {
  osp_status s = check_ready(ctx, false);
  if (s != OSP_OK) return s;
  if (!(eps > 0)) return fail(ctx, OSP_EINVAL, "eps must be > 0");
  ctx->launches = 0;
  if (ctx->opt.autotune && !ctx->opt.deterministic) {  // a timed choice would vary the bits
    s = autotune(ctx, eps);
    if (s != OSP_OK) return s;
    ctx->launches = 0;
  }
  if (!ctx->qslots.empty()) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_queries, 0));
  CK(cudaEventRecord(ctx->ev[0], ctx->stream));
  ctx->res_bound = 0.0;
  s = enqueue_cpi_start(ctx);
  if (s != OSP_OK) return s;
  s = run_propagation(ctx, eps, ctx->n, ctx->m, true);
  if (s != OSP_OK) return s;
  s = finish_call(ctx, ctx->m, stats);
  if (s == OSP_OK || s == OSP_ENOCONV) ctx->scored = true;
  return s;
}

osp_status osp_apply_updates_device(osp_ctx* ctx, const osp_update* ops_device, int64_t U,
                                    double eps, osp_batch_stats* stats) {
  osp_status s = check_ready(ctx, true);
  if (s != OSP_OK) return s;
  if (U < 0 || U > kMaxLargeBatch) return fail(ctx, OSP_EINVAL, "batch size outside [0, 2^22]");
  if (U > 0 && !ops_device) return fail(ctx, OSP_EINVAL, "null ops");
  if (U > kMaxBatch) return apply_large(ctx, ops_device, false, U, eps, stats);
  return apply_common(ctx, ops_device, U, eps, stats);
}

osp_status osp_apply_updates(osp_ctx* ctx, const osp_update* ops, int64_t U, double eps,
                             osp_batch_stats* stats) {
  osp_status s = check_ready(ctx, true);
  if (s != OSP_OK) return s;
  if (U < 0 || U > kMaxLargeBatch) return fail(ctx, OSP_EINVAL, "batch size outside [0, 2^22]");
  if (U > 0 && !ops) return fail(ctx, OSP_EINVAL, "null ops");
  if (U > kMaxBatch) return apply_large(ctx, ops, true, U, eps, stats);
  if (U > 0) {
    const size_t bytes = sizeof(osp_update) * (size_t)U;
    std::memcpy(ctx->pinned, ops, bytes);
    CK(cudaMemcpyAsync(ctx->ops_stage, ctx->pinned, bytes, cudaMemcpyHostToDevice, ctx->stream));
  }
  return apply_common(ctx, ctx->ops_stage, U, eps, stats);
}

// Scores of seed column col in caller order into dst (device), optionally
// divided by their L1 norm.
osp_status scores_in_caller_order(osp_ctx* ctx, int col, int normalize, double* dst) {
  const int n = (int)ctx->n;
  cudaStream_t st = ctx->stream;
  if (ctx->S > 1)
    k_gather_col<<<ctx->num_sms * 4, 256, 0, st>>>(ctx->d.mu.r, ctx->d.mu.Sp, col, ctx->d.ext2int, n, dst);
  else
    k_gather_ext<<<ctx->num_sms * 4, 256, 0, st>>>(ctx->d.r, ctx->d.ext2int, n, dst);
  if (normalize) {
    k_abs_sum<<<abs_grid(ctx), 256, 0, st>>>(dst, n, ctx->dsum, ctx->dsum + 1);
    k_scale_copy<<<ctx->num_sms * 2, 256, 0, st>>>(dst, n, ctx->dsum, dst);
  }
  CK(cudaGetLastError());
  return OSP_OK;
}

osp_status osp_query_device(osp_ctx* ctx, int32_t seed_idx, int normalize, double* out_device) {
  osp_status s = check_ready(ctx, true);
  if (s != OSP_OK) return s;
  if (seed_idx < 0 || seed_idx >= ctx->S || !out_device)
    return fail(ctx, OSP_EINVAL, "bad seed index or output");
  s = scores_in_caller_order(ctx, col_for(ctx, seed_idx), normalize, out_device);
  if (s != OSP_OK) return s;
  CK(cudaStreamSynchronize(ctx->stream));
  return OSP_OK;
}

osp_status osp_query(osp_ctx* ctx, int32_t seed_idx, int normalize, double* out) {
  osp_status s = check_ready(ctx, true);
  if (s != OSP_OK) return s;
  if (seed_idx < 0 || seed_idx >= ctx->S || !out)
    return fail(ctx, OSP_EINVAL, "bad seed index or output");
  s = scores_in_caller_order(ctx, col_for(ctx, seed_idx), normalize, ctx->dtmp);
  if (s != OSP_OK) return s;
  CK(cudaMemcpyAsync(out, ctx->dtmp, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return OSP_OK;
}

osp_status osp_topk(osp_ctx* ctx, int32_t seed_idx, int32_t k, int normalize, int32_t* ids,
                    double* scores, int32_t* k_out) {
  osp_status s = check_ready(ctx, true);
  if (s != OSP_OK) return s;
  if (seed_idx < 0 || seed_idx >= ctx->S || k <= 0 || k > kTopkMaxK || !ids || !scores || !k_out)
    return fail(ctx, OSP_EINVAL, "bad seed index, k outside [1, 4096] or null output");
  cudaStream_t st = ctx->stream;
  // rank the scores in caller order, so that ties go to the smaller caller id
  const int col = col_for(ctx, seed_idx);
  double* dst = ctx->dtmp;
  s = enqueue_gather(ctx, st, &col, &dst, 1);
  if (s != OSP_OK) return s;
  const TopkScratch t{ctx->tk_state, ctx->tk_hist, ctx->tk_blk_a, ctx->tk_blk_b, ctx->tk_keys,
                      ctx->tk_ids, ctx->tk_out_ids, ctx->tk_out_sc, ctx->tk_out_k, ctx->dsum};
  TopkJobs J{};
  J.m = 1;
  J.n = (int)ctx->n;
  J.k = k;
  J.j[0] = topk_job(ctx->dtmp, t, normalize != 0);
  s = enqueue_topk(ctx, st, J);
  if (s != OSP_OK) return s;
  CK(cudaMemcpyAsync(k_out, ctx->tk_out_k, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ids, ctx->tk_out_ids, sizeof(int) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(scores, ctx->tk_out_sc, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return OSP_OK;
}

osp_status osp_query_slots(osp_ctx* ctx, int32_t nslots) {
  if (!ctx) return OSP_EINVAL;
  if (!ctx->loaded) return fail(ctx, OSP_ESTATE, "no graph loaded");
  if (nslots < 0 || nslots > kMaxQuerySlots) return fail(ctx, OSP_EINVAL, "slots outside [0, 64]");
  CK(cudaSetDevice(ctx->device));
  free_slots(ctx);
  if (nslots == 0) return OSP_OK;
  if (!ctx->qstream) {
    CK(cudaStreamCreateWithFlags(&ctx->qstream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_scores, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_queries, cudaEventDisableTiming));
    // the scores as they stand are the first snapshot queries wait for
    CK(cudaEventRecord(ctx->ev_scores, ctx->stream));
  }
  const int64_t nc = ctx->nc;
  ctx->qslots.resize(nslots);
  for (auto& q : ctx->qslots) {
    TopkScratch& t = q.t;
    osp_status s = OSP_OK;
#define QL(p, cnt)                                               \
  do {                                                           \
    s = dalloc(ctx, &(p), (size_t)(cnt), 0, &ctx->qallocs);      \
    if (s != OSP_OK) {                                           \
      free_slots(ctx);                                           \
      return s;                                                  \
    }                                                            \
  } while (0)
    QL(q.col, nc);
    QL(t.st, 1);
    QL(t.hist, 4096);
    QL(t.blk_a, nc / kTopkChunk + 2);
    QL(t.blk_b, nc / kTopkChunk + 2);
    QL(t.keys, kTopkMaxK + kTopkCand);
    QL(t.ids, kTopkMaxK + kTopkCand);
    QL(t.dsum, kAbsParts + 2);
#undef QL
    // results go straight to host-mapped memory: collecting them is a wait
    // and a host copy, with no device-to-host transfer call
    CK(cudaHostAlloc(&q.host_out, kSlotHostBytes, cudaHostAllocMapped));
    void* dev = nullptr;
    CK(cudaHostGetDevicePointer(&dev, q.host_out, 0));
    t.out_sc = (double*)dev;
    t.out_ids = (int*)((char*)dev + sizeof(double) * kTopkMaxK);
    t.out_k = t.out_ids + kTopkMaxK;
    CK(cudaEventCreateWithFlags(&q.done, cudaEventDisableTiming));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return OSP_OK;
}

osp_status osp_topk_async_many(osp_ctx* ctx, const int32_t* slots, const int32_t* seed_idx,
                               int32_t m, int32_t k, int normalize) {
  osp_status s = check_ready(ctx, true);
  if (s != OSP_OK) return s;
  if (m < 1 || m > kTopkMaxJobs || !slots || !seed_idx)
    return fail(ctx, OSP_EINVAL, "between 1 and 32 queries per call, non-null arrays");
  if (k <= 0 || k > kTopkMaxK) return fail(ctx, OSP_EINVAL, "k outside [1, 4096]");
  for (int i = 0; i < m; ++i) {
    if (slots[i] < 0 || slots[i] >= (int)ctx->qslots.size())
      return fail(ctx, OSP_EINVAL, "no such query slot");
    if (ctx->qslots[slots[i]].busy)
      return fail(ctx, OSP_ESTATE, "query slot busy (collect it with osp_topk_wait)");
    for (int j = 0; j < i; ++j)
      if (slots[j] == slots[i]) return fail(ctx, OSP_EINVAL, "a slot named twice");
    if (seed_idx[i] < 0 || seed_idx[i] >= ctx->S) return fail(ctx, OSP_EINVAL, "bad seed index");
  }
  cudaStream_t qs = ctx->qstream;
  CK(cudaStreamWaitEvent(qs, ctx->ev_scores, 0));
  int cols[kTopkMaxJobs];
  double* dsts[kTopkMaxJobs];
  TopkJobs J{};
  J.m = m;
  J.n = (int)ctx->n;
  J.k = k;
  for (int i = 0; i < m; ++i) {
    QuerySlot& q = ctx->qslots[slots[i]];
    cols[i] = col_for(ctx, seed_idx[i]);
    dsts[i] = q.col;
    J.j[i] = topk_job(q.col, q.t, normalize != 0);
  }
  s = enqueue_gather(ctx, qs, cols, dsts, m);
  if (s == OSP_OK) s = enqueue_topk(ctx, qs, J);
  if (s != OSP_OK) return s;
  for (int i = 0; i < m; ++i) {
    QuerySlot& q = ctx->qslots[slots[i]];
    CK(cudaEventRecord(q.done, qs));
    q.busy = 1;
    q.k = k;
  }
  CK(cudaEventRecord(ctx->ev_queries, qs));
  return OSP_OK;
}

osp_status osp_topk_async(osp_ctx* ctx, int32_t slot, int32_t seed_idx, int32_t k, int normalize) {
  return osp_topk_async_many(ctx, &slot, &seed_idx, 1, k, normalize);
}

osp_status osp_topk_wait(osp_ctx* ctx, int32_t slot, int32_t* ids, double* scores, int32_t* k_out) {
  if (!ctx) return OSP_EINVAL;
  if (slot < 0 || slot >= (int)ctx->qslots.size()) return fail(ctx, OSP_EINVAL, "no such query slot");
  QuerySlot& q = ctx->qslots[slot];
  if (!q.busy) return fail(ctx, OSP_ESTATE, "query slot holds no query");
  if (!ids || !scores || !k_out) return fail(ctx, OSP_EINVAL, "null output");
  CK(cudaSetDevice(ctx->device));
  CK(cudaEventSynchronize(q.done));
  q.busy = 0;
  const double* sc = (const double*)q.host_out;
  const int* id = (const int*)(sc + kTopkMaxK);
  const int kk = id[kTopkMaxK];
  std::memcpy(ids, id, sizeof(int) * kk);
  std::memcpy(scores, sc, sizeof(double) * kk);
  *k_out = kk;
  return OSP_OK;
}

osp_status osp_export_graph(osp_ctx* ctx, int direction, int64_t* ptr, int32_t* idx) {
  if (!ctx) return OSP_EINVAL;
  if (!ctx->loaded) return fail(ctx, OSP_ESTATE, "no graph loaded");
  if ((direction != 0 && direction != 1) || !ptr || (ctx->m > 0 && !idx))
    return fail(ctx, OSP_EINVAL, "bad direction or output");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  const int64_t n = ctx->n;
  const bool rows = direction == 0;
  std::vector<unsigned> off(n);
  std::vector<int> len(n);
  const unsigned long long top = rows ? ctx->top_r : ctx->top_c;
  std::vector<int> pool(std::max<unsigned long long>(top, 1));
  CK(cudaMemcpy(off.data(), rows ? ctx->d.off_r : ctx->d.off_c, sizeof(unsigned) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(len.data(), rows ? ctx->d.len_r : ctx->d.len_c, sizeof(int) * n, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(pool.data(), rows ? ctx->d.pool_r : ctx->d.pool_c, sizeof(int) * top, cudaMemcpyDeviceToHost));
  int64_t e = 0;
  for (int64_t u = 0; u < n; ++u) {  // caller node u is internal node e2i[u]
    ptr[u] = e;
    const int32_t i = ctx->e2i[u];
    for (int k = 0; k < len[i]; ++k) idx[e + k] = ctx->i2e[pool[off[i] + k]];
    std::sort(idx + e, idx + e + len[i]);
    e += len[i];
  }
  ptr[n] = e;
  return OSP_OK;
}

osp_status osp_get_size(osp_ctx* ctx, int64_t* n, int64_t* m) {
  if (!ctx || !n || !m) return OSP_EINVAL;
  *n = ctx->n;
  *m = ctx->m;
  return OSP_OK;
}

osp_status osp_get_l1_history(osp_ctx* ctx, double* out, int32_t cap, int32_t* count) {
  if (!ctx || !out || !count || cap < 0) return OSP_EINVAL;
  if (!ctx->loaded) return fail(ctx, OSP_ESTATE, "no graph loaded");
  const int k = std::min(std::min(ctx->last_iters + 1, kMaxHist), (int)cap);
  CK(cudaMemcpy(out, ctx->d.l1_hist, sizeof(double) * k, cudaMemcpyDeviceToHost));
  *count = k;
  return OSP_OK;
}

osp_status osp_get_step_times(osp_ctx* ctx, double* us, int32_t cap, int32_t* count) {
  if (!ctx || !us || !count || cap < 0) return OSP_EINVAL;
  if (!ctx->loaded) return fail(ctx, OSP_ESTATE, "no graph loaded");
  const int k = std::min(std::min(ctx->last_iters + 1, kMaxHist), (int)cap);
  std::vector<unsigned long long> t(k + 1);
  CK(cudaMemcpy(t.data(), ctx->d.step_ns, sizeof(unsigned long long) * (k + 1), cudaMemcpyDeviceToHost));
  for (int i = 0; i < k; ++i) us[i] = (double)(t[i + 1] - t[i]) * 1e-3;
  *count = k;
  return OSP_OK;
}

osp_status osp_get_seed_stats(osp_ctx* ctx, int32_t* iterations, double* qoff_l1,
                              double* last_l1, int32_t cap, int32_t* count) {
  if (!ctx || !count || cap < 0) return OSP_EINVAL;
  if (!ctx->seeded) return fail(ctx, OSP_ESTATE, "no seed set");
  CK(cudaSetDevice(ctx->device));
  const int k = std::min<int>(ctx->S, cap);
  cudaStream_t st = ctx->stream;
  if (ctx->S > 1) {
    const Multi& M = ctx->d.mu;
    const int S = ctx->S;
    std::vector<int32_t> it(S);
    std::vector<double> q(S), last(S);
    CK(cudaMemcpyAsync(it.data(), M.col_iters, sizeof(int32_t) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(q.data(), M.col_q, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(last.data(), M.col_last, sizeof(double) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int j = 0; j < k; ++j) {
      const int c = ctx->col_of[j];
      if (iterations) iterations[j] = it[c];
      if (qoff_l1) qoff_l1[j] = q[c];
      if (last_l1) last_l1[j] = last[c];
    }
  } else if (k > 0) {
    if (iterations) iterations[0] = ctx->last_iters;
    const int last = std::min(ctx->last_iters, kMaxHist - 1);
    if (qoff_l1) CK(cudaMemcpyAsync(qoff_l1, ctx->d.l1_hist, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (last_l1)
      CK(cudaMemcpyAsync(last_l1, ctx->d.l1_hist + last, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  *count = k;
  return OSP_OK;
}

osp_status osp_get_schedule(osp_ctx* ctx, int32_t* out) {
  if (!ctx || !out) return OSP_EINVAL;
  const int* sc = schedule(ctx);
  for (int i = 0; i < 4; ++i) out[i] = sc[i];
  return OSP_OK;
}

osp_status osp_set_seed_iterations(osp_ctx* ctx, const int32_t* k, int32_t S) {
  if (!ctx) return OSP_EINVAL;
  if (!ctx->seeded) return fail(ctx, OSP_ESTATE, "no seed set");
  if (k && S != ctx->S) return fail(ctx, OSP_EINVAL, "need one step count per seed");
  for (int j = 0; k && j < S; ++j)
    if (k[j] < 0 || k[j] >= kMaxHist) return fail(ctx, OSP_EINVAL, "step count out of range");
  if (ctx->S == 1) {
    ctx->fixed_iters = k ? k[0] : 0;
    return OSP_OK;
  }
  CK(cudaSetDevice(ctx->device));
  const Multi& M = ctx->d.mu;
  std::vector<int32_t> f(M.Sp, 0);
  for (int j = 0; k && j < S; ++j) f[ctx->col_of[j]] = k[j];
  int mx = 0;
  for (int v : f) mx = std::max(mx, v);
  ctx->seed_force_max = mx;
  CK(cudaMemcpyAsync(M.force, f.data(), sizeof(int32_t) * M.Sp, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return OSP_OK;
}

int64_t osp_num_nodes(const osp_ctx* ctx) { return ctx ? ctx->n : -1; }

int64_t osp_device_bytes(const osp_ctx* ctx) { return ctx ? ctx->hbm_used : -1; }

osp_status osp_get_residual_bounds(osp_ctx* ctx, double* out, int32_t cap, int32_t* count) {
  if (!ctx || !out || !count || cap < 0) return OSP_EINVAL;
  if (!ctx->seeded) return fail(ctx, OSP_ESTATE, "no seed set");
  CK(cudaSetDevice(ctx->device));
  const int k = std::min<int>(ctx->S, cap);
  if (ctx->S > 1) {
    std::vector<double> rb(ctx->S);
    CK(cudaMemcpyAsync(rb.data(), ctx->d.mu.res_bound, sizeof(double) * ctx->S,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < k; ++j) out[j] = rb[ctx->col_of[j]];
  } else if (k > 0) {
    out[0] = ctx->res_bound;
  }
  *count = k;
  return OSP_OK;
}

osp_status osp_set_fixed_iterations(osp_ctx* ctx, int32_t k) {
  if (!ctx || k < 0 || k >= kMaxHist) return OSP_EINVAL;
  ctx->fixed_iters = k;
  return OSP_OK;
}

}  // extern "C"

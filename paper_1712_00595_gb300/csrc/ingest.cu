// Batch ingest: validation, canonical ordering and net edits (one CTA), then
// the expansion of node deletions to the rows and columns they touch.
//
// Semantics (osp.h): ops apply in order; the net effect on an edge (u,v) is
// the last edge op naming it, unless u or v is deleted by the batch, in which
// case the edge is gone. Delta A (Algorithm 1) is therefore "rows after the
// whole batch minus rows before it" (Sec. 3.1, Sec. 3.4.1).
#include "common.cuh"
#include "kernels.h"

namespace osp {
namespace {

constexpr unsigned long long kNoKey = ~0ull;
constexpr int kIngestThreads = 1024;

// Exclusive scan over a 1024-thread block. Returns the prefix; *total gets the sum.
__device__ int block_exscan(int v, int* total) {
  __shared__ int s_w[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = s_w[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  int res = (w ? s_w[w - 1] : 0) + x - v;
  *total = s_w[31];
  __syncthreads();
  return res;
}

// In-place ascending bitonic sort of N (a power of two) keys in shared memory.
__device__ void bitonic_sort(unsigned long long* a, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
        int lo = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        int hi = lo | j;
        bool asc = (lo & k) == 0;
        unsigned long long x = a[lo], y = a[hi];
        if ((x > y) == asc) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

// An op with its node ids mapped to the engine's internal order. The map is a
// permutation of the loaded ids and the identity above them, so an id is in
// range before the mapping exactly when it is in range after it.
__device__ __forceinline__ osp_update load_op(const osp_update* ops, int p, const Dev& d) {
  osp_update o = ops[p];
  if (o.u >= 0 && o.u < d.nc) o.u = d.ext2int[o.u];
  if (o.v >= 0 && o.v < d.nc) o.v = d.ext2int[o.v];
  return o;
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 2;
  while (p < x) p <<= 1;
  return p;
}

// From N sorted keys whose per-position edit flags are known, write the
// insert / delete lists (ascending within each group) and one record per
// group that has at least one edit. group_of(key) gives the group node,
// member_of(key) the list value. flags[k] for k < per: bit0 insert, bit1 delete.
template <typename GroupF, typename MemberF>
__device__ void emit_groups(const unsigned long long* skey, int N, int per, int pi0,
                            const unsigned* flagbits, GroupF group_of, MemberF member_of,
                            int* ins_out, int* del_out, int* gi, int* gd, int* rec_node,
                            int* rec_is, int* rec_ic, int* rec_ds, int* rec_dc, int* flag_arr,
                            int* n_rec_out, long long* n_ins_out, long long* n_del_out) {
  unsigned fb = *flagbits;
  int my_ins = 0, my_del = 0;
  for (int k = 0; k < per; ++k) {
    my_ins += (fb >> (2 * k)) & 1;
    my_del += (fb >> (2 * k + 1)) & 1;
  }
  int tot_ins, tot_del;
  int ib = block_exscan(my_ins, &tot_ins);
  int db = block_exscan(my_del, &tot_del);
  for (int k = 0; k < per; ++k) {
    int i = pi0 + k;
    if (i >= N) break;
    gi[i] = ib;
    gd[i] = db;
    unsigned long long key = skey[i];
    if ((fb >> (2 * k)) & 1) ins_out[ib++] = member_of(key);
    if ((fb >> (2 * k + 1)) & 1) del_out[db++] = member_of(key);
  }
  if (threadIdx.x == 0) {
    gi[N] = tot_ins;
    gd[N] = tot_del;
  }
  __syncthreads();
  // one record per group (equal group node) holding at least one edit
  int my_rec = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int rb = 0;
    if (pass == 1) {
      int tot_rec;
      rb = block_exscan(my_rec, &tot_rec);
      if (threadIdx.x == 0) *n_rec_out = tot_rec;
    }
    for (int k = 0; k < per; ++k) {
      int i = pi0 + k;
      if (i >= N) break;
      unsigned long long key = skey[i];
      if (key == kNoKey) break;
      int g = group_of(key);
      if (i > 0 && group_of(skey[i - 1]) == g) continue;
      int j = i;
      while (j + 1 < N && skey[j + 1] != kNoKey && group_of(skey[j + 1]) == g) ++j;
      int ic = gi[j + 1] - gi[i], dc = gd[j + 1] - gd[i];
      if (ic + dc == 0) continue;
      if (pass == 0) {
        ++my_rec;
      } else {
        rec_node[rb] = g;
        rec_is[rb] = gi[i];
        rec_ic[rb] = ic;
        rec_ds[rb] = gd[i];
        rec_dc[rb] = dc;
        flag_arr[g] = 1;
        ++rb;
      }
    }
  }
  if (threadIdx.x == 0) {
    *n_ins_out = tot_ins;
    *n_del_out = tot_del;
  }
  __syncthreads();
}

}  // namespace

// cont != 0: a later sub-batch of one large batch. The offset accumulated so
// far (xacc, stamps, first frontier), the edge-count change and the edit
// counts carry over; only the per-sub-batch records restart.
__global__ void k_reset_batch(Dev d, int cont) {
  Ctl* c = d.ctl;
  c->status = 0;
  c->bad_op = -1;
  c->n_old = c->n;
  c->n_rec_r = 0;
  c->n_rec_c = 0;
  c->n_del = 0;
  if (cont) return;
  c->m_delta = 0;
  c->net_ins = 0;
  c->net_del = 0;
  c->n_rec_r = 0;
  c->n_rec_c = 0;
  c->n_del = 0;
  c->q_size[0] = 0;
  c->q_size[1] = 0;
  c->dense0 = 0;
  c->n_dst_nz = 0;
  c->n_src_nz = 0;
  for (int i = 0; i < 4; ++i) c->ctr[i] = 0;
  c->bar_count = 0;
  c->iter = 0;
  c->mode = kPush;
  c->push_iters = 0;
  c->stop = 0;
  c->pull_used = 0;
  c->noconv = 0;
  c->visited = 0;
  c->ef = 0;
  c->push_f = 0;
  c->push_r = 0;
}

// CPI start (Sec. 2.2): x(0) = c e_s, r = 0 before the propagation adds x(0).
// CPI start with the uniform restart vector q = 1/n0 over nodes 0..n0-1
// (PageRank mode): x(0) = c q, collected by the dense x(0) scan.
__global__ void k_cpi_begin_uniform(Dev d, int n0) {
  Ctl* c = d.ctl;
  const double x = c->c / (double)n0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x)
    d.xacc[v] = x;
  if (blockIdx.x == 0 && threadIdx.x == 0) c->dense0 = 1;
}

__global__ void k_cpi_begin(Dev d) {
  Ctl* c = d.ctl;
  int s = c->seed;
  d.xacc[s] = c->c;
  d.mark[s] = c->epoch;
  d.q0[0] = s;
  c->q_size[0] = 1;
}

__global__ void __launch_bounds__(kIngestThreads) k_ingest(Dev d, const osp_update* __restrict__ ops,
                                                           int U) {
  extern __shared__ unsigned long long skey[];
  __shared__ int s_bad, s_ndel, s_nclr, s_anyclr;
  __shared__ long long s_reins;
  __shared__ unsigned s_flags[kIngestThreads];
  Ctl* ctl = d.ctl;
  if (U < 0) U = ctl->batch_U;  // replayed from a CUDA graph: the size is set per call
  const int tid = threadIdx.x;
  const int n_old = ctl->n;
  // rows zeroed by the previous batch (merged by now) lose their mark
  const int n_clr_prev = ctl->n_clr;
  for (int i = tid; i < n_clr_prev; i += kIngestThreads) d.clr_pos[d.clr_nodes[i]] = -1;
  if (tid == 0) {
    s_bad = kNoPos;
    s_ndel = 0;
    s_nclr = 0;
    s_anyclr = 0;
    s_reins = 0;
  }
  __syncthreads();

  // ---- validation (sequential rules checked in parallel) ----
  const int per_op = (U + kIngestThreads - 1) / kIngestThreads;
  const int lo = min(U, tid * per_op), hi = min(U, lo + per_op);
  int adds = 0;
  for (int p = lo; p < hi; ++p) adds += ops[p].op == OSP_OP_ADD_NODE;
  int tot_adds;
  const int add_base = block_exscan(adds, &tot_adds);
  int run = add_base;
  for (int p = lo; p < hi; ++p) {
    osp_update o = load_op(ops, p, d);
    if (o.op == OSP_OP_ADD_NODE) {
      ++run;
    } else if (o.op == OSP_OP_DELETE_NODE) {
      const int na = n_old + run;
      const int w = o.u;
      if (w >= 0 && w < na && !d.dead[w] && !d.seedflag[w]) atomicMin(&d.del_pos[w], p);
      else atomicMin(&s_bad, p);
    } else if (o.op == OSP_OP_ZERO_ROW) {
      // the last zeroing of a row in the batch voids the row's earlier edge ops
      s_anyclr = 1;
      if (o.u >= 0 && o.u < n_old + run) atomicMax(&d.clr_pos[o.u], p);
      else atomicMin(&s_bad, p);
    }
  }
  __syncthreads();
  run = add_base;
  for (int p = lo; p < hi; ++p) {
    osp_update o = load_op(ops, p, d);
    const int na = n_old + run;
    bool ok;
    if (o.op == OSP_OP_INSERT_EDGE || o.op == OSP_OP_DELETE_EDGE) {
      ok = o.u >= 0 && o.u < na && o.v >= 0 && o.v < na && !d.dead[o.u] && !d.dead[o.v] &&
           d.del_pos[o.u] > p && d.del_pos[o.v] > p;
    } else if (o.op == OSP_OP_ADD_NODE) {
      ok = true;
      ++run;
    } else if (o.op == OSP_OP_DELETE_NODE) {
      ok = o.u >= 0 && o.u < na && !d.dead[o.u] && !d.seedflag[o.u] && d.del_pos[o.u] == p;
    } else if (o.op == OSP_OP_ZERO_ROW) {
      ok = o.u >= 0 && o.u < na && !d.dead[o.u] && d.del_pos[o.u] > p;
    } else {
      ok = false;
    }
    if (!ok) atomicMin(&s_bad, p);
  }
  __syncthreads();
  if (s_bad != kNoPos) {
    for (int p = lo; p < hi; ++p) {
      const int op = ops[p].op;
      if (op == OSP_OP_DELETE_NODE || op == OSP_OP_ZERO_ROW) {
        const osp_update o = load_op(ops, p, d);
        if (o.u >= 0 && o.u < d.nc) {
          if (op == OSP_OP_DELETE_NODE) d.del_pos[o.u] = kNoPos;
          else d.clr_pos[o.u] = -1;
        }
      }
    }
    if (tid == 0) {
      ctl->status = OSP_EINVAL;
      ctl->bad_op = s_bad;
      ctl->n_clr = 0;
    }
    return;
  }

  // ---- canonical order: sort edge ops by (u, v, position) ----
  const int N = next_pow2(U);
  for (int p = lo; p < hi; ++p) {
    osp_update o = load_op(ops, p, d);
    unsigned long long key = kNoKey;
    if ((o.op == OSP_OP_INSERT_EDGE || o.op == OSP_OP_DELETE_EDGE) && d.del_pos[o.u] == kNoPos &&
        d.del_pos[o.v] == kNoPos && (!s_anyclr || d.clr_pos[o.u] < p))
      key = ((unsigned long long)o.u << 39) | ((unsigned long long)o.v << 14) | (unsigned)p;
    skey[p] = key;
  }
  for (int i = U + tid; i < N; i += kIngestThreads) skey[i] = kNoKey;
  __syncthreads();
  bitonic_sort(skey, N);

  // ---- net edits: the last op of each (u, v) against the current row ----
  const int per = max(1, N / kIngestThreads);
  const int pi0 = tid * per;
  unsigned fb = 0;
  int reins = 0;
  for (int k = 0; k < per; ++k) {
    int i = pi0 + k;
    if (i >= N) break;
    unsigned long long key = skey[i];
    if (key == kNoKey) break;
    bool last = (i == N - 1) || ((skey[i + 1] >> 14) != (key >> 14));
    if (!last) continue;
    int p = (int)(key & 0x3FFF);
    int u = (int)(key >> 39);
    int v = (int)((key >> 14) & 0x1FFFFFF);
    bool present_after = ops[p].op == OSP_OP_INSERT_EDGE;
    bool present_before = false;
    if (u < n_old && v < n_old) {
      // u -> v exists iff v is in u's out-list, or u in v's in-list: search the shorter
      const int lr = d.len_r[u], lc = d.len_c[v];
      present_before = lr <= lc ? contains_i(d.pool_r + d.off_r[u], lr, v)
                                : contains_i(d.pool_c + d.off_c[v], lc, u);
    }
    if (s_anyclr && d.clr_pos[u] >= 0) {
      // u's row was zeroed before this op: the merge drops every old entry of
      // the row (and u from the old in-lists), so a surviving edge is written
      // again as an insertion, but it is not a new edge
      reins += present_after && present_before;
      present_before = false;
    }
    if (present_after && !present_before) fb |= 1u << (2 * k);
    if (!present_after && present_before) fb |= 2u << (2 * k);
  }
  s_flags[tid] = fb;
  if (reins) atomicAdd((unsigned long long*)&s_reins, (unsigned long long)reins);
  long long n_ins = 0, n_del = 0;
  emit_groups(
      skey, N, per, pi0, &s_flags[tid], [](unsigned long long k) { return (int)(k >> 39); },
      [](unsigned long long k) { return (int)((k >> 14) & 0x1FFFFFF); }, d.ins_r, d.del_r, d.gi,
      d.gd, d.rec_r_node, d.rec_r_is, d.rec_r_ic, d.rec_r_ds, d.rec_r_dc, d.rflag, &ctl->n_rec_r,
      &n_ins, &n_del);
  if (tid == 0) {  // summed over the sub-batches of a large batch
    ctl->net_ins += n_ins - s_reins;
    ctl->net_del += n_del;
  }

  // ---- the same edits keyed (v, u) for the in-lists ----
  // edit e of row u (in row order) -> key (v << 32) | (u << 1) | is_delete
  unsigned long long my_keys[16];
  int my_nk = 0;
  for (int k = 0; k < per && k < 16; ++k) {
    int i = pi0 + k;
    if (i >= N) break;
    if (!((fb >> (2 * k)) & 3)) continue;
    unsigned long long key = skey[i];
    unsigned long long u = key >> 39, v = (key >> 14) & 0x1FFFFFF;
    my_keys[my_nk++] = (v << 32) | (u << 1) | ((fb >> (2 * k + 1)) & 1);
  }
  int tot_e;
  const int ebase = block_exscan(my_nk, &tot_e);  // also orders the reads of skey above
  for (int t = 0; t < my_nk; ++t) skey[ebase + t] = my_keys[t];
  const int N2 = next_pow2(tot_e);
  for (int i = tot_e + tid; i < N2; i += kIngestThreads) skey[i] = kNoKey;
  __syncthreads();
  bitonic_sort(skey, N2);
  const int per2 = max(1, N2 / kIngestThreads);
  const int pj0 = tid * per2;
  unsigned fb2 = 0;
  for (int k = 0; k < per2; ++k) {
    int i = pj0 + k;
    if (i >= N2) break;
    unsigned long long key = skey[i];
    if (key == kNoKey) break;
    fb2 |= ((key & 1) ? 2u : 1u) << (2 * k);
  }
  s_flags[tid] = fb2;
  __syncthreads();
  long long c_ins = 0, c_del = 0;
  emit_groups(
      skey, N2, per2, pj0, &s_flags[tid], [](unsigned long long k) { return (int)(k >> 32); },
      [](unsigned long long k) { return (int)((unsigned)k >> 1); }, d.ins_c, d.del_c, d.gi, d.gd,
      d.rec_c_node, d.rec_c_is, d.rec_c_ic, d.rec_c_ds, d.rec_c_dc, d.cflag, &ctl->n_rec_c, &c_ins,
      &c_del);

  // ---- node deletions and additions ----
  for (int p = lo; p < hi; ++p) {
    if (ops[p].op == OSP_OP_DELETE_NODE) d.del_nodes[atomicAdd(&s_ndel, 1)] = load_op(ops, p, d).u;
    if (s_anyclr && ops[p].op == OSP_OP_ZERO_ROW) {
      const int u = load_op(ops, p, d).u;
      if (d.clr_pos[u] == p) d.clr_nodes[atomicAdd(&s_nclr, 1)] = u;  // once per row
    }
  }
  __syncthreads();
  for (int p = lo; p < hi; ++p)
    if (ops[p].op == OSP_OP_DELETE_NODE) d.del_pos[load_op(ops, p, d).u] = kNoPos;
  if (tid == 0) {
    ctl->n_del = s_ndel;
    ctl->n_clr = s_nclr;
    ctl->n = n_old + tot_adds;
  }
}

// Node deletions: the deleted node's own row and column are cleared, and every
// row / column holding it as a neighbour is re-written without it. A zeroed
// row (OSP_OP_ZERO_ROW) is re-written empty but for its insertions after the
// op, and so is every in-list holding it.
__global__ void k_expand(Dev d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int nd = ctl->n_del;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int k = gw; k < nd; k += nw) {
    const int w = d.del_nodes[k];
    if (lane == 0) {
      d.dead[w] = 1;
      if (atomicExch(&d.rflag[w], 1) == 0) {
        int at = atomicAdd(&ctl->n_rec_r, 1);
        d.rec_r_node[at] = w;
        d.rec_r_is[at] = d.rec_r_ic[at] = d.rec_r_ds[at] = d.rec_r_dc[at] = 0;
      }
      if (atomicExch(&d.cflag[w], 1) == 0) {
        int at = atomicAdd(&ctl->n_rec_c, 1);
        d.rec_c_node[at] = w;
        d.rec_c_is[at] = d.rec_c_ic[at] = d.rec_c_ds[at] = d.rec_c_dc[at] = 0;
      }
    }
    // out-neighbours x of w: column x loses source w
    const unsigned orow = d.off_r[w];
    const int lrow = d.len_r[w];
    for (int j = lane; j < lrow; j += 32) {
      int x = d.pool_r[orow + j];
      if (atomicExch(&d.cflag[x], 1) == 0) {
        int at = atomicAdd(&ctl->n_rec_c, 1);
        d.rec_c_node[at] = x;
        d.rec_c_is[at] = d.rec_c_ic[at] = d.rec_c_ds[at] = d.rec_c_dc[at] = 0;
      }
    }
    // in-neighbours x of w: row x loses target w
    const unsigned ocol = d.off_c[w];
    const int lcol = d.len_c[w];
    for (int j = lane; j < lcol; j += 32) {
      int x = d.pool_c[ocol + j];
      if (atomicExch(&d.rflag[x], 1) == 0) {
        int at = atomicAdd(&ctl->n_rec_r, 1);
        d.rec_r_node[at] = x;
        d.rec_r_is[at] = d.rec_r_ic[at] = d.rec_r_ds[at] = d.rec_r_dc[at] = 0;
      }
    }
  }
  const int nz = ctl->n_clr;
  for (int k = gw; k < nz; k += nw) {
    const int w = d.clr_nodes[k];
    if (lane == 0 && atomicExch(&d.rflag[w], 1) == 0) {
      int at = atomicAdd(&ctl->n_rec_r, 1);
      d.rec_r_node[at] = w;
      d.rec_r_is[at] = d.rec_r_ic[at] = d.rec_r_ds[at] = d.rec_r_dc[at] = 0;
    }
    // old out-neighbours x of w: column x loses source w (re-inserted if kept)
    const unsigned orow = d.off_r[w];
    const int lrow = d.len_r[w];
    for (int j = lane; j < lrow; j += 32) {
      int x = d.pool_r[orow + j];
      if (atomicExch(&d.cflag[x], 1) == 0) {
        int at = atomicAdd(&ctl->n_rec_c, 1);
        d.rec_c_node[at] = x;
        d.rec_c_is[at] = d.rec_c_ic[at] = d.rec_c_ds[at] = d.rec_c_dc[at] = 0;
      }
    }
  }
}

}  // namespace osp

// Delta-merge of the slotted graph store, fused with the offset vector.
//
// Every changed list (out-list row u, or in-list column v) is cut into pieces
// of kPiece old entries, and independent warps handle the pieces in three
// passes, so a hub list costs no more latency than a short one:
//   count  survivors of each piece (an entry goes if the batch deletes it or
//          its other end is a node deleted by the batch); for out-lists the
//          removed entries contribute q_offset[v] += (1-c) r_old[u] (0 - 1/d_u)
//   plan   per list: exclusive scan of its pieces' survivor counts, new length
//          d' = survivors + insertions, fresh pool space, new slot and (for
//          out-lists) the new (1-c)/d'
//   write  survivors go to rank + (insertions below them); each insertion goes
//          to its index + (survivors below it); for out-lists survivors
//          contribute (1-c) r_old[u] (1/d'_u - 1/d_u) and insertions
//          (1-c) r_old[u] / d'_u.
// The contributions add up to q_offset = (1-c) (B~^T - A~^T) r_old over the
// rows where B~ differs from A~ (Sec. 3.1, Algorithm 1 first step; Sec. 3.3:
// only the modified rows contribute). Every node that receives a contribution
// joins the first frontier.
#include "common.cuh"
#include "kernels.h"

namespace osp {
namespace {

// queue == false: the batch may touch more than n/beta nodes, and x(0) will be
// found by a dense scan of xacc, so no mark or queue entry is made here.
__device__ __forceinline__ void offset_add(const Dev& d, bool want, int v, double val, int epoch,
                                           bool queue) {
  if (want && !OSP_GUARD(d.ctl, v >= 0 && v < d.nc, "offset target", v, 0, 0)) want = false;
  if (d.xfix) {
    // deterministic mode: exact integer sums in units of 2^-62 (|q_offset_v| <=
    // (1-c) ||r_old||_1 < 2, and two's-complement wrap-around leaves partial
    // sums harmless), collected by the x(0) scan, so no queue either
    if (want) atomicAdd(d.xfix + v, (unsigned long long)__double2ll_rn(val * 0x1p62));
    return;
  }
  if (want) atomicAdd(&d.xacc[v], val);
  if (!queue) return;
  bool need = want && (d.mark[v] != epoch) && (atomicExch(&d.mark[v], epoch) != epoch);
  warp_append(need, v, d.q0, &d.ctl->q_size[0]);
}

// One changed list, seen through the combined record index c (out-lists first).
struct ListRec {
  bool rows;
  int node, is, ic, ds, dc;
  const int* ins;
  const int* del;
  int* pool;
};

__device__ __forceinline__ ListRec list_rec(const Dev& d, int c, int n_rows) {
  ListRec L;
  L.rows = c < n_rows;
  const int k = L.rows ? c : c - n_rows;
  if (L.rows) {
    L.node = d.rec_r_node[k];
    L.is = d.rec_r_is[k];
    L.ic = d.rec_r_ic[k];
    L.ds = d.rec_r_ds[k];
    L.dc = d.rec_r_dc[k];
    L.ins = d.ins_r;
    L.del = d.del_r;
    L.pool = d.pool_r;
  } else {
    L.node = d.rec_c_node[k];
    L.is = d.rec_c_is[k];
    L.ic = d.rec_c_ic[k];
    L.ds = d.rec_c_ds[k];
    L.dc = d.rec_c_dc[k];
    L.ins = d.ins_c;
    L.del = d.del_c;
    L.pool = d.pool_c;
  }
  return L;
}

}  // namespace

// One CTA: list each changed list's pieces and remember its old slot.
__global__ void __launch_bounds__(1024) k_merge_pieces(Dev d, double beta) {
  __shared__ int s_w[32];
  __shared__ long long s_b[32];
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int nr = ctl->n_rec_r;
  const int R = nr + ctl->n_rec_c;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (R + 1023) / 1024;
  const int lo = min(R, tid * per), hi = min(R, lo + per);
  int mine = 0;
  long long touch = 0;  // out-list entries old and new of the changed rows
  for (int c = lo; c < hi; ++c) {
    const bool rows = c < nr;
    const int node = rows ? d.rec_r_node[c] : d.rec_c_node[c - nr];
    const unsigned o = rows ? d.off_r[node] : d.off_c[node];
    const int L = rows ? d.len_r[node] : d.len_c[node];
    d.rec_old_off[c] = o;
    d.rec_old_len[c] = L;
    mine += L > 0 ? (L + kPiece - 1) / kPiece : 1;
    if (rows) touch += L + d.rec_r_ic[c];
  }
  touch = warp_sum(touch);
  if (lane == 0) s_b[w] = touch;
  int x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = s_w[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  int base = (w ? s_w[w - 1] : 0) + x - mine;
  for (int c = lo; c < hi; ++c) {
    const int L = d.rec_old_len[c];
    const int np = L > 0 ? (L + kPiece - 1) / kPiece : 1;
    d.rec_pstart[c] = base;
    for (int q = 0; q < np; ++q) d.piece_rec[base + q] = c;
    base += np;
  }
  if (tid == 0) {
    ctl->n_mpieces = s_w[31];
    d.rec_pstart[R] = s_w[31];
    long long t = 0;
    for (int i = 0; i < 32; ++i) t += s_b[i];
    // the offset reaches at most `t` nodes; above n/beta the first step is
    // dense anyway and x(0) is collected by a scan instead of a queue
    ctl->dense0 |= (double)t > (double)ctl->n / beta;  // sticky over sub-batches
  }
}

// Survivors per piece; removed out-list entries contribute to q_offset.
__global__ void __launch_bounds__(256) k_merge_count(Dev d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int np = ctl->n_mpieces, nr = ctl->n_rec_r;
  const double c1 = 1.0 - ctl->c;
  const int epoch = ctl->epoch;
  const bool queue = !ctl->dense0;
  const bool multi = ctl->multi;
  const bool any_dead = ctl->n_del > 0;  // only nodes deleted by this batch still have edges
  const bool any_clr = ctl->n_clr > 0;   // rows zeroed by this batch
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = gw; p < np; p += nw) {
    const int c = d.piece_rec[p];
    const ListRec R = list_rec(d, c, nr);
    const int q = p - d.rec_pstart[c];
    const unsigned o = d.rec_old_off[c];
    const int L = d.rec_old_len[c];
    const bool cleared =
        (any_dead && d.dead[R.node]) || (any_clr && R.rows && d.clr_pos[R.node] >= 0);
    const bool drop_clr = any_clr && !R.rows;  // in-lists drop sources whose row was zeroed
    const double ru = R.rows && !multi ? d.r[R.node] : 0.0;  // the seed block has its own offset kernel
    const bool contrib = R.rows && ru != 0.0;
    const double wa = L ? 1.0 / (double)L : 0.0;
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < kPiece / 32; ++r) {
      const int i = q * kPiece + r * 32 + lane;
      const bool in = i < L;
      int a = in ? R.pool[o + i] : 0;
      if (in && !OSP_GUARD(d.ctl, a >= 0 && a < d.nc, "merge count entry", c, i, a)) a = 0;
      const bool keep = in && !cleared && !(any_dead && d.dead[a]) &&
                        !(drop_clr && d.clr_pos[a] >= 0) && !contains_i(R.del + R.ds, R.dc, a);
      cnt += __popc(__ballot_sync(0xffffffffu, keep));
      if (contrib) offset_add(d, in && !keep, a, c1 * ru * (0.0 - wa), epoch, queue);
    }
    if (lane == 0) d.piece_cnt[p] = cnt;
  }
}

// Per list: piece bases, new length, fresh pool space, new slot.
__global__ void __launch_bounds__(256) k_merge_plan(Dev d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int nr = ctl->n_rec_r;
  const int R = nr + ctl->n_rec_c;
  const double c1 = 1.0 - ctl->c;
  const unsigned long long cap_r = ctl->pool_cap_r, cap_c = ctl->pool_cap_c;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  long long mdelta = 0;
  for (int c = gw; c < R; c += nw) {
    const ListRec L = list_rec(d, c, nr);
    const int p0 = d.rec_pstart[c], p1 = d.rec_pstart[c + 1];
    int run = 0;
    for (int b = p0; b < p1; b += 32) {  // exclusive scan of the piece counts
      const int p = b + lane;
      const int v = p < p1 ? d.piece_cnt[p] : 0;
      int x = v;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (p < p1) d.piece_base[p] = run + x - v;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    const int dp = run + L.ic;
    unsigned long long fb = 0;
    if (lane == 0 && dp > 0)
      fb = atomicAdd(L.rows ? &ctl->pool_top_r : &ctl->pool_top_c, (unsigned long long)dp);
    fb = __shfl_sync(0xffffffffu, fb, 0);
    if (fb + (unsigned long long)dp > (L.rows ? cap_r : cap_c)) {
      if (lane == 0) atomicCAS(&ctl->status, 0, (int)OSP_ENOMEM);
      return;
    }
    if (lane == 0) {
      d.rec_fbase[c] = (unsigned)fb;
      d.rec_dp[c] = dp;
      if (L.rows) {
        d.off_r[L.node] = (unsigned)fb;
        d.len_r[L.node] = dp;
        const double s = dp ? c1 / (double)dp : 0.0;
        d.scale_d[L.node] = s;
        d.scale_f[L.node] = (float)s;
        mdelta += dp - d.rec_old_len[c];
        d.rflag[L.node] = 0;
      } else {
        d.off_c[L.node] = (unsigned)fb;
        d.len_c[L.node] = dp;
        d.cflag[L.node] = 0;
      }
    }
  }
  mdelta = warp_sum(mdelta);
  if (lane == 0 && mdelta) atomicAdd((unsigned long long*)&ctl->m_delta, (unsigned long long)mdelta);
}

// Survivors and insertions to their final positions; out-list contributions.
__global__ void __launch_bounds__(256) k_merge_write(Dev d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int np = ctl->n_mpieces, nr = ctl->n_rec_r;
  const double c1 = 1.0 - ctl->c;
  const int epoch = ctl->epoch;
  const bool queue = !ctl->dense0;
  const bool multi = ctl->multi;
  const bool any_dead = ctl->n_del > 0;
  const bool any_clr = ctl->n_clr > 0;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = gw; p < np; p += nw) {
    const int c = d.piece_rec[p];
    const ListRec R = list_rec(d, c, nr);
    const int q = p - d.rec_pstart[c];
    const int npieces = d.rec_pstart[c + 1] - d.rec_pstart[c];
    const unsigned o = d.rec_old_off[c];
    const int L = d.rec_old_len[c];
    const int dp = d.rec_dp[c];
    int* F = R.pool + d.rec_fbase[c];
    const int base = d.piece_base[p];
    const int* I = R.ins + R.is;
    const int ic = R.ic;
    const bool cleared =
        (any_dead && d.dead[R.node]) || (any_clr && R.rows && d.clr_pos[R.node] >= 0);
    const bool drop_clr = any_clr && !R.rows;  // in-lists drop sources whose row was zeroed
    const double ru = R.rows && !multi ? d.r[R.node] : 0.0;  // the seed block has its own offset kernel
    const bool contrib = R.rows && ru != 0.0;
    const double wa = L ? 1.0 / (double)L : 0.0;
    const double wb = dp ? 1.0 / (double)dp : 0.0;
    const bool shift = contrib && dp != L;
    unsigned masks[kPiece / 32];
    int run = 0;
#pragma unroll
    for (int r = 0; r < kPiece / 32; ++r) {
      const int i = q * kPiece + r * 32 + lane;
      const bool in = i < L;
      int a = in ? R.pool[o + i] : 0;
      if (in && !OSP_GUARD(d.ctl, a >= 0 && a < d.nc, "merge write entry", c, i, a)) a = 0;
      const bool keep = in && !cleared && !(any_dead && d.dead[a]) &&
                        !(drop_clr && d.clr_pos[a] >= 0) && !contains_i(R.del + R.ds, R.dc, a);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      masks[r] = m;
      if (keep) {
        const int pos = base + run + __popc(m & lanemask_lt()) + lower_bound_i(I, ic, a);
        if (OSP_GUARD(d.ctl, pos >= 0 && pos < dp, "merge write position", c, pos, dp)) F[pos] = a;
      }
      run += __popc(m);
      if (shift) offset_add(d, keep, a, c1 * ru * (wb - wa), epoch, queue);
    }
    // insertions that fall inside this piece of the old list
    if (ic > 0) {
      const int* A = R.pool + o;
      const int a0 = q * kPiece;
      const int a1 = min(L, a0 + kPiece);
      const int jlo = q == 0 ? 0 : lower_bound_i(I, ic, A[a0 - 1] + 1);
      // piece q takes the insertions whose place among the old entries is in [a0, a1)
      // (the last piece also those above every old entry)
      const int jhi = q == npieces - 1 ? ic : lower_bound_i(I, ic, A[a1 - 1]);
      for (int jb = jlo; jb < jhi; jb += 32) {
        const int j = jb + lane;
        const bool in = j < jhi;
        const int e = in ? I[j] : 0;
        if (in) {
          const int t = lower_bound_i(A + a0, a1 - a0, e);  // old entries of this piece below e
          int kept = 0;
#pragma unroll
          for (int r = 0; r < kPiece / 32; ++r) {
            const int lo_r = r * 32;
            if (t >= lo_r + 32) kept += __popc(masks[r]);
            else if (t > lo_r) kept += __popc(masks[r] & ((1u << (t - lo_r)) - 1u));
          }
          if (OSP_GUARD(d.ctl, j + base + kept < dp, "merge insert position", c, j + base + kept, dp))
            F[j + base + kept] = e;
        }
        if (contrib) offset_add(d, in, e, c1 * ru * (wb - 0.0), epoch, queue);
      }
    }
  }
}

// Fold the batch's edge-count change into m.
__global__ void k_merge_finish(Dev d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  ctl->m += ctl->m_delta;
  ctl->m_delta = 0;
  ctl->n_hubs = 0;
  // a dense first frontier is rebuilt by the x(0) scan: drop entries queued by
  // earlier sub-batches of the same batch
  if (ctl->dense0) ctl->q_size[0] = 0;
}

// Pull-step plan, part 1: warp task t starts at the first node v with
// pc[v] + node_w v >= t * task_items (so a task holds about task_items items,
// an edge counting 1 and a node node_w, and never splits a list); in-lists
// longer than hub_thr are listed for piecewise summation.
__global__ void k_pull_plan(Dev d, int hub_thr, int node_w, int task_items) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int n = ctl->n;
  const long long W = (long long)node_w * n + ctl->m;
  const int nt = (int)((W + task_items - 1) / task_items);
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  if (tid == 0) {
    ctl->n_tasks = nt;
    ctl->hub_thr = hub_thr;
  }
  // f(v) = pc[v] + node_w v is nondecreasing with f(0) = 0, so the tasks t with
  // f(v-1) < t * task_items <= f(v) are exactly those starting at node v: one
  // coalesced pass over the nodes writes every task start.
  if (tid == 0) {
    d.task_first[0] = 0;
    d.task_first[nt] = n;
  }
  for (int v = tid + 1; v <= n; v += nth) {
    const long long f0 = (long long)d.pc[v - 1] + (long long)node_w * (v - 1);
    const long long f1 = (long long)d.pc[v] + (long long)node_w * v;
    const long long t0 = f0 / task_items + 1;
    const long long t1 = min(f1 / task_items, (long long)nt - 1);
    for (long long t = t0; t <= t1; ++t) d.task_first[t] = v;
  }
  const int lane = threadIdx.x & 31;
  __shared__ unsigned long long s_cnt[2];
  if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0;
  __syncthreads();
  unsigned nd = 0, ns = 0;  // destinations and sources of the pull steps (byte accounting)
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += nth) {
    const int v = base + lane;
    const int lc = v < n ? d.len_c[v] : 0;
    const bool h = lc > hub_thr;
    warp_append(h, v, d.hubs, &ctl->n_hubs);
    nd += __popc(__ballot_sync(0xffffffffu, lc > 0));
    ns += __popc(__ballot_sync(0xffffffffu, v < n && d.len_r[v] > 0));
  }
  if (lane == 0) {
    atomicAdd(&s_cnt[0], (unsigned long long)nd);
    atomicAdd(&s_cnt[1], (unsigned long long)ns);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd((unsigned long long*)&ctl->n_dst_nz, s_cnt[0]);
    if (s_cnt[1]) atomicAdd((unsigned long long*)&ctl->n_src_nz, s_cnt[1]);
  }
}

// Pull-step plan, part 2 (one CTA): piece prefix over the long in-lists.
// det != 0: the list of long in-lists, appended in whatever order the warps of
// k_pull_plan ran, is first rebuilt in ascending node order (one ordered
// compaction over all nodes), so that the pieces and the per-list norm slots
// have the same positions on every run.
__global__ void __launch_bounds__(1024) k_hub_prefix(Dev d, int hub_piece, int det) {
  __shared__ int s_w[32];
  __shared__ int s_base;
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (det) {
    const int n = ctl->n, thr = ctl->hub_thr;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += 1024) {
      const int v = b0 + tid;
      const bool h = v < n && d.len_c[v] > thr;
      const unsigned bm = __ballot_sync(0xffffffffu, h);
      if (lane == 0) s_w[w] = __popc(bm);
      __syncthreads();
      if (w == 0) {
        int x = s_w[lane];
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        s_w[lane] = x;
      }
      __syncthreads();
      if (h) d.hubs[s_base + (w ? s_w[w - 1] : 0) + __popc(bm & lanemask_lt())] = v;
      __syncthreads();
      if (tid == 0) s_base += s_w[31];
      __syncthreads();
    }
  }
  const int nh = ctl->n_hubs;
  const int per = (nh + 1023) / 1024;
  const int lo = min(nh, tid * per), hi = min(nh, lo + per);
  int mine = 0;
  for (int h = lo; h < hi; ++h) mine += (d.len_c[d.hubs[h]] + hub_piece - 1) / hub_piece;
  int x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = s_w[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  int base = (w ? s_w[w - 1] : 0) + x - mine;
  for (int h = lo; h < hi; ++h) {
    d.hub_pstart[h] = base;
    const int np = (d.len_c[d.hubs[h]] + hub_piece - 1) / hub_piece;
    for (int q = 0; q < np; ++q) d.piece_hub[base + q] = h;  // a piece finds its list in one load
    base += np;
    d.hub_acc[h] = 0.0;
    d.hub_cnt[h] = 0;
  }
  if (tid == 0) {
    d.hub_pstart[nh] = s_w[31];
    ctl->n_pieces = s_w[31];
    ctl->hub_piece = hub_piece;
  }
}

// (1-c) / d_u for every node (0 for dead-ends).
__global__ void k_set_scale(Dev d, int n, double c) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const int l = d.len_r[u];
    const double s = l ? (1.0 - c) / (double)l : 0.0;
    d.scale_d[u] = s;
    d.scale_f[u] = (float)s;
  }
}

// ---------------------------------------------------------------------------
// Compaction: exclusive scan of list lengths, then one warp per list copies it.
// ---------------------------------------------------------------------------
constexpr int kScanPer = 4;
constexpr int kScanTile = 1024 * kScanPer;

__global__ void __launch_bounds__(1024) k_scan_local(const int* __restrict__ len, unsigned* out,
                                                     unsigned* bsum, int n) {
  __shared__ unsigned s_w[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int base = blockIdx.x * kScanTile + tid * kScanPer;
  unsigned v[kScanPer];
  unsigned mine = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = base + k < n ? (unsigned)len[base + k] : 0u;
    mine += v[k];
  }
  unsigned x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned t = s_w[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  unsigned run = (w ? s_w[w - 1] : 0u) + x - mine;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (tid == 0) bsum[blockIdx.x] = s_w[31];
}

__global__ void __launch_bounds__(1024) k_scan_top(unsigned* bsum, int nb) {
  __shared__ unsigned s_w[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (nb + 1023) / 1024;
  const int lo = min(nb, tid * per), hi = min(nb, lo + per);
  unsigned mine = 0;
  for (int i = lo; i < hi; ++i) mine += bsum[i];
  unsigned x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned t = s_w[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  unsigned run = (w ? s_w[w - 1] : 0u) + x - mine;
  for (int i = lo; i < hi; ++i) {
    unsigned t = bsum[i];
    bsum[i] = run;
    run += t;
  }
}

__global__ void k_scan_add(unsigned* out, const unsigned* __restrict__ bsum, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += bsum[i / kScanTile];
}

__global__ void k_compact_copy(const unsigned* __restrict__ off_old, const int* __restrict__ len,
                               const int* __restrict__ pool_old, const unsigned* __restrict__ off_new,
                               int* pool_new, int n) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int u = gw; u < n; u += nw) {
    const unsigned a = off_old[u], b = off_new[u];
    const int l = len[u];
    for (int j = lane; j < l; j += 32) pool_new[b + j] = pool_old[a + j];
  }
}

// ||r||_1 and r / ||r||_1. With parts == nullptr the per-CTA partials are
// added atomically into *out (cleared by the caller); otherwise each CTA
// stores its partial in parts[blockIdx.x] and the last CTA to finish adds them
// in index order into *out, so the norm has the same bits on every run.
// parts[kAbsParts] (as an unsigned int) counts finished CTAs; the grid must
// not exceed kAbsParts, and the last CTA resets the count.
__global__ void k_abs_sum(const double* __restrict__ r, int n, double* out, double* parts) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += fabs(r[i]);
  s = warp_sum(s);
  __shared__ double sw[32];
  __shared__ bool s_last;
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      if (!parts) {
        atomicAdd(out, t);
      } else {
        parts[blockIdx.x] = t;
        __threadfence();
        unsigned* cnt = (unsigned*)(parts + kAbsParts);
        s_last = atomicAdd(cnt, 1u) == gridDim.x - 1;
      }
    }
  }
  if (!parts) return;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) t += __ldcg(parts + i);
    t = warp_sum(t);
    if (threadIdx.x == 0) {
      *out = t;
      *(unsigned*)(parts + kAbsParts) = 0u;
    }
  }
}

// Scores in caller order: out[x] = r[ext2int[x]].
__global__ void k_gather_ext(const double* __restrict__ r, const int* __restrict__ ext2int, int n,
                             double* out) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
    out[x] = r[ext2int[x]];
}

__global__ void k_scale_copy(const double* r, int n, const double* __restrict__ sum, double* out) {
  const double s = *sum;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = s > 0.0 ? r[i] / s : 0.0;
}

}  // namespace osp

// Delta-merge of the slotted graph store, fused with the offset vector.
//
// For every changed row u of the out-lists (one warp per row):
//   * the old list A~[u] is read once; entries that survive go to scratch
//     pool space, entries removed by the batch contribute
//       q_offset[v] += (1-c) r_old[u] (0 - 1/d_u)
//   * the surviving entries and the inserted ones are merged into fresh pool
//     space (final positions by binary search, so every lane works alone);
//     survivors contribute (1-c) r_old[u] (1/d'_u - 1/d_u) and insertions
//     (1-c) r_old[u] / d'_u.
// Together that is q_offset = (1-c) (B~^T - A~^T) r_old restricted to the rows
// where B~ differs from A~ (Sec. 3.1, Algorithm 1 first step; Sec. 3.3 notes
// that only the modified rows contribute). Every v that receives a
// contribution enters the first frontier. The in-lists are merged the same
// way without the offset.
#include "common.cuh"
#include "kernels.h"

namespace osp {
namespace {

__device__ __forceinline__ void offset_add(const Dev& d, bool want, int v, double val, int epoch) {
  if (want) atomicAdd(&d.xacc[v], val);
  bool need = want && (d.mark[v] != epoch) && (atomicExch(&d.mark[v], epoch) != epoch);
  warp_append(need, v, d.q0, &d.ctl->q_size[0]);
}

template <bool kRows>
__device__ void merge_lists(const Dev& d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int nrec = kRows ? ctl->n_rec_r : ctl->n_rec_c;
  unsigned* off = kRows ? d.off_r : d.off_c;
  int* len = kRows ? d.len_r : d.len_c;
  int* pool = kRows ? d.pool_r : d.pool_c;
  const int* ins = kRows ? d.ins_r : d.ins_c;
  const int* del = kRows ? d.del_r : d.del_c;
  const int* rnode = kRows ? d.rec_r_node : d.rec_c_node;
  const int* ris = kRows ? d.rec_r_is : d.rec_c_is;
  const int* ric = kRows ? d.rec_r_ic : d.rec_c_ic;
  const int* rds = kRows ? d.rec_r_ds : d.rec_c_ds;
  const int* rdc = kRows ? d.rec_r_dc : d.rec_c_dc;
  unsigned long long* top = kRows ? &ctl->pool_top_r : &ctl->pool_top_c;
  const unsigned long long cap = kRows ? ctl->pool_cap_r : ctl->pool_cap_c;
  const double c = ctl->c;
  const int epoch = ctl->epoch;
  const bool any_dead = ctl->n_del > 0;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  long long mdelta = 0;

  for (int rec = gw; rec < nrec; rec += nw) {
    const int u = rnode[rec];
    const int is = ris[rec], ic = ric[rec], ds = rds[rec], dc = rdc[rec];
    const unsigned o = off[u];
    const int L = len[u];
    const bool cleared = d.dead[u];
    const double ru = kRows ? d.r[u] : 0.0;
    const bool contrib = kRows && ru != 0.0;
    const double wa = L ? 1.0 / (double)L : 0.0;

    // survivors of the old list
    const int* S;
    int K;
    if (dc == 0 && !any_dead && !cleared) {
      S = pool + o;  // nothing removed: the old list is the survivor list
      K = L;
    } else {
      unsigned long long sb = 0;
      if (lane == 0 && L > 0) sb = atomicAdd(top, (unsigned long long)L);
      sb = __shfl_sync(0xffffffffu, sb, 0);
      if (sb + (unsigned long long)L > cap) {
        if (lane == 0) atomicCAS(&ctl->status, 0, (int)OSP_ENOMEM);
        return;
      }
      int* Sw = pool + sb;
      K = 0;
      for (int b = 0; b < L; b += 32) {
        const int j = b + lane;
        const bool in = j < L;
        const int a = in ? pool[o + j] : 0;
        const bool keep = in && !cleared && !d.dead[a] && !contains_i(del + ds, dc, a);
        const unsigned bm = __ballot_sync(0xffffffffu, keep);
        if (keep) Sw[K + __popc(bm & lanemask_lt())] = a;
        K += __popc(bm);
        if (contrib) offset_add(d, in && !keep, a, (1.0 - c) * ru * (0.0 - wa), epoch);
      }
      __syncwarp();
      S = Sw;
    }
    const int dp = K + ic;
    unsigned long long fb = 0;
    if (lane == 0 && dp > 0) fb = atomicAdd(top, (unsigned long long)dp);
    fb = __shfl_sync(0xffffffffu, fb, 0);
    if (fb + (unsigned long long)dp > cap) {
      if (lane == 0) atomicCAS(&ctl->status, 0, (int)OSP_ENOMEM);
      return;
    }
    int* F = pool + fb;
    const double wb = dp ? 1.0 / (double)dp : 0.0;
    const bool shift = contrib && dp != L;
    for (int b = 0; b < K; b += 32) {
      const int k = b + lane;
      const bool in = k < K;
      const int a = in ? S[k] : 0;
      if (in) F[k + lower_bound_i(ins + is, ic, a)] = a;
      if (shift) offset_add(d, in, a, (1.0 - c) * ru * (wb - wa), epoch);
    }
    for (int b = 0; b < ic; b += 32) {
      const int j = b + lane;
      const bool in = j < ic;
      const int e = in ? ins[is + j] : 0;
      if (in) F[j + lower_bound_i(S, K, e)] = e;
      if (contrib) offset_add(d, in, e, (1.0 - c) * ru * (wb - 0.0), epoch);
    }
    if (lane == 0) {
      off[u] = (unsigned)fb;
      len[u] = dp;
      if (kRows) {
        const double s = dp ? (1.0 - c) / (double)dp : 0.0;
        d.scale_d[u] = s;
        d.scale_f[u] = (float)s;
        mdelta += dp - L;
        d.rflag[u] = 0;
      } else {
        d.cflag[u] = 0;
      }
    }
  }
  if (kRows) {
    mdelta = warp_sum(mdelta);
    if (lane == 0 && mdelta) atomicAdd((unsigned long long*)&ctl->m_delta, (unsigned long long)mdelta);
  }
}

}  // namespace

__global__ void __launch_bounds__(256) k_merge_rows(Dev d) { merge_lists<true>(d); }
__global__ void __launch_bounds__(256) k_merge_cols(Dev d) { merge_lists<false>(d); }

// In-lists longer than kHubThreshold are summed in pieces by the pull step.
__global__ void k_hubs(Dev d) {
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int n = ctl->n;
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int v = base + lane;
    const bool h = v < n && d.len_c[v] > kHubThreshold;
    warp_append(h, v, d.hubs, &ctl->n_hubs);
  }
}

// Piece prefix over the hub list; also folds the batch's edge-count change into m.
__global__ void __launch_bounds__(1024) k_hub_prefix(Dev d) {
  __shared__ int s_w[32];
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int nh = ctl->n_hubs;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (nh + 1023) / 1024;
  const int lo = min(nh, tid * per), hi = min(nh, lo + per);
  int mine = 0;
  for (int h = lo; h < hi; ++h) mine += (d.len_c[d.hubs[h]] + kHubPiece - 1) / kHubPiece;
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
    base += (d.len_c[d.hubs[h]] + kHubPiece - 1) / kHubPiece;
    d.hub_acc[h] = 0.0;
    d.hub_cnt[h] = 0;
  }
  if (tid == 0) {
    d.hub_pstart[nh] = s_w[31];
    ctl->n_pieces = s_w[31];
    ctl->m += ctl->m_delta;
    ctl->m_delta = 0;
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

// ||r||_1 (one partial per CTA added atomically) and r / ||r||_1.
__global__ void k_abs_sum(const double* __restrict__ r, int n, double* out) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s += fabs(r[i]);
  s = warp_sum(s);
  __shared__ double sw[32];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sw[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) atomicAdd(out, t);
  }
}

__global__ void k_scale_copy(const double* __restrict__ r, int n, const double* __restrict__ sum,
                             double* out) {
  const double s = *sum;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = s > 0.0 ? r[i] / s : 0.0;
}

}  // namespace osp

// Offset score propagation: the cumulative power iteration of Algorithm 1,
//   x(i) = (1-c) B~^T x(i-1),  r += x(i),  until ||x(i)||_1 <= eps,
// run as one persistent cooperative kernel per call.
//
// The kernel keeps the gather vector y(i) = (1-c) x(i) / d (the scale is
// applied once per source node, so a step is a plain sum over in-edges) and
// moves between two step kinds:
//   push: x(i) is sparse. Each frontier node u scatters y(i-1)[u] to its
//         out-neighbours (atomic adds into xacc, first touch appends to the
//         next frontier); an epilogue over the new frontier adds x(i) into r,
//         forms y(i) and sums |x(i)|.
//   pull: x(i) is dense. Each node v sums y(i-1) over its in-list and the
//         same pass adds x(i) into r, writes y(i) and sums |x(i)|. Warps take
//         tasks of consecutive nodes (about equal edges + nodes) from a
//         shared counter; long lists are summed in pieces by all warps.
// The step switches to pull once the frontier's out-edges exceed m / alpha or
// its size exceeds n / beta, and stays there. Between steps a grid barrier
// (bounded wait) reduces the per-CTA |x| partials in a fixed order and takes
// the do-while stopping decision on the device, so a whole call needs no
// host round trip.
#include <type_traits>

#include "common.cuh"
#include "gridbar.cuh"
#include "kernels.h"

namespace osp {
namespace {

__device__ __forceinline__ void block_partials(const Dev& d, double l1, long long ef, double* s_l1,
                                               long long* s_ef) {
  l1 = warp_sum(l1);
  ef = warp_sum(ef);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_l1[w] = l1;
    s_ef[w] = ef;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    long long b = 0;
    for (int i = 0; i < kPropWarps; ++i) {
      a += s_l1[i];
      b += s_ef[i];
    }
    d.part_l1[blockIdx.x] = a;
    d.part_ef[blockIdx.x] = b;
  }
}

// Run by the whole last-arriving CTA: fixed-order sum of the partials and the
// stopping / step-kind decision (Algorithm 1 loop test, do-while form).
__device__ void decide(const Dev& d, const PropParams& pp, int step_mode, int n, long long m,
                       double* s_l1, long long* s_ef) {
  Ctl* ctl = d.ctl;
  double a = 0.0;
  long long b = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    a += __ldcg(d.part_l1 + i);
    b += __ldcg(d.part_ef + i);
  }
  if (pp.det && step_mode == kPull) {  // the long in-lists' |x|, in a fixed order too
    const int nh = ctl->n_hubs;
    for (int i = threadIdx.x; i < nh; i += blockDim.x) a += __ldcg(d.hub_l1 + i);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_l1[w] = a;
    s_ef[w] = b;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double L1 = 0.0;
  long long EF = 0;
  for (int i = 0; i < kPropWarps; ++i) {
    L1 += s_l1[i];
    EF += s_ef[i];
  }
  int it;
  int stop;
  if (step_mode < 0) {  // x(0)
    it = 0;
    d.l1_hist[0] = L1;
    d.step_ns[1] = global_ns();
    stop = 0;  // at least one step always runs
  } else {
    it = ctl->iter + 1;
    ctl->iter = it;
    if (it < kMaxHist) {
      d.l1_hist[it] = L1;
      d.step_ns[it + 1] = global_ns();
    }
    if (step_mode == kPush) {
      ctl->visited += ctl->ef;
      ctl->push_iters += 1;
      ctl->push_f += *(volatile int*)&ctl->q_size[(it + 1) & 1];
      ctl->push_r += *(volatile int*)&ctl->q_size[it & 1];
    } else {
      ctl->visited += m;
      ctl->pull_used = 1;
    }
    if (pp.force_iters > 0) {
      stop = it >= pp.force_iters;
    } else {
      stop = L1 <= pp.eps;
      if (!stop && it >= pp.max_iter) {
        stop = 1;
        ctl->noconv = 1;
      }
    }
    if (pp.force_iters > 0 && it >= pp.max_iter && !stop) {
      stop = 1;
      ctl->noconv = 1;
    }
  }
  int next = kPull;
  if (step_mode != kPull && !pp.det) {
    const int qs = *(volatile int*)&ctl->q_size[it & 1];
    const bool dense = (double)EF > (double)m / pp.alpha || (double)qs > (double)n / pp.beta;
    next = dense ? kPull : kPush;
  }
  ctl->ef = EF;
  ctl->mode = next;
  ctl->stop = stop;
  ctl->q_size[(it + 1) & 1] = 0;
  for (int i = 0; i < 4; ++i) ctl->ctr[i] = 0;
}

template <typename T>
__device__ void push_scatter(const Dev& d, const int* qsrc, int qs, T* ys, int* qdst,
                             int* qdst_size, int ep, int* ctr, int* big_count) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ctr, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    const int i0 = t * 32;
    if (i0 >= qs) break;
    const int i = i0 + lane;
    const bool valid = i < qs;
    int u = valid ? __ldcg(qsrc + i) : 0;
    if (!OSP_GUARD(d.ctl, u >= 0 && u < d.nc, "push frontier id", i, u, qs)) u = 0;
    T val = (T)0;
    if (valid) {
      val = __ldcg(ys + u);
      ys[u] = (T)0;
    }
    unsigned o = 0;
    int len = 0;
    if (valid && val != (T)0) {
      o = __ldg(d.off_r + u);
      len = __ldg(d.len_r + u);
    }
    const bool light = len <= kLight;
    const int ll = light ? len : 0;
    const int maxl = warp_max(ll);
    for (int j = 0; j < maxl; ++j) {
      const bool act = j < ll;
      int v = act ? __ldg(d.pool_r + o + j) : 0;
      const bool okv = !act || OSP_GUARD(d.ctl, v >= 0 && v < d.nc, "push light target", u, j, v);
      const bool act2 = act && okv;
      if (!okv) v = 0;
      if (act2) atomicAdd(&d.xacc[v], (double)val);
      const bool need = act2 && d.mark[v] != ep && atomicExch(&d.mark[v], ep) != ep;
      warp_append(need, v, qdst, qdst_size);
    }
    // rows above kHubThreshold are scattered in pieces by all warps afterwards
    const bool big = len > kHubThreshold;
    {
      const unsigned bm = __ballot_sync(0xffffffffu, big);
      if (bm) {
        int at = 0;
        const int leader = __ffs(bm) - 1;
        if (lane == leader) at = atomicAdd(big_count, __popc(bm));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (big) {
          const int slot = at + __popc(bm & lanemask_lt());
          d.big_u[slot] = u;
          d.big_y[slot] = (double)val;
        }
      }
    }
    unsigned hm = __ballot_sync(0xffffffffu, !light && !big);
    while (hm) {
      const int l = __ffs(hm) - 1;
      hm &= hm - 1;
      const unsigned ho = __shfl_sync(0xffffffffu, o, l);
      const int hl = __shfl_sync(0xffffffffu, len, l);
      const T hv = __shfl_sync(0xffffffffu, val, l);
      for (int b = 0; b < hl; b += 32) {
        const int j = b + lane;
        const bool act = j < hl;
        int v = act ? __ldg(d.pool_r + ho + j) : 0;
        const bool okv = !act || OSP_GUARD(d.ctl, v >= 0 && v < d.nc, "push heavy target", ho, j, v);
        const bool act2 = act && okv;
        if (!okv) v = 0;
        if (act2) atomicAdd(&d.xacc[v], (double)hv);
        const bool need = act2 && d.mark[v] != ep && atomicExch(&d.mark[v], ep) != ep;
        warp_append(need, v, qdst, qdst_size);
      }
    }
  }
}

// Pieces of the push rows longer than kHubThreshold, spread over all warps.
__device__ void push_big_rows(const Dev& d, int nb, int* qdst, int* qdst_size, int ep) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  int base = 0;
  for (int b = 0; b < nb; ++b) {
    const int u = __ldcg(d.big_u + b);
    const double val = __ldcg(d.big_y + b);
    const unsigned o = __ldg(d.off_r + u);
    const int len = __ldg(d.len_r + u);
    const int np = (len + kHubPiece - 1) / kHubPiece;
    for (int q = ((gw - base) % nw + nw) % nw; q < np; q += nw) {
      const int j0 = q * kHubPiece, j1 = min(len, j0 + kHubPiece);
      for (int jb = j0; jb < j1; jb += 32) {
        const int j = jb + lane;
        const bool act = j < j1;
        int v = act ? __ldg(d.pool_r + o + j) : 0;
        const bool okv = !act || OSP_GUARD(d.ctl, v >= 0 && v < d.nc, "push big target", u, j, v);
        const bool act2 = act && okv;
        if (!okv) v = 0;
        if (act2) atomicAdd(&d.xacc[v], val);
        const bool need = act2 && d.mark[v] != ep && atomicExch(&d.mark[v], ep) != ep;
        warp_append(need, v, qdst, qdst_size);
      }
    }
    base += np;
  }
}

__device__ __forceinline__ void finish_node(const Dev& d, int v, double x, void* yd, bool fp32,
                                            double& l1) {
  if (!OSP_GUARD(d.ctl, v >= 0 && v < d.nc, "finish node", v, 0, 0)) return;
  if (x != 0.0) d.r[v] += x;  // an empty in-list leaves r as it is
  l1 += fabs(x);
  if (fp32) ((float*)yd)[v] = (float)x * __ldg(d.scale_f + v);
  else ((double*)yd)[v] = x * __ldg(d.scale_d + v);
}

// Dense step. Warp tasks of about kTaskItems edges + nodes (planned per batch,
// lists never split) are taken from a shared counter; a task is walked 32
// consecutive nodes at a time. The short in-lists of such a chunk are summed as
// one flattened, coalesced stream of edges (segmented warp scan, four rounds
// of 32 edges with their loads in flight), a longer list by the whole warp
// with eight coalesced loads and gathers in flight per lane, and a list above
// kHubThreshold is cut into pieces dealt to all warps before the chunks (the
// piece that completes a list finishes it).
template <typename T>
__device__ double pull_step(const Dev& d, const T* ys, T* yd, int n_hubs, int n_pieces,
                            int n_tasks, T* wacc, int* grab, int hub_thr, int hub_piece,
                            bool det) {
  constexpr bool kF32 = std::is_same<T, float>::value;
  double l1 = 0.0;
  const int lane = threadIdx.x & 31;
  // Work items 0 .. n_pieces-1 are pieces of the long in-lists, the rest the
  // warp tasks; each warp takes the next item from a grid-wide counter, so the
  // long lists go first and warps that finish early take more of the rest.
  const int n_items = n_pieces + n_tasks;
  // Tasks are taken in a scrambled order, t -> t * P mod n_tasks (P prime and
  // coprime to n_tasks), so that the warps busy at any moment hold a mix of
  // list lengths rather than one run of neighbouring (similar) nodes.
  long long P = 7919;
  if (n_tasks % 7919 == 0) P = 7907;
  if (n_tasks % P == 0) P = 1;
  // Deterministic mode: warp gw takes items gw, gw + nw, ... instead, so every
  // lane sums its |x| terms in the same order on every run.
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int k = 0;; ++k) {
    int t = 0;
    if (det) {
      t = gw + k * nw;
    } else {
      if (lane == 0) t = atomicAdd(grab, 1);
      t = __shfl_sync(0xffffffffu, t, 0);
    }
    if (t >= n_items) break;
    if (t < n_pieces) {
      const int h = __ldg(d.piece_hub + t);  // the long list this piece belongs to
      const int v = __ldg(d.hubs + h);
      const int piece = t - __ldg(d.hub_pstart + h);
      const int full = __ldg(d.len_c + v);
      const int* p = d.pool_c + __ldg(d.off_c + v) + (unsigned)(piece * hub_piece);
      const int L = min(hub_piece, full - piece * hub_piece);
      T acc = (T)0;
      int j = lane;
      for (; j + 96 < L; j += 128) {
        const int a0 = __ldg(p + j), a1 = __ldg(p + j + 32), a2 = __ldg(p + j + 64),
                  a3 = __ldg(p + j + 96);
        acc += (ys[a0] + ys[a1]) + (ys[a2] + ys[a3]);
      }
      for (; j < L; j += 32) acc += ys[__ldg(p + j)];
      acc = warp_sum(acc);
      if (lane == 0) {
        const int np = (full + hub_piece - 1) / hub_piece;
        if (det) {
          // pieces leave their sums in slots; the last one adds them up in
          // piece order and parks |x_v| for the step's fixed-order norm sum
          d.piece_part[t] = (double)acc;
          __threadfence();
          if (atomicAdd(&d.hub_cnt[h], 1) == np - 1) {
            __threadfence();
            const double* slots = d.piece_part + (t - piece);
            double x = 0.0;
            for (int q = 0; q < np; ++q) x += __ldcg(slots + q);
            d.hub_cnt[h] = 0;
            double hl = 0.0;
            finish_node(d, v, x, yd, kF32, hl);
            d.hub_l1[h] = hl;
          }
        } else {
          atomicAdd(&d.hub_acc[h], (double)acc);
          __threadfence();
          if (atomicAdd(&d.hub_cnt[h], 1) == np - 1) {
            __threadfence();
            const double x = __longlong_as_double(
                (long long)atomicExch((unsigned long long*)&d.hub_acc[h], 0ull));
            d.hub_cnt[h] = 0;
            finish_node(d, v, x, yd, kF32, l1);
          }
        }
      }
      continue;
    }
    const int task = (int)(((long long)(t - n_pieces) * P) % n_tasks);
    const int c0 = __ldg(d.task_first + task), c1 = __ldg(d.task_first + task + 1);
    for (int vb = c0; vb < c1; vb += 32) {
      const int v = vb + lane;
      const bool valid = v < c1;
      unsigned o = 0;
      int len = 0;
      if (valid) {
        o = __ldg(d.off_c + v);
        len = __ldg(d.len_c + v);
      }
      const bool hub = len > hub_thr;
      const bool light = len <= kLight;
      // the chunk's short lists as one flattened edge stream: 32 consecutive
      // edges per round, coalesced index loads; edge e belongs to the lane l
      // with P_l <= e < P_l + len_l (P = exclusive prefix of the lengths)
      const int ll = light ? len : 0;
      int P = ll;
  #pragma unroll
      for (int q = 1; q < 32; q <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, P, q);
        if (lane >= q) P += y;
      }
      const int total = __shfl_sync(0xffffffffu, P, 31);
      P -= ll;
      wacc[lane] = (T)0;
      __syncwarp();
      constexpr int R = 4;  // rounds of 32 edges with their loads in flight together
      for (int eb = 0; eb < total; eb += 32 * R) {
        int li[R];
        unsigned addr[R];
  #pragma unroll
        for (int r = 0; r < R; ++r) {
          const int e = eb + 32 * r + lane;
          int lo = 0;  // largest lane with P <= e (lanes with empty lists share P with the next)
  #pragma unroll
          for (int q = 16; q > 0; q >>= 1) {
            const int pm = __shfl_sync(0xffffffffu, P, lo + q);
            if (pm <= e) lo += q;
          }
          const unsigned ob = __shfl_sync(0xffffffffu, o, lo);
          const int pb = __shfl_sync(0xffffffffu, P, lo);
          li[r] = e < total ? lo : -1;
          addr[r] = ob + (unsigned)(e - pb);
        }
  #pragma unroll
        for (int r = 0; r < R; ++r) addr[r] = li[r] >= 0 ? __ldg(d.pool_c + addr[r]) : 0u;
        T val[R];
  #pragma unroll
        for (int r = 0; r < R; ++r) val[r] = li[r] >= 0 ? ys[addr[r]] : (T)0;
  #pragma unroll
        for (int r = 0; r < R; ++r) {
          T v = val[r];
          const int prev = __shfl_up_sync(0xffffffffu, li[r], 1);
          const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != li[r]);
          const int seg0 = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  #pragma unroll
          for (int q = 1; q < 32; q <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, v, q);
            if (lane - q >= seg0) v += t;
          }
          const int nxt = __shfl_down_sync(0xffffffffu, li[r], 1);
          if (li[r] >= 0 && (lane == 31 || nxt != li[r])) wacc[li[r]] += v;  // one tail per list
          __syncwarp();
        }
      }
      T s = wacc[lane];
      // longer lists: the whole warp, blocks of 256 entries (eight coalesced id
      // loads and gathers per lane); the ids of the next block (of this list or
      // the next one) load while the current block's gathers are in flight
      unsigned hm = __ballot_sync(0xffffffffu, !light && !hub);
      if (hm) {
        int l = __ffs(hm) - 1;
        hm &= hm - 1;
        const int* p = d.pool_c + __shfl_sync(0xffffffffu, o, l);
        int hl = __shfl_sync(0xffffffffu, len, l);
        int jb = 0;
        int a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = 32 * q + lane < hl ? __ldg(p + 32 * q + lane) : -1;
        T acc = (T)0;
        for (;;) {
          T t[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) t[q] = a[q] >= 0 ? ys[a[q]] : (T)0;
          // the next block: the rest of this list, else the next long list
          const bool same = jb + 256 < hl;
          int nl = l, nhl = hl, njb = jb + 256;
          const int* np = p;
          if (!same && hm) {
            nl = __ffs(hm) - 1;
            nhl = __shfl_sync(0xffffffffu, len, nl);
            np = d.pool_c + __shfl_sync(0xffffffffu, o, nl);
            njb = 0;
          }
          const bool more = same || hm != 0;
          if (more) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = njb + 32 * q + lane;
              a[q] = j < nhl ? __ldg(np + j) : -1;
            }
          }
          acc += ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
          if (!same) {  // list l is complete
            const T tot = warp_sum(acc);
            if (lane == l) s = tot;
            acc = (T)0;
            if (!hm) break;
            hm &= hm - 1;
          }
          l = nl;
          hl = nhl;
          p = np;
          jb = njb;
        }
      }
      if (valid && !hub) finish_node(d, v, (double)s, yd, kF32, l1);
    }
  }
  return l1;
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kPropThreads, 4) k_propagate(Dev d, PropParams pp) {
  __shared__ BarShared sh;
  __shared__ double s_l1[kPropWarps];
  __shared__ long long s_ef[kPropWarps];
  __shared__ T s_wacc[kPropThreads];  // per-warp accumulators of the short-list stream
  __shared__ int s_qw[kPropWarps];     // dense x(0) scan: queue offsets of the warps
  __shared__ int s_qbase;
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int n = ctl->n;
  const long long m = ctl->m;
  const int epoch = ctl->epoch;
  const int n_hubs = ctl->n_hubs;
  const int n_pieces = ctl->n_pieces;
  const int n_tasks = ctl->n_tasks;
  const int hub_thr = ctl->hub_thr, hub_piece = ctl->hub_piece;
  T* yb[2] = {(T*)d.y0, (T*)d.y1};
  int* qb[2] = {d.q0, d.q1};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  if (tid == 0) d.step_ns[0] = global_ns();

  // x(0) (the offset vector, or c e_s for CPI) sits in xacc over queue 0
  {
    double l1 = 0.0;
    long long ef = 0;
    const int qs = *(volatile int*)&ctl->q_size[0];
    if (!OSP_GUARD(ctl, qs >= 0 && qs <= d.nc, "first frontier size", qs, 0, 0)) return;
    if (pp.det) {
      // Deterministic mode: every step pulls, so no frontier queue is kept; a
      // fixed pass over all nodes collects x(0) from xacc and from the merge's
      // fixed-point accumulator (exact integer sums, so their order is moot).
      for (int v = tid; v < n; v += nthreads) {
        double x = __ldcg(d.xacc + v);
        const long long q = (long long)__ldcg(d.xfix + v);
        if (q != 0) {
          x += (double)q * 0x1p-62;
          d.xfix[v] = 0ull;
        }
        if (x != 0.0) {
          d.xacc[v] = 0.0;
          d.r[v] += x;
          l1 += fabs(x);
          yb[0][v] = (T)(x * __ldg(d.scale_d + v));
          ef += __ldg(d.len_r + v);
        }
      }
    } else if (*(volatile int*)&ctl->dense0) {
      // The merge reached more than n/beta nodes and queued none of them: one
      // coalesced pass over all nodes collects x(0) (xacc is zero off its
      // support) and builds the frontier queue of its nonzero entries.
      // One queue reservation per CTA tile of 4 x blockDim.x nodes, whose x
      // values load together (the loop is uniform over the CTA).
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      for (int base = blockIdx.x * 4 * blockDim.x; base < n; base += 4 * nthreads) {
        double xs[4];
        int vs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          vs[k] = base + k * blockDim.x + threadIdx.x;
          xs[k] = vs[k] < n ? __ldcg(d.xacc + vs[k]) : 0.0;
        }
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (xs[k] != 0.0) {
            const int v = vs[k];
            d.xacc[v] = 0.0;
            d.r[v] += xs[k];
            l1 += fabs(xs[k]);
            yb[0][v] = (T)(xs[k] * __ldg(d.scale_d + v));
            ef += __ldg(d.len_r + v);
            ++cnt;
          }
        }
        int inc = cnt;  // inclusive warp scan of the counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        if (lane == 31) s_qw[w] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
          int t = 0;
          for (int i = 0; i < kPropWarps; ++i) {
            const int c = s_qw[i];
            s_qw[i] = t;
            t += c;
          }
          s_qbase = t ? atomicAdd(&ctl->q_size[0], t) : 0;
        }
        __syncthreads();
        int pos = s_qbase + s_qw[w] + inc - cnt;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (xs[k] != 0.0) d.q0[pos++] = vs[k];
        __syncthreads();
      }
    } else {
      for (int k = tid; k < qs; k += nthreads) {
        const int v = __ldcg(d.q0 + k);
        if (!OSP_GUARD(ctl, v >= 0 && v < d.nc, "first frontier id", k, v, qs)) continue;
        const double x = __ldcg(d.xacc + v);
        d.xacc[v] = 0.0;
        d.r[v] += x;
        l1 += fabs(x);
        yb[0][v] = (T)(x * __ldg(d.scale_d + v));
        ef += __ldg(d.len_r + v);
      }
    }
    block_partials(d, l1, ef, s_l1, s_ef);
    if (bar_arrive(ctl, sh)) decide(d, pp, -1, n, m, s_l1, s_ef);
    if (!bar_release(ctl, sh)) return;
  }

  for (int it = 1;; ++it) {
    if (*(volatile int*)&ctl->stop) break;
    const int mode = *(volatile int*)&ctl->mode;
    const int src = (it - 1) & 1, dst = it & 1;
    double l1 = 0.0;
    long long ef = 0;
    if (mode == kPush) {
      const int qs = *(volatile int*)&ctl->q_size[src];
      push_scatter<T>(d, qb[src], qs, yb[src], qb[dst], &ctl->q_size[dst], epoch + it,
                      &ctl->ctr[0], &ctl->ctr[2]);
      if (bar_arrive(ctl, sh) && threadIdx.x == 0) ctl->ctr[0] = 0;
      if (!bar_release(ctl, sh)) return;
      const int nbig = *(volatile int*)&ctl->ctr[2];
      if (nbig > 0) {  // uniform: every CTA read the same count after the barrier
        push_big_rows(d, nbig, qb[dst], &ctl->q_size[dst], epoch + it);
        if (bar_arrive(ctl, sh) && threadIdx.x == 0) ctl->ctr[2] = 0;
        if (!bar_release(ctl, sh)) return;
      }
      const int qn = *(volatile int*)&ctl->q_size[dst];
      T* yd = yb[dst];
      for (int k = tid; k < qn; k += nthreads) {
        const int v = __ldcg(qb[dst] + k);
        if (!OSP_GUARD(ctl, v >= 0 && v < d.nc && qn <= d.nc, "frontier id", k, v, qn)) continue;
        const double x = __ldcg(d.xacc + v);
        d.xacc[v] = 0.0;
        d.r[v] += x;
        l1 += fabs(x);
        yd[v] = (T)(x * __ldg(d.scale_d + v));
        ef += __ldg(d.len_r + v);
      }
    } else {
      l1 = pull_step<T>(d, yb[src], yb[dst], n_hubs, n_pieces, n_tasks,
                        s_wacc + (threadIdx.x & ~31), &ctl->ctr[1], hub_thr, hub_piece,
                        pp.det != 0);
    }
    block_partials(d, l1, ef, s_l1, s_ef);
    if (bar_arrive(ctl, sh)) decide(d, pp, mode, n, m, s_l1, s_ef);
    if (!bar_release(ctl, sh)) return;
  }

  // leave both gather vectors all-zero for the next call
  const int k_last = *(volatile int*)&ctl->iter;
  if (*(volatile int*)&ctl->pull_used) {
    T* a = yb[0];
    T* b = yb[1];
    for (int v = tid; v < n; v += nthreads) {
      a[v] = (T)0;
      b[v] = (T)0;
    }
  } else {
    const int last = k_last & 1;
    const int qs = *(volatile int*)&ctl->q_size[last];
    for (int k = tid; k < qs; k += nthreads) yb[last][__ldcg(qb[last] + k)] = (T)0;
  }
  if (tid == 0) ctl->epoch = epoch + k_last + 1;
}

template __global__ void k_propagate<double>(Dev, PropParams);
template __global__ void k_propagate<float>(Dev, PropParams);

int propagate_grid(int fp32, int num_sms) {
  int bps = 0;
  cudaError_t e = fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_propagate<float>,
                                                                       kPropThreads, 0)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_propagate<double>,
                                                                       kPropThreads, 0);
  if (e != cudaSuccess || bps <= 0) return 0;
  bps = bps > 4 ? 4 : bps;
  int g = bps * num_sms;
  return g > kMaxGrid ? kMaxGrid : g;
}

cudaError_t launch_propagate(const Dev& d, const PropParams& pp, int grid, cudaStream_t s) {
  Dev dd = d;
  PropParams p = pp;
  void* args[] = {&dd, &p};
  const void* fn = pp.fp32 ? (const void*)k_propagate<float> : (const void*)k_propagate<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPropThreads), args, 0, s);
}

}  // namespace osp

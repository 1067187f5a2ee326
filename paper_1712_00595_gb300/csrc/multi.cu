// Several seeds at once: the columns of an n x Sp block (Sp = 32 K) each hold
// the RWR vector of one seed, so every step of Algorithm 1 becomes a sparse
// matrix times a dense block (SpMM) and every gathered source brings K
// contiguous values per lane instead of one.
//
//   offset   q_offset = (1-c)(B~^T - A~^T) R_old over the changed rows u
//            (Sec. 3.1, 3.3): row u adds (1-c) R_old[u] / d'_u to every entry
//            of its new out-list and subtracts (1-c) R_old[u] / d_u from every
//            entry of its old out-list (old lists stay readable: the merge
//            writes new lists out of place); an entry in both lists gets the
//            difference in one addition. Targets get this call's stamp.
//   x(0)     one pass over all nodes: stamped rows move from xacc into R and
//            the first gather block y(0) = x(0) (1-c) / d; other rows of y(0)
//            are written as zero.
//   steps    pull only: x(i)[v] = sum over the in-list of v of y(i-1)[u],
//            a warp per node, lanes over columns; long in-lists in pieces.
//   stop     per column (Algorithm 1 loop test, do-while form): a column whose
//            ||x(i)||_1 <= eps stops adding and propagating; the call ends
//            when no column is left or at the iteration cap.
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "gridbar.cuh"
#include "kernels.h"

namespace osp {
namespace {

template <typename TY> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ __nv_bfloat16 from_acc(float v, __nv_bfloat16*) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from_acc(float v, float*) { return v; }
__device__ __forceinline__ double from_acc(double v, double*) { return v; }

// K contiguous elements (K * sizeof(T) bytes, naturally aligned) through L2.
template <typename T, int K>
__device__ __forceinline__ void load_cg(const T* p, T (&out)[K]) {
  constexpr int B = K * (int)sizeof(T);
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i)
      reinterpret_cast<uint4*>(out)[i] = __ldcg(reinterpret_cast<const uint4*>(p) + i);
  } else if constexpr (B == 8) {
    *reinterpret_cast<uint2*>(out) = __ldcg(reinterpret_cast<const uint2*>(p));
  } else if constexpr (B == 4) {
    *reinterpret_cast<unsigned*>(out) = __ldcg(reinterpret_cast<const unsigned*>(p));
  } else {
    *reinterpret_cast<unsigned short*>(out) = __ldcg(reinterpret_cast<const unsigned short*>(p));
  }
}

template <typename T, int K>
__device__ __forceinline__ void store_k(T* p, const T (&v)[K]) {
  constexpr int B = K * (int)sizeof(T);
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i)
      reinterpret_cast<uint4*>(p)[i] = reinterpret_cast<const uint4*>(v)[i];
  } else if constexpr (B == 8) {
    *reinterpret_cast<uint2*>(p) = *reinterpret_cast<const uint2*>(v);
  } else if constexpr (B == 4) {
    *reinterpret_cast<unsigned*>(p) = *reinterpret_cast<const unsigned*>(v);
  } else {
    *reinterpret_cast<unsigned short*>(p) = *reinterpret_cast<const unsigned short*>(v);
  }
}

// Per-column |x| partials of this CTA: lanes hold their K columns; warps are
// combined in shared memory in a fixed order.
template <int K>
__device__ __forceinline__ void column_partials(const Multi& M, const double (&l1)[K],
                                                double* s_part) {
  constexpr int Sp = 32 * K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) s_part[w * Sp + lane * K + k] = l1[k];
  __syncthreads();
  for (int j = threadIdx.x; j < Sp; j += blockDim.x) {
    double a = 0.0;
    for (int i = 0; i < kPropWarps; ++i) a += s_part[i * Sp + j];
    M.part[(size_t)blockIdx.x * Sp + j] = a;
  }
  __threadfence();
}

// Whole last CTA: per-column sums of the partials (fixed order over CTAs),
// per-column stopping, the call's stop and the history entry (max over the
// columns that ran the step).
template <int K>
__device__ void decide_multi(const Dev& d, const PropParams& pp, int it, long long m) {
  constexpr int Sp = 32 * K;
  const Multi& M = d.mu;
  Ctl* ctl = d.ctl;
  __shared__ double s_max[kPropThreads / 32];
  __shared__ double s_sum[kPropThreads];
  // thread t sums column t % Sp over the CTAs b = t / Sp (mod Q) with eight
  // independent accumulators; the Q slices are then added in a fixed order
  const int Q = (int)blockDim.x / Sp;
  const int G = (int)gridDim.x;
  {
    const int jc = threadIdx.x % Sp, q = threadIdx.x / Sp;
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 0.0;
    for (int b = q; b < G; b += 8 * Q) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int bb = b + u * Q;
        if (bb < G) a[u] += __ldcg(M.part + (size_t)bb * Sp + jc);
      }
    }
    s_sum[threadIdx.x] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  __syncthreads();
  double seen = 0.0;
  int live = 0;
  for (int j = threadIdx.x; j < Sp; j += blockDim.x) {
    double L = 0.0;
    for (int q = 0; q < Q; ++q) L += s_sum[q * Sp + j];
    if (j >= M.S) continue;
    if (it == 0) {
      M.col_q[j] = L;
      M.col_last[j] = L;
      M.col_iters[j] = 0;
      M.active[j] = 1;
      seen = fmax(seen, L);
      live = 1;
    } else if (*(volatile int*)&M.active[j]) {
      M.col_iters[j] = it;
      M.col_last[j] = L;
      seen = fmax(seen, L);
      const int f = pp.force_iters > 0 ? pp.force_iters : M.force[j];
      int stop = f > 0 ? it >= f : L <= pp.eps;
      if (!stop && it >= pp.max_iter) {
        stop = 1;
        ctl->noconv = 1;
      }
      if (stop) M.active[j] = 0;
      else live = 1;
    }
  }
  seen = warp_max(seen);
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = seen;
  const int any = __syncthreads_or(live);
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < kPropWarps; ++i) mx = fmax(mx, s_max[i]);
    if (it < kMaxHist) {
      d.l1_hist[it] = mx;
      d.step_ns[it + 1] = global_ns();
    }
    ctl->iter = it;
    if (it > 0) {
      ctl->visited += m;
      ctl->pull_used = 1;
    }
    ctl->stop = !any;
    for (int i = 0; i < 4; ++i) ctl->ctr[i] = 0;
  }
}

// x(i)[v] from the K-column sums acc: add into R for running columns (rr is
// the row of R, loaded before the sums), write the next gather row (zero for
// stopped columns), accumulate |x|.
template <typename TY, int K, typename A>
__device__ __forceinline__ void finish_row(const Dev& d, int v, const A (&acc)[K], A s,
                                           double (&rr)[K], unsigned act, TY* yd,
                                           double (&l1)[K]) {
  constexpr int Sp = 32 * K;
  const int lane = threadIdx.x & 31;
  const size_t base = (size_t)v * Sp + lane * K;
  alignas(16) TY yv[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (act & (1u << k)) {
      const double x = (double)acc[k];
      rr[k] += x;
      l1[k] += fabs(x);
      yv[k] = from_acc((A)(acc[k] * s), (TY*)nullptr);
    } else {
      yv[k] = from_acc((A)0, (TY*)nullptr);
    }
  }
  store_k(d.mu.r + base, rr);
  store_k(yd + base, yv);
}

template <typename A>
__device__ __forceinline__ A scale_of(const Dev& d, int v) {
  return std::is_same<A, double>::value ? (A)__ldg(d.scale_d + v) : (A)__ldg(d.scale_f + v);
}

// Sum of y rows over in-list entries p[0 .. len): 32 ids per coalesced load,
// then up to eight rows in flight.
template <typename TY, int K, typename A>
__device__ __forceinline__ void sum_rows(const int* p, int len, const TY* ys, A (&acc)[K],
                                         int idx0 = -1) {
  constexpr int Sp = 32 * K;
  const int lane = threadIdx.x & 31;
  for (int b = 0; b < len; b += 32) {
    const int cnt = min(32, len - b);
    // ids of the first block may come preloaded (idx0 >= 0 on every lane)
    const int idx = (b == 0 && __all_sync(0xffffffffu, idx0 >= 0)) ? idx0
                    : (lane < cnt ? __ldg(p + b + lane) : 0);
    int j = 0;
    for (; j + 8 <= cnt; j += 8) {
      alignas(16) TY a[8][K];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int u = __shfl_sync(0xffffffffu, idx, j + q);
        load_cg(ys + (size_t)u * Sp + lane * K, a[q]);
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
        acc[k] += ((to_acc(a[0][k]) + to_acc(a[1][k])) + (to_acc(a[2][k]) + to_acc(a[3][k]))) +
                  ((to_acc(a[4][k]) + to_acc(a[5][k])) + (to_acc(a[6][k]) + to_acc(a[7][k])));
    }
    if (j + 4 <= cnt) {
      alignas(16) TY a[4][K];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = __shfl_sync(0xffffffffu, idx, j + q);
        load_cg(ys + (size_t)u * Sp + lane * K, a[q]);
      }
#pragma unroll
      for (int k = 0; k < K; ++k)
        acc[k] += (to_acc(a[0][k]) + to_acc(a[1][k])) + (to_acc(a[2][k]) + to_acc(a[3][k]));
      j += 4;
    }
    for (; j < cnt; ++j) {
      const int u = __shfl_sync(0xffffffffu, idx, j);
      alignas(16) TY a[K];
      load_cg(ys + (size_t)u * Sp + lane * K, a);
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += to_acc(a[k]);
    }
  }
}

// ---------------------------------------------------------------------------
// Whole-row staging through shared memory. Each warp owns two buffers of
// RingCfg::kRows source rows; a batch of rows of one in-list is copied into a
// buffer by cp.async.bulk (one copy per row, issued by one lane each), and the
// buffer's mbarrier completes once the batch's bytes have landed (transaction
// count = rows x row bytes). The copies need no registers, so many more rows
// are in flight per warp than with register gathers.
// ---------------------------------------------------------------------------
constexpr int kRingBytesPerWarp = 11 * 1024;
constexpr unsigned long long kRingTimeoutNs = 2000000000ull;  // 2 s

template <typename TY, int K>
struct RingCfg {
  static constexpr int kRowBytes = 32 * K * (int)sizeof(TY);  // a multiple of 16
  static constexpr int kFit = kRingBytesPerWarp / (2 * kRowBytes);
  static constexpr int kRows = kFit < 1 ? 1 : (kFit > 32 ? 32 : kFit);
  static constexpr int kBarBytes = 16 * kPropWarps;  // two mbarriers per warp
  static constexpr int kSmem = kBarBytes + kPropWarps * 2 * kRows * kRowBytes;
  // bulk copies need 16-byte aligned addresses and sizes
  static_assert(kRowBytes % 16 == 0 && kBarBytes % 16 == 0, "staged rows must stay 16-byte aligned");
  static_assert(kSmem <= 100 * 1024, "two CTAs per SM must fit with the static shared memory");
};

struct Ring {
  unsigned bar;                 // shared address of the warp's mbarrier 0 (mbarrier 1 follows)
  unsigned rows;                // shared address of the warp's buffer 0 (buffer 1 follows)
  const unsigned char* rows_g;  // the same, as a generic pointer
  unsigned phase;               // bit b: parity of buffer b's next completion
  int buf;                      // the buffer the next batch goes to
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive (the barrier's one expected arrival) and add `bytes` to the
// transaction count the current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Order this thread's generic-proxy accesses to shared memory before later
// async-proxy ones (a bulk copy overwriting rows that were just read).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_row(unsigned dst, const void* src, unsigned bytes,
                                              unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Rows u (lane j < cnt holds row j's id) of the gather block into buffer b.
template <typename TY, int K>
__device__ __forceinline__ void ring_issue(const Ring& rg, int b, int cnt, int u, const TY* ys) {
  using C = RingCfg<TY, K>;
  const int lane = threadIdx.x & 31;
  const unsigned bar = rg.bar + 8u * (unsigned)b;
  __syncwarp();  // the warp's reads of buffer b are done ...
  fence_proxy_async_smem();  // ... and come before the copies that overwrite it
  if (lane == 0) mbar_arrive_expect(bar, (unsigned)(cnt * C::kRowBytes));
  __syncwarp();
  if (lane < cnt)
    bulk_copy_row(rg.rows + (unsigned)((b * C::kRows + lane) * C::kRowBytes),
                  ys + (size_t)u * (32 * K), (unsigned)C::kRowBytes, bar);
}

// Wait for buffer b's batch. Bounded: after 2 s the call's status becomes
// OSP_ETIMEOUT (the next grid barrier then ends the kernel) and the warp
// waits once more, again bounded, for its copies in flight.
__device__ __forceinline__ void ring_wait(Ring& rg, int b, Ctl* ctl) {
  const unsigned bar = rg.bar + 8u * (unsigned)b;
  const unsigned par = (rg.phase >> b) & 1u;
  if (!mbar_try_wait(bar, par)) {
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (!mbar_try_wait(bar, par)) {
      if ((++spins & 255u) == 0 && global_ns() - t0 > kRingTimeoutNs) {
        if ((threadIdx.x & 31) == 0) atomicCAS(&ctl->status, 0, (int)OSP_ETIMEOUT);
        const unsigned long long t1 = global_ns();
        while (!mbar_try_wait(bar, par) && global_ns() - t1 < kRingTimeoutNs) {
        }
        break;
      }
    }
  }
  rg.phase ^= 1u << b;
}

// K-element slice of a staged row (plain loads from shared memory).
template <typename T, int K>
__device__ __forceinline__ void load_k(const T* p, T (&out)[K]) {
  constexpr int B = K * (int)sizeof(T);
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i)
      reinterpret_cast<uint4*>(out)[i] = reinterpret_cast<const uint4*>(p)[i];
  } else if constexpr (B == 8) {
    *reinterpret_cast<uint2*>(out) = *reinterpret_cast<const uint2*>(p);
  } else if constexpr (B == 4) {
    *reinterpret_cast<unsigned*>(out) = *reinterpret_cast<const unsigned*>(p);
  } else {
    *reinterpret_cast<unsigned short*>(out) = *reinterpret_cast<const unsigned short*>(p);
  }
}

// acc += the cnt rows staged in buffer b (this lane's K columns).
template <typename TY, int K, typename A>
__device__ __forceinline__ void ring_sum(const Ring& rg, int b, int cnt, A (&acc)[K]) {
  using C = RingCfg<TY, K>;
  constexpr int Sp = 32 * K;
  const int lane = threadIdx.x & 31;
  const TY* row = reinterpret_cast<const TY*>(rg.rows_g + (size_t)b * C::kRows * C::kRowBytes) +
                  lane * K;
  int j = 0;
  if constexpr (K * sizeof(TY) < 64) {  // four rows at a time while they fit in few registers
    for (; j + 4 <= cnt; j += 4) {
      alignas(16) TY a[4][K];
#pragma unroll
      for (int q = 0; q < 4; ++q) load_k(row + (j + q) * Sp, a[q]);
#pragma unroll
      for (int k = 0; k < K; ++k)
        acc[k] += (to_acc(a[0][k]) + to_acc(a[1][k])) + (to_acc(a[2][k]) + to_acc(a[3][k]));
    }
  } else {
    for (; j + 2 <= cnt; j += 2) {
      alignas(16) TY a[2][K];
#pragma unroll
      for (int q = 0; q < 2; ++q) load_k(row + (j + q) * Sp, a[q]);
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] += to_acc(a[0][k]) + to_acc(a[1][k]);
    }
  }
  for (; j < cnt; ++j) {
    alignas(16) TY a[K];
    load_k(row + j * Sp, a);
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += to_acc(a[k]);
  }
}

// acc += the rows of y over in-list entries p[0 .. L), L >= 1, staged in
// batches of kRows, two batches in flight.
template <typename TY, int K, typename A>
__device__ void ring_sum_list(Ring& rg, const Dev& d, const int* p, int L, const TY* ys,
                              A (&acc)[K]) {
  constexpr int G = RingCfg<TY, K>::kRows;
  const int lane = threadIdx.x & 31;
  auto ids = [&](int s0) -> int {
    const bool in = lane < min(G, L - s0);
    int u = in ? __ldg(p + s0 + lane) : 0;
    if (in && !OSP_GUARD(d.ctl, u >= 0 && u < d.nc, "multi staged piece id", s0, lane, u)) u = 0;
    return u;
  };
  int b = rg.buf;
  ring_issue<TY, K>(rg, b, min(G, L), ids(0), ys);
  for (int s0 = 0; s0 < L; s0 += G) {
    if (s0 + G < L) ring_issue<TY, K>(rg, b ^ 1, min(G, L - s0 - G), ids(s0 + G), ys);
    ring_wait(rg, b, d.ctl);
    ring_sum<TY, K, A>(rg, b, min(G, L - s0), acc);
    b ^= 1;
  }
  rg.buf = b;
}

// A batch of the staged stream: rows s .. s + cnt - 1 of the in-list of the
// chunk's node lane jc (list at pool_c + off).
struct RowBatch {
  int jc, s, cnt;
  unsigned off;
  bool first, last;
};

}  // namespace

// One CTA: offset items of the changed rows (256 entries of old + new list each).
__global__ void __launch_bounds__(1024) k_offset_multi_plan(Dev d) {
  __shared__ int s_w[32];
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int nr = ctl->n_rec_r;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (nr + 1023) / 1024;
  const int lo = min(nr, tid * per), hi = min(nr, lo + per);
  int mine = 0;
  for (int c = lo; c < hi; ++c) mine += (d.rec_old_len[c] + d.rec_dp[c] + kPiece - 1) / kPiece;
  int x = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = s_w[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s_w[lane] = t;
  }
  __syncthreads();
  int base = (w ? s_w[w - 1] : 0) + x - mine;
  for (int c = lo; c < hi; ++c) {
    const int np = (d.rec_old_len[c] + d.rec_dp[c] + kPiece - 1) / kPiece;
    d.rec_pstart[c] = base;
    for (int q = 0; q < np; ++q) d.piece_rec[base + q] = c;
    base += np;
  }
  if (tid == 0) ctl->n_opieces = s_w[31];
}

// Warp per offset item: R_old[u] times -(1-c)/d_u into xacc over the old
// out-list entries, times +(1-c)/d'_u over the new ones (one combined term
// for an entry in both lists); stamps the targets.
template <int K>
__global__ void __launch_bounds__(256) k_offset_multi(Dev d) {
  constexpr int Sp = 32 * K;
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  const int np = ctl->n_opieces;
  const double c1 = 1.0 - ctl->c;
  const int epoch = ctl->epoch;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int p = gw; p < np; p += nw) {
    const int c = d.piece_rec[p];
    const int q = p - d.rec_pstart[c];
    const int u = d.rec_r_node[c];
    const int L = d.rec_old_len[c], dp = d.rec_dp[c];
    alignas(16) double ru[K];
    load_cg(d.mu.r + (size_t)u * Sp + lane * K, ru);
    bool nz = false;
#pragma unroll
    for (int k = 0; k < K; ++k) nz |= ru[k] != 0.0;
    if (!__any_sync(0xffffffffu, nz)) continue;
    const double wa = L ? c1 / (double)L : 0.0;
    const double wb = dp ? c1 / (double)dp : 0.0;
    const int* oldl = d.pool_r + d.rec_old_off[c];
    const int* newl = d.pool_r + d.rec_fbase[c];
    const int e0 = q * kPiece, e1 = min(e0 + kPiece, L + dp);
    for (int eb = e0; eb < e1; eb += 32) {
      const int e = eb + lane;
      int a = 0;
      double wgt = 0.0;
      if (e < e1) {
        // an entry kept in the new list carries both terms at once:
        // (1-c)(1/d' - 1/d), zero when the degree did not change
        if (e < L) {
          a = oldl[e];
          wgt = contains_i(newl, dp, a) ? wb - wa : -wa;
        } else {
          a = newl[e - L];
          wgt = contains_i(oldl, L, a) ? 0.0 : wb;
        }
      }
      if (!OSP_GUARD(ctl, a >= 0 && a < d.nc, "multi offset target", c, e, a)) a = 0;
      const int cnt = min(32, e1 - eb);
      for (int j = 0; j < cnt; ++j) {
        const double wj = __shfl_sync(0xffffffffu, wgt, j);
        if (wj == 0.0) continue;  // warp-uniform
        const int aj = __shfl_sync(0xffffffffu, a, j);
        double* row = d.mu.xacc + (size_t)aj * Sp + lane * K;
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (ru[k] != 0.0) atomicAdd(row + k, wj * ru[k]);
        if (lane == 0) d.mark[aj] = epoch;
      }
    }
  }
}

// CPI start for every column: x(0) = c e_{s_j} in column j.
__global__ void k_multi_cpi_begin(Dev d) {
  const Multi& M = d.mu;
  const int j = threadIdx.x;
  if (j < M.S) {
    const int s = M.seeds[j];
    M.xacc[(size_t)s * M.Sp + j] = d.ctl->c;
    d.mark[s] = d.ctl->epoch;
  }
}

// Column col of R in caller order.
__global__ void k_gather_col(const double* __restrict__ r, int Sp, int col,
                             const int* __restrict__ ext2int, int n, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = r[(size_t)ext2int[i] * Sp + col];
}

// kBulk: short and medium in-lists stage whole source rows in shared memory
// by bulk asynchronous copies (dynamic shared memory RingCfg<TY, K>::kSmem);
// else each lane gathers its columns of up to eight rows into registers.
template <typename TY, int K, bool kBulk>
__global__ void __launch_bounds__(kPropThreads, 2) k_propagate_multi(Dev d, PropParams pp) {
  using A = typename AccOf<TY>::type;
  constexpr int Sp = 32 * K;
  __shared__ BarShared sh;
  __shared__ double s_part[kPropWarps * Sp];
  extern __shared__ __align__(128) unsigned char dsm[];
  Ctl* ctl = d.ctl;
  if (*(volatile int*)&ctl->status) return;
  Ring rg{};
  if constexpr (kBulk) {
    using C = RingCfg<TY, K>;
    const int w = threadIdx.x >> 5;
    rg.bar = smem_u32(dsm) + 16u * (unsigned)w;
    const int off = C::kBarBytes + w * 2 * C::kRows * C::kRowBytes;
    rg.rows = smem_u32(dsm) + (unsigned)off;
    rg.rows_g = dsm + off;
    if ((threadIdx.x & 31) == 0) {
      mbar_init(rg.bar, 1);
      mbar_init(rg.bar + 8u, 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  const Multi& M = d.mu;
  const int n = ctl->n;
  const long long m = ctl->m;
  const int epoch = ctl->epoch;
  const int n_hubs = ctl->n_hubs;
  const int n_pieces = ctl->n_pieces;
  const int n_tasks = ctl->n_tasks;
  const int hub_thr = ctl->hub_thr, hub_piece = ctl->hub_piece;
  TY* yb[2] = {(TY*)M.y0, (TY*)M.y1};
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) d.step_ns[0] = global_ns();

  // x(0): stamped rows from xacc into R and y(0); other rows of y(0) are zero
  {
    double l1[K];
#pragma unroll
    for (int k = 0; k < K; ++k) l1[k] = 0.0;
    for (int vb = gw * 32; vb < n; vb += nw * 32) {
     const int vl = vb + lane;
     const unsigned stamped = __ballot_sync(0xffffffffu, vl < n && __ldcg(d.mark + vl) == epoch);
     const int cnt = min(32, n - vb);
     for (int jj = 0; jj < cnt; ++jj) {
      const int v = vb + jj;
      const size_t base = (size_t)v * Sp + lane * K;
      alignas(16) TY yv[K];
      if ((stamped >> jj) & 1u) {
        alignas(16) double x[K], rr[K], z[K];
        load_cg(M.xacc + base, x);
        load_cg(M.r + base, rr);
        const A s = scale_of<A>(d, v);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          rr[k] += x[k];
          l1[k] += fabs(x[k]);
          yv[k] = from_acc((A)((A)x[k] * s), (TY*)nullptr);
          z[k] = 0.0;
        }
        store_k(M.r + base, rr);
        store_k(M.xacc + base, z);
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) yv[k] = from_acc((A)0, (TY*)nullptr);
      }
      store_k(yb[0] + base, yv);
     }
    }
    column_partials<K>(M, l1, s_part);
    if (bar_arrive(ctl, sh)) decide_multi<K>(d, pp, 0, m);
    if (!bar_release(ctl, sh)) return;
  }

  A* hub_acc = (A*)M.hub_acc;
  for (int it = 1;; ++it) {
    if (*(volatile int*)&ctl->stop) break;
    unsigned act = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) act |= (unsigned)(*(volatile int*)&M.active[lane * K + k] != 0) << k;
    const TY* ys = yb[(it - 1) & 1];
    TY* yd = yb[it & 1];
    double l1[K];
#pragma unroll
    for (int k = 0; k < K; ++k) l1[k] = 0.0;
    const int n_items = n_pieces + n_tasks;
    for (;;) {
      int t = 0;
      if (lane == 0) t = atomicAdd(&ctl->ctr[1], 1);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= n_items) break;
      if (t < n_pieces) {
        // a piece of a long in-list; the piece that completes the list finishes it
        int lo = 0, hi = n_hubs;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (__ldg(d.hub_pstart + mid) <= t) lo = mid;
          else hi = mid;
        }
        const int h = lo;
        const int v = __ldg(d.hubs + h);
        const int piece = t - __ldg(d.hub_pstart + h);
        const int full = __ldg(d.len_c + v);
        const int* p = d.pool_c + __ldg(d.off_c + v) + (unsigned)(piece * hub_piece);
        const int L = min(hub_piece, full - piece * hub_piece);
        A acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = (A)0;
        if constexpr (kBulk) ring_sum_list<TY, K, A>(rg, d, p, L, ys, acc);
        else sum_rows<TY, K, A>(p, L, ys, acc);
        A* ha = hub_acc + (size_t)h * Sp + lane * K;
#pragma unroll
        for (int k = 0; k < K; ++k) atomicAdd(ha + k, acc[k]);
        __threadfence();
        int last = 0;
        if (lane == 0) {
          const int np = (full + hub_piece - 1) / hub_piece;
          last = atomicAdd(&d.hub_cnt[h], 1) == np - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
          __threadfence();
#pragma unroll
          for (int k = 0; k < K; ++k) {
            acc[k] = __ldcg(ha + k);
            ha[k] = (A)0;
          }
          if (lane == 0) d.hub_cnt[h] = 0;
          alignas(16) double rr[K];
          load_cg(M.r + (size_t)v * Sp + lane * K, rr);
          finish_row<TY, K, A>(d, v, acc, scale_of<A>(d, v), rr, act, yd, l1);
        }
        continue;
      }
      const int task = t - n_pieces;
      const int c0 = __ldg(d.task_first + task), c1 = __ldg(d.task_first + task + 1);
      for (int vb = c0; vb < c1; vb += 32) {
        // offsets and lengths of up to 32 consecutive nodes in one coalesced load
        const int vl = vb + lane;
        int my_len = 0;
        unsigned my_off = 0;
        if (vl < c1) {
          my_len = __ldg(d.len_c + vl);
          my_off = __ldg(d.off_c + vl);
        }
        const int cnt = min(32, c1 - vb);
        // empty in-lists: x(i)[v] = 0, R unchanged, the next gather row is zero
        unsigned empty = __ballot_sync(0xffffffffu, lane < cnt && my_len == 0);
        while (empty) {
          const int jj = __ffs(empty) - 1;
          empty &= empty - 1;
          alignas(16) TY z[K];
#pragma unroll
          for (int k = 0; k < K; ++k) z[k] = from_acc((A)0, (TY*)nullptr);
          store_k(yd + (size_t)(vb + jj) * Sp + lane * K, z);
        }
        // the others (hubs excepted) in order, two deep: the first 32 in-list ids
        // and the row of R of the next node load while the current one is summed
        unsigned todo = __ballot_sync(0xffffffffu, lane < cnt && my_len > 0 && my_len <= hub_thr);
        if (!todo) continue;
        if constexpr (kBulk) {
          // batches of up to kRows rows of one in-list, nodes in order: the next
          // batch's copies and the ids of the one after are in flight while a
          // batch is summed; a node's row of R loads with its first batch
          constexpr int G = RingCfg<TY, K>::kRows;
          int pj = 0, plen = 0, ps = 0;
          unsigned poff = 0;
          auto next = [&](RowBatch& o) -> bool {
            if (ps >= plen) {
              if (!todo) return false;
              pj = __ffs(todo) - 1;
              todo &= todo - 1;
              plen = __shfl_sync(0xffffffffu, my_len, pj);
              poff = __shfl_sync(0xffffffffu, my_off, pj);
              ps = 0;
            }
            o.jc = pj;
            o.off = poff;
            o.s = ps;
            o.cnt = min(G, plen - ps);
            o.first = ps == 0;
            o.last = ps + G >= plen;
            ps += G;
            return true;
          };
          auto ids_of = [&](const RowBatch& o) -> int {
            int u = lane < o.cnt ? __ldg(d.pool_c + o.off + (unsigned)(o.s + lane)) : 0;
            if (lane < o.cnt && !OSP_GUARD(ctl, u >= 0 && u < d.nc, "multi staged id", o.jc, o.s, u))
              u = 0;
            return u;
          };
          RowBatch c0, c1, c2;
          next(c0);
          ring_issue<TY, K>(rg, rg.buf, c0.cnt, ids_of(c0), ys);
          alignas(16) double rr_n[K];
          load_cg(M.r + (size_t)(vb + c0.jc) * Sp + lane * K, rr_n);
          A s_n = scale_of<A>(d, vb + c0.jc);
          bool h1 = next(c1);
          int u1 = h1 ? ids_of(c1) : 0;
          alignas(16) double rr[K];
          A s = (A)0;
          A acc[K];
#pragma unroll
          for (int k = 0; k < K; ++k) acc[k] = (A)0;
          for (;;) {
            if (c0.first) {
#pragma unroll
              for (int k = 0; k < K; ++k) {
                rr[k] = rr_n[k];
                acc[k] = (A)0;
              }
              s = s_n;
            }
            const int b = rg.buf;
            if (h1) {
              ring_issue<TY, K>(rg, b ^ 1, c1.cnt, u1, ys);
              if (c1.first) {
                load_cg(M.r + (size_t)(vb + c1.jc) * Sp + lane * K, rr_n);
                s_n = scale_of<A>(d, vb + c1.jc);
              }
            }
            const bool h2 = h1 && next(c2);
            const int u2 = h2 ? ids_of(c2) : 0;
            ring_wait(rg, b, ctl);
            ring_sum<TY, K, A>(rg, b, c0.cnt, acc);
            if (c0.last) finish_row<TY, K, A>(d, vb + c0.jc, acc, s, rr, act, yd, l1);
            if (!h1) break;
            rg.buf = b ^ 1;
            c0 = c1;
            c1 = c2;
            h1 = h2;
            u1 = u2;
          }
          continue;
        }
        int jn = __ffs(todo) - 1;
        todo &= todo - 1;
        int len_n = __shfl_sync(0xffffffffu, my_len, jn);
        unsigned off_n = __shfl_sync(0xffffffffu, my_off, jn);
        int idx_n = lane < len_n ? __ldg(d.pool_c + off_n + lane) : 0;
        alignas(16) double rr_n[K];
        load_cg(M.r + (size_t)(vb + jn) * Sp + lane * K, rr_n);
        for (;;) {
          const int jc = jn, len = len_n;
          const unsigned off = off_n;
          const int idx = idx_n;
          alignas(16) double rr[K];
#pragma unroll
          for (int k = 0; k < K; ++k) rr[k] = rr_n[k];
          const bool more = todo != 0;
          if (more) {
            jn = __ffs(todo) - 1;
            todo &= todo - 1;
            len_n = __shfl_sync(0xffffffffu, my_len, jn);
            off_n = __shfl_sync(0xffffffffu, my_off, jn);
            idx_n = lane < len_n ? __ldg(d.pool_c + off_n + lane) : 0;
            load_cg(M.r + (size_t)(vb + jn) * Sp + lane * K, rr_n);
          }
          const int v = vb + jc;
          const A s = scale_of<A>(d, v);
          A acc[K];
#pragma unroll
          for (int k = 0; k < K; ++k) acc[k] = (A)0;
          sum_rows<TY, K, A>(d.pool_c + off, len, ys, acc, idx);
          finish_row<TY, K, A>(d, v, acc, s, rr, act, yd, l1);
          if (!more) break;
        }
      }
    }
    column_partials<K>(M, l1, s_part);
    if (bar_arrive(ctl, sh)) decide_multi<K>(d, pp, it, m);
    if (!bar_release(ctl, sh)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->epoch = epoch + 1;
}

namespace {

struct MultiFn {
  const void* fn;
  int smem;  // dynamic shared memory bytes
};

template <typename TY, int K>
MultiFn multi_fn_k(bool bulk) {
  if (bulk) return {(const void*)k_propagate_multi<TY, K, true>, RingCfg<TY, K>::kSmem};
  return {(const void*)k_propagate_multi<TY, K, false>, 0};
}

template <typename TY>
MultiFn multi_fn(int K, bool bulk) {
  switch (K) {
    case 1: return multi_fn_k<TY, 1>(bulk);
    case 2: return multi_fn_k<TY, 2>(bulk);
    case 4: return multi_fn_k<TY, 4>(bulk);
    default: return multi_fn_k<TY, 8>(bulk);
  }
}

MultiFn pick_multi(int precision, int K, bool bulk) {
  if (precision == OSP_PREC_FP64) return multi_fn<double>(K, bulk);
  if (precision == OSP_PREC_FP32_ACC64) return multi_fn<float>(K, bulk);
  return multi_fn<__nv_bfloat16>(K, bulk);
}

}  // namespace

int propagate_multi_grid(int precision, int K, int num_sms, bool bulk) {
  const MultiFn f = pick_multi(precision, K, bulk);
  if (f.smem > 0 &&
      cudaFuncSetAttribute(f.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, f.smem) != cudaSuccess)
    return 0;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, f.fn, kPropThreads, f.smem) != cudaSuccess ||
      bps <= 0)
    return 0;
  bps = bps > 4 ? 4 : bps;
  const int g = bps * num_sms;
  return g > kMaxGrid ? kMaxGrid : g;
}

cudaError_t launch_propagate_multi(const Dev& d, const PropParams& pp, int precision, int grid,
                                   bool bulk, cudaStream_t s) {
  Dev dd = d;
  PropParams p = pp;
  void* args[] = {&dd, &p};
  const MultiFn f = pick_multi(precision, d.mu.K, bulk);
  return cudaLaunchCooperativeKernel(f.fn, dim3(grid), dim3(kPropThreads), args, (size_t)f.smem, s);
}

// ---------------------------------------------------------------------------
// Failure-detection self-tests: the bounded waits of the persistent kernels
// are made to run out on purpose (a CTA that never arrives; an mbarrier whose
// announced bytes never all land), and the status word must report it.
// ---------------------------------------------------------------------------
__global__ void k_selftest_barrier(Ctl* ctl, int lose) {
  __shared__ BarShared sh;
  if (lose && blockIdx.x == 0) return;  // this CTA never arrives
  if (bar_arrive(ctl, sh) && threadIdx.x == 0) ctl->iter = 1;
  bar_release(ctl, sh);
}

__global__ void k_selftest_stage(Ctl* ctl, const float* src, int lose) {
  using C = RingCfg<float, 1>;
  extern __shared__ __align__(128) unsigned char dsm[];
  Ring rg{};
  rg.bar = smem_u32(dsm);
  rg.rows = smem_u32(dsm) + C::kBarBytes;
  rg.rows_g = dsm + C::kBarBytes;
  if (threadIdx.x == 0) {
    mbar_init(rg.bar, 1);
    mbar_init(rg.bar + 8u, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // two rows announced; with `lose` only the first is copied
    mbar_arrive_expect(rg.bar, 2u * C::kRowBytes);
    bulk_copy_row(rg.rows, src, C::kRowBytes, rg.bar);
    if (!lose) bulk_copy_row(rg.rows + C::kRowBytes, src + 32, C::kRowBytes, rg.bar);
  }
  __syncwarp();
  ring_wait(rg, 0, ctl);
  if (threadIdx.x == 0 && *(volatile int*)&ctl->status == 0) {
    const float* r = reinterpret_cast<const float*>(rg.rows_g);
    ctl->iter = (r[0] == src[0] && r[63] == src[63]) ? 1 : 2;  // both rows arrived intact
  }
}

cudaError_t launch_selftest(Ctl* ctl, const float* src, int which, int lose, cudaStream_t s) {
  if (which == 0) {
    k_selftest_barrier<<<4, 64, 0, s>>>(ctl, lose);
  } else {
    k_selftest_stage<<<1, 32, RingCfg<float, 1>::kBarBytes + 2 * RingCfg<float, 1>::kRowBytes, s>>>(
        ctl, src, lose);
  }
  return cudaGetLastError();
}

cudaError_t launch_offset_multi(const Dev& d, int grid, cudaStream_t s) {
  switch (d.mu.K) {
    case 1: k_offset_multi<1><<<grid, 256, 0, s>>>(d); break;
    case 2: k_offset_multi<2><<<grid, 256, 0, s>>>(d); break;
    case 4: k_offset_multi<4><<<grid, 256, 0, s>>>(d); break;
    default: k_offset_multi<8><<<grid, 256, 0, s>>>(d); break;
  }
  return cudaGetLastError();
}

}  // namespace osp

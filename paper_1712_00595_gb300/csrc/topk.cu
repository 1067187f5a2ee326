// Top-k query (ranking by score descending, then id ascending).
//
// Radix select over order-preserving 64-bit keys of the scores: each pass
// histograms the next digit of the keys that still match the selected prefix
// and keeps the digit holding the k-th largest key, until the remaining bin is
// small enough to sort. The survivors (keys at or above the prefix) are then
// sorted in one CTA by (key descending, id ascending).
#include "common.cuh"
#include "kernels.h"

namespace osp {

namespace {
constexpr int kDigitBits = 12;
constexpr int kBins = 1 << kDigitBits;

__device__ __forceinline__ unsigned long long order_key(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
}  // namespace

__global__ void k_topk_reset(TopkState* st, unsigned* hist, int k) {
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) {
    st->prefix = 0;
    st->bits = 0;
    st->k_rem = k;
    st->done = 0;
    st->count = 0;
  }
}

__global__ void __launch_bounds__(256) k_topk_hist(const double* __restrict__ r, int n,
                                                   const TopkState* __restrict__ st,
                                                   unsigned* hist, int width) {
  __shared__ unsigned sh[kBins];
  if (st->done) return;
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int bits = st->bits;
  const unsigned long long prefix = st->prefix;
  const int shift = 64 - bits - width;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long key = order_key(r[i]);
    if (bits == 0 || (key >> (64 - bits)) == prefix)
      atomicAdd(&sh[(key >> shift) & ((1ull << width) - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << width); i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// One CTA: pick the digit that holds the k_rem-th largest key, extend the prefix.
__global__ void __launch_bounds__(1024) k_topk_select(TopkState* st, unsigned* hist, int width,
                                                      int cand_max) {
  __shared__ unsigned s_cnt[kBins];
  if (st->done) return;
  const int nb = 1 << width;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s_cnt[i] = hist[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int k_rem = st->k_rem;
    long long above = 0;
    int d = nb - 1;
    for (; d >= 0; --d) {
      if (above + s_cnt[d] >= k_rem) break;
      above += s_cnt[d];
    }
    if (d < 0) d = 0;  // fewer than k_rem keys match: keep everything
    st->k_rem = k_rem - (int)above;
    st->prefix = (st->prefix << width) | (unsigned long long)d;
    st->bits += width;
    if ((int)s_cnt[d] <= cand_max || st->bits >= 64) st->done = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
}

constexpr int kChunk = 4096;  // elements per CTA in the ordered compaction (1024 threads x 4)

__device__ __forceinline__ void bin_range(const TopkState* st, unsigned long long* lo,
                                          unsigned long long* hi) {
  const int bits = st->bits;
  if (bits == 0) {
    *lo = 0ull;
    *hi = ~0ull;
  } else {
    *lo = st->prefix << (64 - bits);
    *hi = bits >= 64 ? *lo : (*lo | ((1ull << (64 - bits)) - 1));
  }
}

// Per chunk: how many keys lie above the selected bin and how many inside it.
__global__ void __launch_bounds__(1024) k_topk_count(const double* __restrict__ r, int n,
                                                     const TopkState* __restrict__ st,
                                                     int* blk_above, int* blk_bin) {
  __shared__ int s_a, s_b;
  unsigned long long lo, hi;
  bin_range(st, &lo, &hi);
  if (threadIdx.x == 0) s_a = s_b = 0;
  __syncthreads();
  int a = 0, b = 0;
  const int base = blockIdx.x * kChunk;
  for (int j = threadIdx.x; j < kChunk; j += blockDim.x) {
    const int i = base + j;
    if (i >= n) break;
    const unsigned long long key = order_key(r[i]);
    a += key > hi;
    b += key >= lo && key <= hi;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_a, a);
    atomicAdd(&s_b, b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    blk_above[blockIdx.x] = s_a;
    blk_bin[blockIdx.x] = s_b;
  }
}

// One CTA: exclusive scans of the chunk counts; how many bin keys to keep.
__global__ void __launch_bounds__(1024) k_topk_scan(TopkState* st, int* blk_above, int* blk_bin,
                                                    int nb, int cand_max) {
  if (threadIdx.x != 0) return;
  int a = 0, b = 0;
  for (int i = 0; i < nb; ++i) {
    const int ta = blk_above[i], tb = blk_bin[i];
    blk_above[i] = a;
    blk_bin[i] = b;
    a += ta;
    b += tb;
  }
  st->above = a;
  st->bin_count = b;
  // the whole bin when it is small; otherwise it is one key value and ties go by id
  st->keep = b <= cand_max ? b : min(b, st->k_rem);
  st->count = a + st->keep;
}

// Ordered compaction: chunk by chunk in id order, keys above the bin go first,
// then the first `keep` keys of the bin.
__global__ void __launch_bounds__(1024) k_topk_emit(const double* __restrict__ r, int n,
                                                    const TopkState* __restrict__ st,
                                                    const int* __restrict__ blk_above,
                                                    const int* __restrict__ blk_bin,
                                                    unsigned long long* keys, int* ids) {
  __shared__ int s_w[2][32];
  __shared__ int s_run[2];
  unsigned long long lo, hi;
  bin_range(st, &lo, &hi);
  const int above_total = st->above, keep = st->keep;
  int ra = blk_above[blockIdx.x], rb = blk_bin[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int base = blockIdx.x * kChunk;
  for (int round = 0; round < kChunk / 1024; ++round) {
    const int i = base + round * 1024 + threadIdx.x;
    unsigned long long key = 0;
    int fa = 0, fb = 0;
    if (i < n) {
      key = order_key(r[i]);
      fa = key > hi;
      fb = key >= lo && key <= hi;
    }
    const unsigned ba = __ballot_sync(0xffffffffu, fa), bb = __ballot_sync(0xffffffffu, fb);
    if (lane == 0) {
      s_w[0][w] = __popc(ba);
      s_w[1][w] = __popc(bb);
    }
    __syncthreads();
    int pa = 0, pb = 0;
    for (int q = 0; q < w; ++q) {
      pa += s_w[0][q];
      pb += s_w[1][q];
    }
    pa += __popc(ba & lanemask_lt());
    pb += __popc(bb & lanemask_lt());
    if (fa) {
      keys[ra + pa] = key;
      ids[ra + pa] = i;
    }
    if (fb && rb + pb < keep) {
      keys[above_total + rb + pb] = key;
      ids[above_total + rb + pb] = i;
    }
    if (threadIdx.x == 0) {
      int ta = 0, tb = 0;
      for (int q = 0; q < 32; ++q) {
        ta += s_w[0][q];
        tb += s_w[1][q];
      }
      s_run[0] = ta;
      s_run[1] = tb;
    }
    __syncthreads();
    ra += s_run[0];
    rb += s_run[1];
    __syncthreads();
  }
}

// One CTA: bitonic sort of the survivors by (key desc, id asc); write the first k.
__global__ void __launch_bounds__(1024) k_topk_sort(const double* __restrict__ r,
                                                    const TopkState* __restrict__ st,
                                                    const unsigned long long* keys,
                                                    const int* ids, int cap, int k,
                                                    const double* __restrict__ norm,
                                                    int* out_ids, double* out_scores,
                                                    int* out_k) {
  extern __shared__ unsigned char smem[];
  const int cnt = min(st->count, cap);  // count <= k + cand_max <= cap by construction
  int N = 2;
  while (N < cnt) N <<= 1;
  unsigned long long* sk = (unsigned long long*)smem;
  int* si = (int*)(sk + N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sk[i] = i < cnt ? keys[i] : 0ull;
    si[i] = i < cnt ? ids[i] : 0x7FFFFFFF;
  }
  __syncthreads();
  // "a before b": larger key, then smaller id
  for (int kk = 2; kk <= N; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (N >> 1); t += blockDim.x) {
        const int a = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int b = a | j;
        const bool first = (a & kk) == 0;
        const bool b_before_a = sk[b] > sk[a] || (sk[b] == sk[a] && si[b] < si[a]);
        if (b_before_a == first) {
          const unsigned long long tk = sk[a];
          sk[a] = sk[b];
          sk[b] = tk;
          const int ti = si[a];
          si[a] = si[b];
          si[b] = ti;
        }
      }
      __syncthreads();
    }
  }
  const int kk = min(k, cnt);
  const double s = norm ? *norm : 1.0;
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {
    out_ids[i] = si[i];
    out_scores[i] = norm ? (s > 0.0 ? r[si[i]] / s : 0.0) : r[si[i]];
  }
  if (threadIdx.x == 0) *out_k = kk;
}

}  // namespace osp

// Top-k query (ranking by score descending, then id ascending).
//
// Radix select over order-preserving 64-bit keys of the scores: each pass
// histograms the next digit of the keys that still match the selected prefix
// and keeps the digit holding the k-th largest key, until the remaining bin is
// small enough to sort, or holds a single key value. The survivors (keys at or
// above the prefix) are then sorted in one CTA by (key descending, id
// ascending).
//
// Every kernel serves a table of independent jobs (one score vector and its
// scratch each): blockIdx.y is the job, so the top-k of many seeds costs one
// launch sequence.
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
}  // namespace

__global__ void k_topk_reset(TopkJobs J) {
  const TopkJob& jb = J.j[blockIdx.y];
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) jb.hist[i] = 0;
  if (threadIdx.x == 0) {
    TopkState* st = jb.st;
    st->prefix = 0;
    st->bits = 0;
    st->k_rem = J.k;
    st->done = 0;
    st->count = 0;
    st->kmin = ~0ull;
    st->kmax = 0ull;
  }
}

// Histogram of the next digit over the keys that match the prefix; also the
// smallest and largest such key, so that a prefix holding one key value (ties,
// typically of zero scores) ends the selection at once.
__global__ void __launch_bounds__(256) k_topk_hist(TopkJobs J, int width) {
  __shared__ unsigned sh[kBins];
  const TopkJob& jb = J.j[blockIdx.y];
  TopkState* st = jb.st;
  if (st->done) return;
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const double* __restrict__ r = jb.src;
  const int n = J.n;
  const int bits = st->bits;
  const unsigned long long prefix = st->prefix;
  const int shift = 64 - bits - width;
  unsigned long long kmin = ~0ull, kmax = 0ull;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long key = order_key(r[i]);
    if (bits == 0 || (key >> (64 - bits)) == prefix) {
      atomicAdd(&sh[(key >> shift) & ((1ull << width) - 1)], 1u);
      kmin = key < kmin ? key : kmin;
      kmax = key > kmax ? key : kmax;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, o);
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, o);
    kmin = a < kmin ? a : kmin;
    kmax = b > kmax ? b : kmax;
  }
  if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
    atomicMin(&st->kmin, kmin);
    atomicMax(&st->kmax, kmax);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << width); i += blockDim.x)
    if (sh[i]) atomicAdd(&jb.hist[i], sh[i]);
}

// One CTA of 1024 threads per job: pick the digit d that holds the k_rem-th
// largest key (the largest d whose bins d.. hold at least k_rem keys; suffix
// sums by a CTA scan), extend the prefix.
__global__ void __launch_bounds__(1024) k_topk_select(TopkJobs J, int width, int cand_max) {
  __shared__ unsigned s_cnt[kBins];
  __shared__ long long s_w[32];
  __shared__ int s_d;
  __shared__ long long s_above;
  const TopkJob& jb = J.j[blockIdx.y];
  TopkState* st = jb.st;
  if (st->done) return;
  unsigned* hist = jb.hist;
  const int nb = 1 << width;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int i = t; i < nb; i += blockDim.x) s_cnt[i] = hist[i];
  if (t == 0) {
    s_d = -1;
    s_above = 0;
  }
  __syncthreads();
  const int k_rem = st->k_rem;
  // thread t owns the bins [b0, b1) counted from the top: bin nb-1-q for q in [b0, b1)
  const int per = (nb + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
  long long mine = 0;
  for (int q = b0; q < b1; ++q) mine += s_cnt[nb - 1 - q];
  long long inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = (int)blockDim.x >> 5;
    long long x = lane < nw ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_w[lane] = x;
  }
  __syncthreads();
  long long above = (w ? s_w[w - 1] : 0) + inc - mine;  // keys in the bins above b0
  for (int q = b0; q < b1; ++q) {
    const int d = nb - 1 - q;
    if (above < k_rem && above + s_cnt[d] >= k_rem) {
      s_d = d;
      s_above = above;
    }
    above += s_cnt[d];
  }
  __syncthreads();
  if (t == 0) {
    int d = s_d;
    long long ab = s_above;
    if (d < 0) {  // fewer than k_rem keys match: keep everything
      d = 0;
      ab = 0;
      for (int i = 0; i < nb; ++i) ab += s_cnt[i];
    }
    st->k_rem = k_rem - (int)ab;
    st->prefix = (st->prefix << width) | (unsigned long long)d;
    st->bits += width;
    // one key value left under the prefix (the last pass saw a single value)
    const bool one = st->kmin == st->kmax;
    if ((int)s_cnt[d] <= cand_max || st->bits >= 64 || one) st->done = 1;
    st->kmin = ~0ull;
    st->kmax = 0ull;
  }
  __syncthreads();
  for (int i = t; i < nb; i += blockDim.x) hist[i] = 0;
}

// Per chunk of kTopkChunk ids: how many keys lie above the selected bin and
// how many inside it.
__global__ void __launch_bounds__(1024) k_topk_count(TopkJobs J) {
  __shared__ int s_a, s_b;
  const TopkJob& jb = J.j[blockIdx.y];
  const double* __restrict__ r = jb.src;
  const int n = J.n;
  unsigned long long lo, hi;
  bin_range(jb.st, &lo, &hi);
  if (threadIdx.x == 0) s_a = s_b = 0;
  __syncthreads();
  int a = 0, b = 0;
  const int base = blockIdx.x * kTopkChunk;
  for (int j = threadIdx.x; j < kTopkChunk; j += blockDim.x) {
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
    jb.blk_a[blockIdx.x] = s_a;
    jb.blk_b[blockIdx.x] = s_b;
  }
}

// One CTA per job (any multiple of 32 threads): exclusive scans of the chunk
// counts; how many bin keys to keep. Thread t scans a run of consecutive
// chunks, the runs' totals are scanned across the CTA.
__global__ void __launch_bounds__(1024) k_topk_scan(TopkJobs J, int nb, int cand_max) {
  __shared__ int s_a[32], s_b[32];
  const TopkJob& jb = J.j[blockIdx.y];
  int* blk_above = jb.blk_a;
  int* blk_bin = jb.blk_b;
  const int nt = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int per = (nb + nt - 1) / nt;
  const int lo = min(nb, t * per), hi = min(nb, lo + per);
  int a = 0, b = 0;
  for (int i = lo; i < hi; ++i) {
    a += blk_above[i];
    b += blk_bin[i];
  }
  int ia = a, ib = b;  // inclusive scans over the warp, then over the warps
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += ya;
      ib += yb;
    }
  }
  if (lane == 31) {
    s_a[w] = ia;
    s_b[w] = ib;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = nt >> 5;
    int xa = lane < nw ? s_a[lane] : 0, xb = lane < nw ? s_b[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
      if (lane >= o) {
        xa += ya;
        xb += yb;
      }
    }
    s_a[lane] = xa;
    s_b[lane] = xb;
  }
  __syncthreads();
  int ra = (w ? s_a[w - 1] : 0) + ia - a, rb = (w ? s_b[w - 1] : 0) + ib - b;
  for (int i = lo; i < hi; ++i) {
    const int ta = blk_above[i], tb = blk_bin[i];
    blk_above[i] = ra;
    blk_bin[i] = rb;
    ra += ta;
    rb += tb;
  }
  if (t == nt - 1) {
    TopkState* st = jb.st;
    const int A = s_a[(nt >> 5) - 1], B = s_b[(nt >> 5) - 1];
    st->above = A;
    st->bin_count = B;
    // the whole bin when it is small; otherwise it is one key value and ties go by id
    st->keep = B <= cand_max ? B : min(B, st->k_rem);
    st->count = A + st->keep;
  }
}

// Ordered compaction: chunk by chunk in id order, keys above the bin go first,
// then the first `keep` keys of the bin.
__global__ void __launch_bounds__(1024) k_topk_emit(TopkJobs J) {
  __shared__ int s_w[2][32];
  __shared__ int s_run[2];
  const TopkJob& jb = J.j[blockIdx.y];
  const double* __restrict__ r = jb.src;
  const int n = J.n;
  const TopkState* st = jb.st;
  unsigned long long lo, hi;
  bin_range(st, &lo, &hi);
  const int above_total = st->above, keep = st->keep;
  int ra = jb.blk_a[blockIdx.x], rb = jb.blk_b[blockIdx.x];
  unsigned long long* keys = jb.keys;
  int* ids = jb.ids;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int base = blockIdx.x * kTopkChunk;
  for (int round = 0; round < kTopkChunk / 1024; ++round) {
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

// One CTA per job: bitonic sort of the survivors by (key desc, id asc) over
// the next power of two above their count; write the first k (to device or
// host-mapped memory).
__global__ void __launch_bounds__(1024) k_topk_sort(TopkJobs J, int cap) {
  extern __shared__ unsigned char smem[];
  const TopkJob& jb = J.j[blockIdx.y];
  const int cnt = min(jb.st->count, cap);  // count <= k + cand_max <= cap by construction
  int N = 2;
  while (N < cnt) N <<= 1;
  unsigned long long* sk = (unsigned long long*)smem;
  int* si = (int*)(sk + N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sk[i] = i < cnt ? jb.keys[i] : 0ull;
    si[i] = i < cnt ? jb.ids[i] : 0x7FFFFFFF;
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
  const int kk = min(J.k, cnt);
  const double* norm = jb.norm;
  const double s = norm ? *norm : 1.0;
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {
    const double v = jb.src[si[i]];
    jb.out_ids[i] = si[i];
    jb.out_sc[i] = norm ? (s > 0.0 ? v / s : 0.0) : v;
  }
  if (threadIdx.x == 0) *jb.out_k = kk;
}

// Seed-block columns in caller order: dst_j[x] = r[ext2int[x] Sp + col_j],
// walked in internal order (rows in address order; the scattered writes land
// in L2).
__global__ void k_gather_cols(const double* __restrict__ r, int Sp, const int* __restrict__ int2ext,
                              int n, GatherJobs G) {
  const int col = G.col[blockIdx.y];
  double* dst = G.dst[blockIdx.y];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    dst[int2ext[v]] = r[(size_t)v * Sp + col];
}

int enqueue_topk_select(const TopkJobs& J, int num_sms, cudaStream_t st) {
  const int m = J.m;
  k_topk_reset<<<dim3(1, m), 1024, 0, st>>>(J);
  const int widths[6] = {12, 12, 12, 12, 12, 4};
  for (int w : widths) {
    k_topk_hist<<<dim3(num_sms * 4, m), 256, 0, st>>>(J, w);
    k_topk_select<<<dim3(1, m), 1024, 0, st>>>(J, w, kTopkCand);
  }
  const int nb = (J.n + kTopkChunk - 1) / kTopkChunk;
  k_topk_count<<<dim3(nb, m), 1024, 0, st>>>(J);
  k_topk_scan<<<dim3(1, m), 1024, 0, st>>>(J, nb, kTopkCand);
  k_topk_emit<<<dim3(nb, m), 1024, 0, st>>>(J);
  return 16;
}

int enqueue_topk_sort(const TopkJobs& J, cudaStream_t st) {
  k_topk_sort<<<dim3(1, J.m), 1024, kTopkSortSmem, st>>>(J, kTopkMaxK + kTopkCand);
  return 1;
}

}  // namespace osp

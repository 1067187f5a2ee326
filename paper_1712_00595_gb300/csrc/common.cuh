// Device-side layout and helpers shared by the engine's translation units.
//
// Graph store. Each direction (out-edges = CSR rows for push, in-edges = CSC
// columns for pull) is a "slotted" adjacency: per node an offset into an int32
// pool and a length; the pool holds every list contiguously and ascending.
// A batch never edits a list in place: a changed list is written to fresh pool
// space (bump allocation) and its slot is repointed, so the old list stays
// readable while the offset vector is formed. Stale space is reclaimed by a
// compaction pass when the pool runs low.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#include "../../include/osp.h"

namespace osp {

constexpr int kMaxBatch = 16384;        // ops per sub-batch (keys pack the op index in 14 bits)
constexpr long long kMaxLargeBatch = 1ll << 22;  // ops per apply call, in sub-batches of kMaxBatch
constexpr int kMaxNodes = (1 << 25) - 1; // ids fit in 25 bits
constexpr int kNoPos = 0x7F7F7F7F;       // del_pos of a node not deleted by the batch (memset 0x7F)
constexpr int kLight = 32;               // lists up to this length are walked by one lane
constexpr int kPiece = 256;              // old entries per warp task in the list merge
constexpr int kMaxHist = 4096;           // per-step ||x||_1 history entries
constexpr int kAbsParts = 1024;  // CTAs of the L1-norm reduction (per-CTA partials, summed in order)
constexpr int kMaxGrid = 4096;           // CTAs of the persistent kernel (partials array size)
constexpr int kPropThreads = 256;
constexpr int kPropWarps = kPropThreads / 32;
constexpr int kHubThreshold = 1024;  // pull step: in-lists longer than this are summed in pieces
constexpr int kHubPiece = 1024;      // pull step: edges per hub piece
constexpr int kMultiHub = 256;       // seed block: in-lists longer than this, in pieces of this size
constexpr int kMultiNodeItems = 4;   // seed block: task items per node (a node's score row costs more)
constexpr int kTaskItems = 1024;     // pull step: default items (edges + nodes) per warp task
constexpr int kMinTaskItems = 256;   // smallest task size a schedule may choose (sizes the plan)
constexpr double kPushAlpha = 14.0;  // push step while frontier out-edges <= m / alpha
constexpr double kPushBeta = 24.0;   // ... and frontier size <= n / beta

enum StepMode : int { kPush = 0, kPull = 1 };

// Device control block: counters, sizes, barrier words and statistics.
struct Ctl {
  int status;    // 0 or a negative osp_status
  int bad_op;    // first invalid op of the batch
  int n;         // node ids in use
  int n_old;     // before the current batch
  long long m;   // live edges
  long long m_delta;
  unsigned long long pool_top_r, pool_top_c;
  unsigned long long pool_cap_r, pool_cap_c;
  long long net_ins, net_del;  // edge edits of the batch (node deletions not included)
  int n_rec_r, n_rec_c;        // changed row / column records
  int n_del;                   // nodes deleted by the batch
  int n_clr;                   // rows zeroed by the last ingested batch (clr_nodes)
  int n_hubs, n_pieces;        // pull step: long in-lists and their pieces
  int n_tasks;                 // pull step: warp tasks
  int n_mpieces;               // merge pieces of the current batch
  int dense0;                  // 1: x(0) is found by a dense scan of xacc (no queue from the merge)
  int n_opieces;               // several seeds: offset items (256 entries of a changed row)
  int hub_thr, hub_piece;      // pull step: in-lists longer than hub_thr go in pieces of hub_piece
  int batch_U;                 // ops of the batch, for a k_ingest replayed from a CUDA graph
  long long n_dst_nz, n_src_nz;  // nodes with a nonempty in-list / out-list (pull plan)
  int epoch;                   // frontier mark of x(0); step i uses epoch + i
  int q_size[2];               // frontier queue lengths
  unsigned int bar_count, bar_gen;
  int ctr[4];                  // dynamic work counters, reset at every barrier
  int iter, mode, push_iters, stop, pull_used, noconv;
  long long visited;
  long long ef;                // out-edges of the current frontier
  long long push_f, push_r;    // sums of |F(i-1)| and |F(i)| over push steps
  int seed;
  int multi;                   // 1: several seeds (the Multi block of Dev), 0: one seed
  int n_grp;                   // several seeds: column groups with a running column ...
  int grp[8];                  // ... and their indices, for the next pull step
  int narrow;                  // bf16 seed block: the next step runs on 4-column rows (see multi.cu)
  double c;
};

constexpr int kMaxSeeds = 256;

// Several seeds tracked together: column j of each n x Sp block belongs to
// the seed placed in column j (Sp = 32 K, K in {1, 2, 4, 8}; columns S .. Sp-1
// stay zero). R and the offset accumulator are [node][Sp]. The propagation
// kernel works on column groups of G = 32 KG columns (KG divides K; lane l
// owns columns [KG l, KG l + KG) of a group) and lays its gather blocks out
// group-major, [group][node][G].
struct Multi {
  int S, Sp, K;
  int KG;              // columns per lane in a column group of the batch kernel
  int KG_init;         // ... of the initial CPI (float rows when batches use bf16)
  int pack;            // 1: bf16 32-column groups take their columns through slot_col (set per launch)
  int* slot_col;       // [Sp] packed groups: column held by group slot q (chosen at each x(0))
  int* col_slot;       // [Sp] its inverse
  int* seeds;          // [S] internal ids, by column
  double* r;           // [nc Sp] scores (unnormalised r_temp)
  double* xacc;        // [nc Sp] offset accumulator
  void* y0; void* y1;  // [nc Sp] gather blocks (double, float or bf16), group-major
  void* e;             // [nc Sp] bf16 rounding residuals of the gather block (bf16 only)
  void* yn0; void* yn1;  // [nc 4] bf16 narrow gather rows: group slots 0..3 (packed bf16 blocks)
  double* part;        // [kMaxGrid Sp] per-CTA |x| partials
  int* active;         // [Sp] 1 while the column still propagates
  int* touched;        // [Sp] 1: the column has a nonzero offset entry in this call
  int* col_iters;      // [Sp] steps run per column
  double* col_q;       // [Sp] ||x(0)||_1 per column
  double* col_last;    // [Sp] ||x(k)||_1 at the column's stop
  double* res_bound;   // [Sp] bound on ||rho||_1 of the stored column (see osp_get_residual_bounds)
  int* force;          // [Sp] > 0: the column runs exactly that many steps
  void* hub_acc;       // [hubs Sp] (float or double) partial sums of long in-lists
  int* hub_cnt;        // [hubs 8] pieces done per long in-list and column group
};

// Every device pointer of one engine, passed to kernels by value.
struct Dev {
  int nc;  // node capacity
  // Nodes are stored in an internal order (by default: descending out-degree
  // of the loaded graph, so the gather vector of the most-read sources is
  // dense in memory); the C ABI speaks the caller's ids.
  int* ext2int;  // [nc] caller id -> internal id (identity above the loaded ids)
  int* int2ext;  // [nc] internal id -> caller id
  int grid_prop;
  // graph store
  unsigned* off_r; int* len_r; int* pool_r;
  unsigned* off_c; int* len_c; int* pool_c;
  // per node
  double* r;
  void* y0; void* y1;  // gather vectors y = (1-c) x / d (float or double)
  double* xacc;        // push / offset accumulator
  unsigned long long* xfix;  // deterministic mode: offset accumulator in fixed point (x 2^62), else null
  double* scale_d;     // (1-c) / d_u, 0 for dead-ends
  float* scale_f;
  int* mark;           // frontier membership stamps
  int* q0; int* q1;    // frontier queues
  unsigned char* dead;
  unsigned char* seedflag;  // 1 for the seed node(s): they cannot be deleted
  int* del_pos;        // first deletion position in the batch (kNoPos if none)
  int* clr_pos;        // last OSP_OP_ZERO_ROW position of the last batch (-1 if none)
  int* rflag; int* cflag;
  // batch scratch: net edits grouped per changed row / column
  int* ins_r; int* del_r; int* ins_c; int* del_c;   // [kMaxBatch]
  int* gi; int* gd;                                  // [kMaxBatch + 1] prefix counts
  int* rec_r_node; int* rec_r_is; int* rec_r_ic; int* rec_r_ds; int* rec_r_dc;  // [nc]
  int* rec_c_node; int* rec_c_is; int* rec_c_ic; int* rec_c_ds; int* rec_c_dc;  // [nc]
  int* del_nodes;  // [kMaxBatch]
  int* clr_nodes;  // [kMaxBatch] rows zeroed by the last ingested batch
  // merge plan over the changed lists (out-lists first, then in-lists)
  unsigned* rec_old_off; int* rec_old_len; int* rec_pstart;  // [2 nc + 1]
  unsigned* rec_fbase; int* rec_dp;                          // [2 nc]
  int* piece_rec; int* piece_cnt; int* piece_base;           // [2 nc + 2 pool cap / kPiece + 2]
  // pull-step plan: prefix of in-list lengths, warp tasks of about
  // kTaskItems items (edges + nodes, lists never split), and the long in-lists
  // summed in pieces
  unsigned* pc;                       // [nc + 1]  pc[v] = sum of in-list lengths below v
  int* task_first;                    // [(kMultiNodeItems nc + pool cap) / kMinTaskItems + 2] first node of each warp task
  int* hubs; int* hub_pstart; double* hub_acc; int* hub_cnt;  // [pool cap / kHubThreshold + 2]
  int* piece_hub;  // [2 pool cap / kMultiHub + 4] the long in-list each piece belongs to
  double* piece_part;  // [as piece_hub] deterministic mode: per-piece partial sums
  double* hub_l1;      // [as hubs] deterministic mode: |x_v| of each long in-list's node
  int* big_u; double* big_y;  // push step: rows longer than kHubThreshold [pool cap / kHubThreshold + 2]
  // reductions and history
  double* part_l1; long long* part_ef;  // [kMaxGrid]
  double* l1_hist;                      // [kMaxHist]
  unsigned long long* step_ns;          // [kMaxHist + 1] device clock at kernel start and after each step
  Ctl* ctl;
  Multi mu;  // several seeds (unused with one seed)
};

// Radix-select state of a top-k query.
struct TopkState {
  unsigned long long prefix;  // selected leading bits of the order key
  int bits;                   // how many leading bits are selected
  int k_rem;                  // rank still to find inside the selected bin
  int done;
  int count;                  // survivors handed to the final sort
  int above;                  // keys above the bin (all of them are in the top k)
  int bin_count;              // keys inside the bin
  int keep;                   // bin keys kept (all, or the k_rem smallest ids of one key value)
  int pad;
  unsigned long long kmin;    // smallest and largest key matching the prefix in the last pass
  unsigned long long kmax;
};

// One top-k job: a score vector of n entries, its scratch, its outputs (device
// or host-mapped memory). A launch serves up to kTopkMaxJobs of them.
struct TopkJob {
  const double* src;
  TopkState* st;
  unsigned* hist;            // [4096]
  int* blk_a; int* blk_b;    // [n / kTopkChunk + 2]
  unsigned long long* keys;  // [kTopkMaxK + kTopkCand]
  int* ids;                  // [kTopkMaxK + kTopkCand]
  const double* norm;        // ||src||_1 to divide the output scores by, or null
  int* out_ids; double* out_sc; int* out_k;
};
constexpr int kTopkMaxJobs = 32;
struct TopkJobs {  // passed by value (about 3 KB of kernel parameters)
  int m, n, k, pad;
  TopkJob j[kTopkMaxJobs];
};
struct GatherJobs {
  int col[kTopkMaxJobs];
  double* dst[kTopkMaxJobs];
};

struct PropParams {
  double eps;
  int max_iter;
  int force_iters;
  double alpha;
  double beta;
  int fp32;
  int hot_n;  // seed block: gather rows of internal ids below hot_n are kept in L2 first
  int det;    // one seed: pull steps only, static work order, long lists combined in order
};

// ---------------------------------------------------------------------------
// Checked builds (-DOSP_CHECKED): index checks that report the first bad
// access, set an error status and skip the access instead of performing it.
// ---------------------------------------------------------------------------
#ifdef OSP_CHECKED
#define OSP_GUARD(ctl, cond, what, a, b, c)                                             \
  ((cond) ? true                                                                        \
          : (printf("osp check failed: %s (%lld %lld %lld) block %d thread %d\n", what, \
                    (long long)(a), (long long)(b), (long long)(c), blockIdx.x,         \
                    threadIdx.x),                                                       \
             atomicCAS(&(ctl)->status, 0, (int)OSP_ECUDA), false))
#else
#define OSP_GUARD(ctl, cond, what, a, b, c) true
#endif

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// lower_bound over an ascending int array
__device__ __forceinline__ int lower_bound_i(const int* a, int n, int x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool contains_i(const int* a, int n, int x) {
  int p = lower_bound_i(a, n, x);
  return p < n && a[p] == x;
}

// Warp-aggregated append of `want` lanes' values to a queue (all lanes of the
// warp must call this together).
__device__ __forceinline__ void warp_append(bool want, int val, int* queue, int* counter) {
  unsigned b = __ballot_sync(0xffffffffu, want);
  if (!b) return;
  int leader = __ffs(b) - 1;
  int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(b));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) queue[base + __popc(b & lanemask_lt())] = val;
}

}  // namespace osp

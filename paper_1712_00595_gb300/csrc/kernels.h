// Kernel entry points of the engine (internal).
#pragma once
#include "common.cuh"

namespace osp {

__global__ void k_reset_batch(Dev d, int cont);
__global__ void k_cpi_begin(Dev d);
__global__ void k_cpi_begin_uniform(Dev d, int n0);
__global__ void k_ingest(Dev d, const osp_update* __restrict__ ops, int U);
__global__ void k_expand(Dev d);
__global__ void k_merge_pieces(Dev d, double beta);
__global__ void k_merge_count(Dev d);
__global__ void k_merge_plan(Dev d);
__global__ void k_merge_write(Dev d);
__global__ void k_merge_finish(Dev d);
__global__ void k_pull_plan(Dev d, int hub_thr, int node_w, int task_items);
__global__ void k_hub_prefix(Dev d, int hub_piece, int det);
__global__ void k_set_scale(Dev d, int n, double c);
__global__ void k_scan_local(const int* __restrict__ len, unsigned* out, unsigned* bsum, int n);
__global__ void k_scan_top(unsigned* bsum, int nb);
__global__ void k_scan_add(unsigned* out, const unsigned* __restrict__ bsum, int n);
__global__ void k_compact_copy(const unsigned* __restrict__ off_old, const int* __restrict__ len,
                               const int* __restrict__ pool_old, const unsigned* __restrict__ off_new,
                               int* pool_new, int n);
__global__ void k_abs_sum(const double* __restrict__ r, int n, double* out, double* parts);
__global__ void k_gather_ext(const double* __restrict__ r, const int* __restrict__ ext2int, int n,
                             double* out);
__global__ void k_scale_copy(const double* r, int n, const double* __restrict__ sum, double* out);

// Top-k (radix select + ordered compaction + one-CTA bitonic sort) over a job
// table: enqueue_topk_select runs the selection and compaction (16 launches),
// enqueue_topk_sort the final sort (k_topk_sort needs the dynamic shared
// memory attribute set to kTopkSortSmem). Both return their launch counts.
__global__ void k_topk_sort(TopkJobs J, int cap);
__global__ void k_gather_cols(const double* __restrict__ r, int Sp, const int* __restrict__ int2ext,
                              int n, GatherJobs G);
int enqueue_topk_select(const TopkJobs& J, int num_sms, cudaStream_t st);
int enqueue_topk_sort(const TopkJobs& J, cudaStream_t st);
constexpr int kTopkMaxK = 4096;
constexpr int kTopkCand = 4096;
constexpr int kTopkChunk = 4096;
constexpr int kTopkSortSmem = (kTopkMaxK + kTopkCand) * (int)(sizeof(unsigned long long) + sizeof(int));

// Propagation (persistent, cooperative launch). T = double or float.
template <typename T>
__global__ void k_propagate(Dev d, PropParams pp);

// Several seeds (csrc/multi.cu).
__global__ void k_offset_multi_plan(Dev d);
__global__ void k_multi_cpi_begin(Dev d);
__global__ void k_gather_col(const double* __restrict__ r, int Sp, int col,
                             const int* __restrict__ ext2int, int n, double* out);
// bulk: the variant that stages source rows in shared memory by bulk copies.
int propagate_multi_grid(int precision, int KG, int num_sms, bool bulk);
cudaError_t launch_propagate_multi(const Dev& d, const PropParams& pp, int precision, int KG,
                                   int grid, bool bulk, cudaStream_t s);
cudaError_t launch_offset_multi(const Dev& d, int grid, cudaStream_t s);
// Failure-detection self-test: which 0 = grid barrier, 1 = staged-row mbarrier;
// lose != 0 makes the wait run out (src: 64 floats on the device).
cudaError_t launch_selftest(Ctl* ctl, const float* src, int which, int lose, cudaStream_t s);

// Host helper: the number of CTAs the persistent kernel can keep resident.
int propagate_grid(int fp32, int num_sms);
cudaError_t launch_propagate(const Dev& d, const PropParams& pp, int grid, cudaStream_t s);

}  // namespace osp

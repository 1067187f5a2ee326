// Top-k over a caller's device score vector without any allocation.
//
// Some callers cannot call cudaMalloc at query time: a serving process that
// has handed all free device memory to its own pool allocator has none left to
// give, and a latency-bound loop cannot afford the device-wide synchronisation
// that cudaMalloc and cudaFree may imply. This entry point runs the same radix
// select, ordered compaction and one-CTA sort as osp_topk, but its scratch is a
// fixed array in the library's own device memory (one per device), reserved
// when the module is loaded, so the call itself allocates nothing.
//
// The array is shared by every call on a device, so calls whose kernels could
// overlap on the GPU (two streams, or two host threads) race on it; callers
// must order them, for example by issuing them on one stream. The per-device
// set-up is done once per process; a cudaDeviceReset between calls (which
// recreates the context and reloads the module) is not supported.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace osp {
namespace {

constexpr int kMaxN = OSP_TOPK_NOALLOC_MAX_N;
constexpr int kMaxChunks = kMaxN / kTopkChunk + 2;
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Layout of the scratch array (each part 256-byte aligned).
constexpr size_t kOffState = 0;
constexpr size_t kOffSum = kOffState + align256(sizeof(TopkState));
constexpr size_t kOffHist = kOffSum + align256(sizeof(double));
constexpr size_t kOffKeys = kOffHist + align256(sizeof(unsigned) * 4096);
constexpr size_t kOffIds = kOffKeys + align256(sizeof(unsigned long long) * (kTopkMaxK + kTopkCand));
constexpr size_t kOffBlkA = kOffIds + align256(sizeof(int) * (kTopkMaxK + kTopkCand));
constexpr size_t kOffBlkB = kOffBlkA + align256(sizeof(int) * kMaxChunks);
constexpr size_t kScratchBytes = kOffBlkB + align256(sizeof(int) * kMaxChunks);
static_assert(kScratchBytes <= 180 * 1024, "scratch larger than stated in osp.h");

static __device__ __align__(256) unsigned char g_topk_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSlot {
  unsigned char* base;
  int num_sms;
  bool ready;
};
std::mutex g_mu;
DeviceSlot g_slot[kMaxDevices];

// Once per device, with that device current: the scratch address on it, the
// SM count and the sort kernel's shared-memory limit.
osp_status device_setup(int dev, unsigned char** base, int* num_sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceSlot& s = g_slot[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_topk_scratch) != cudaSuccess) return OSP_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return OSP_ECUDA;
    if (cudaFuncSetAttribute(k_topk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTopkSortSmem) != cudaSuccess)
      return OSP_ECUDA;
    s.base = (unsigned char*)p;
    s.num_sms = sms;
    s.ready = true;
  }
  *base = s.base;
  *num_sms = s.num_sms;
  return OSP_OK;
}

}  // namespace
}  // namespace osp

using namespace osp;

extern "C" osp_status osp_topk_noalloc(const double* scores_device, int64_t n, int32_t k,
                                       int normalize, int32_t* ids_device,
                                       double* out_scores_device, int32_t* k_out_device,
                                       void* stream) {
  if (n < 0 || n > kMaxN || k <= 0 || k > kTopkMaxK || (n > 0 && !scores_device) ||
      !ids_device || !out_scores_device || !k_out_device)
    return OSP_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OSP_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return OSP_EINVAL;
  unsigned char* base = nullptr;
  int sms = 0;
  const osp_status s = device_setup(dev, &base, &sms);
  if (s != OSP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return cudaMemsetAsync(k_out_device, 0, sizeof(int32_t), st) == cudaSuccess
                         ? OSP_OK : OSP_ECUDA;

  TopkState* state = (TopkState*)(base + kOffState);
  double* sum = (double*)(base + kOffSum);
  unsigned* hist = (unsigned*)(base + kOffHist);
  unsigned long long* keys = (unsigned long long*)(base + kOffKeys);
  int* ids = (int*)(base + kOffIds);
  int* blk_a = (int*)(base + kOffBlkA);
  int* blk_b = (int*)(base + kOffBlkB);
  const int nn = (int)n;

  // k_topk_reset clears the state and the histogram; the per-chunk counts are
  // written whole by k_topk_count; only the norm accumulator is cleared here.
  TopkJobs J{};
  J.m = 1;
  J.n = nn;
  J.k = k;
  TopkJob& jb = J.j[0];
  jb.src = scores_device;
  jb.st = state;
  jb.hist = hist;
  jb.blk_a = blk_a;
  jb.blk_b = blk_b;
  jb.keys = keys;
  jb.ids = ids;
  jb.norm = normalize ? sum : nullptr;
  jb.out_ids = ids_device;
  jb.out_sc = out_scores_device;
  jb.out_k = k_out_device;
  if (normalize) {
    if (cudaMemsetAsync(sum, 0, sizeof(double), st) != cudaSuccess) return OSP_ECUDA;
    k_abs_sum<<<sms * 2, 256, 0, st>>>(scores_device, nn, sum, nullptr);
  }
  enqueue_topk_select(J, sms, st);
  enqueue_topk_sort(J, st);
  return cudaGetLastError() == cudaSuccess ? OSP_OK : OSP_ECUDA;
}

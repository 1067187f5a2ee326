// Grid-wide barrier of the persistent cooperative kernels: the last CTA to
// arrive runs the step decision, then opens the barrier; the others wait with
// a bounded spin (time and iteration limits) and stop on a timeout or an
// error status, so a lost CTA cannot hang the device.
#pragma once
#include "common.cuh"

namespace osp {

static constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s
static constexpr unsigned kBarrierMaxSpins = 1u << 26;

struct BarShared {
  unsigned gen;
  int last;
  int ok;
};

static __device__ __forceinline__ bool bar_arrive(Ctl* ctl, BarShared& sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = *(volatile unsigned*)&ctl->bar_gen;
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->bar_count, 1u);
    sh.gen = g;
    sh.last = prev == gridDim.x - 1;
  }
  __syncthreads();
  return sh.last;
}

// The last CTA opens the barrier; the others wait with a time limit. Returns
// false when the kernel must stop (timeout or an error status).
static __device__ __forceinline__ bool bar_release(Ctl* ctl, BarShared& sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (sh.last) {
      ctl->bar_count = 0;
      __threadfence();
      atomicAdd(&ctl->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (*(volatile unsigned*)&ctl->bar_gen == sh.gen) {
        __nanosleep(32);
        ++spins;
        if (spins >= kBarrierMaxSpins ||
            ((spins & 1023u) == 0 && global_ns() - t0 > kBarrierTimeoutNs)) {
          atomicCAS(&ctl->status, 0, (int)OSP_ETIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*(volatile int*)&ctl->status != 0) ok = 0;
    sh.ok = ok;
  }
  __syncthreads();
  return sh.ok;
}

}  // namespace osp

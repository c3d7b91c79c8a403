// device.cuh -- device-side helpers of liblp: control block, bounded grid barrier.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lp {

constexpr unsigned FULL = 0xffffffffu;

// Per-handle control block in device memory; zeroed before every solve.
struct DeviceCtl {
  unsigned long long bar; // grid barrier arrivals in this launch (monotone)
  unsigned flag[3];      // "some row changed" flags, rotating over iterations
  int status;            // lp_status reported by the device
  int iters;             // theta applications (least model) / last tile's count
  unsigned abort;        // set when a block gave up waiting
  int max_tile_iters;    // stable models: largest per-tile iteration count
  long long sum_tile_iters;
  long long n_stable;    // stable guesses found so far
  long long tiles;
  unsigned long long timeout_site;  // where a wait gave up (diagnostics)
  unsigned long long count[3];      // true rows per iteration, rotating (monotone runs)
  unsigned long long init_count;    // true rows of the initial vector
};

// Upper bound of one barrier wait. A healthy wait takes microseconds; after this the waiting
// block records LP_ERR_TIMEOUT, raises the abort flag and returns instead of spinning on.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a co-resident (cooperative) grid. `round` counts the barriers of this
// launch from 1; every block must call it the same number of times. Release: fence before the
// arrival; acquire: acquire loads while waiting and a fence after, then a CTA barrier, so
// ordinary loads after it see every write made before it by any block. Returns false if the
// grid is aborting (this or another block gave up waiting); callers must then return. A wait
// gives up after limit_ns (2 s unless a caller passes less).
__device__ __forceinline__ bool grid_barrier(DeviceCtl* ctl, unsigned long long round, int status_on_timeout,
                                             unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ unsigned s_abort;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&ctl->bar, 1ull);
    const unsigned long long target = round * gridDim.x;
    unsigned polls = 0;
    unsigned long long t0 = 0;
    unsigned ab = 0;
    while (ld_acquire64(&ctl->bar) < target) {
      if ((ab = ld_volatile(&ctl->abort)) != 0) break;
      if (++polls == 64) t0 = global_ns();
      if (polls > 64) {
        __nanosleep(100);
        if ((polls & 255) == 0 && global_ns() - t0 > limit_ns) {
          atomicExch(&ctl->abort, 1u);
          atomicCAS(&ctl->status, 0, status_on_timeout);
          atomicExch(&ctl->timeout_site, round);
          ab = 1;
          break;
        }
      }
    }
    __threadfence();
    s_abort = ab;
  }
  __syncthreads();
  return s_abort == 0;
}

}  // namespace lp

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
  // stable models, frontier schedule: rows re-evaluated, their entries, changed-row list
  // items expanded, and dependents visited, summed over the launch's iterations after the first
  unsigned long long fr_rows, fr_entries, fr_list, fr_deps;
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
// launch from 1; every block must call it the same number of times. Arrival: a release
// reduction on the monotone counter; wait: acquire loads until it counts round x gridDim.x
// blocks; CTA barriers on both sides, so ordinary loads after it see every write made before
// it by any block. Returns false if the grid is aborting (this or another block gave up
// waiting); callers must then return. A wait gives up after limit_ns (2 s unless a caller
// passes less).
__device__ __forceinline__ void red_release_add64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ bool grid_barrier(DeviceCtl* ctl, unsigned long long round, int status_on_timeout,
                                             unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ unsigned s_abort;
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add64(&ctl->bar, 1ull);
    const unsigned long long target = round * gridDim.x;
    unsigned polls = 0;
    unsigned long long t0 = 0;
    unsigned ab = 0;
    while (ld_acquire64(&ctl->bar) < target) {
      if (++polls == 1024) t0 = global_ns();
      if (polls > 1024 && (polls & 63) == 0) {
        if ((ab = ld_volatile(&ctl->abort)) != 0) break;
        __nanosleep(32);
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&ctl->abort, 1u);
          atomicCAS(&ctl->status, 0, status_on_timeout);
          atomicExch(&ctl->timeout_site, round);
          ab = 1;
          break;
        }
      }
    }
    s_abort = ab;
  }
  __syncthreads();
  return s_abort == 0;
}

// Grid-wide barrier that also ORs one flag over the grid, for the least-model loop: a block
// adds 1 + (flag ? 2^32 : 0) to the counter of this round's slot (three slots rotate over the
// rounds) and waits until the low half counts every block; the high half then says whether
// any block raised its flag. One atomic and two CTA barriers per round. The arrival is a
// release reduction and the wait an acquire load (both at GPU scope); with the CTA barriers
// around them every write a block made before the barrier is visible to every block after it.
// Block 0 clears the slot of round + 1 before it arrives: that slot was last used three rounds
// back, and every block finished reading it before arriving at the round in between, while
// nobody adds to it before this round completes, which needs block 0's arrival. `ctl->count`
// must be zero at launch. Returns false if the grid is aborting; *any_flag is valid when it
// returns true.

__device__ __forceinline__ bool grid_barrier_or(DeviceCtl* ctl, unsigned long long round, bool flag,
                                                bool* any_flag, int status_on_timeout,
                                                unsigned long long limit_ns = kWaitLimitNs) {
  __shared__ unsigned s_state;  // bit 0: abort, bit 1: some block raised its flag
  const int mine = __syncthreads_or(flag);
  if (threadIdx.x == 0) {
    unsigned long long* slot = &ctl->count[round % 3];
    if (blockIdx.x == 0) ctl->count[(round + 1) % 3] = 0ull;
    red_release_add64(slot, mine ? (1ull << 32) + 1ull : 1ull);
    const unsigned long long target = gridDim.x;
    unsigned polls = 0;
    unsigned long long t0 = 0, v;
    unsigned ab = 0;
    while (((v = ld_acquire64(slot)) & 0xffffffffull) < target) {
      if (++polls == 1024) t0 = global_ns();
      if (polls > 1024 && (polls & 63) == 0) {
        if ((ab = ld_volatile(&ctl->abort)) != 0) break;
        __nanosleep(32);
        if (global_ns() - t0 > limit_ns) {
          atomicExch(&ctl->abort, 1u);
          atomicCAS(&ctl->status, 0, status_on_timeout);
          atomicExch(&ctl->timeout_site, round);
          ab = 1;
          break;
        }
      }
    }
    s_state = (ab ? 1u : 0u) | ((v >> 32) ? 2u : 0u);
  }
  __syncthreads();
  const unsigned st = s_state;
  *any_flag = (st & 2u) != 0;
  return (st & 1u) == 0;
}

}  // namespace lp

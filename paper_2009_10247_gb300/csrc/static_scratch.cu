// static_scratch.cu -- lp_least_model_static: the least-model loop on a matrix the caller
// already holds in device memory, with no device allocation at all.
//
// Who needs it: code that may not call cudaMalloc/cudaFree on its path -- a caller running
// under another framework's memory budget or pool, a latency-critical loop that cannot take
// the implicit synchronisation an allocation may cause, or a host process that must not grow
// its device footprint after start-up. lp_compile allocates the program matrix and the
// solver scratch behind every handle; this entry point instead takes the matrix and the two
// vectors from the caller and keeps its only scratch (the second iterate vector and the
// control block of the grid barrier) in one fixed array that lives in this library's image.
//
// The array below is a file-scope __device__ variable: every GPU that loads liblp holds it
// (kStaticScratchBytes) until the process exits. Host code must not use its name as a device
// address; the address is looked up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "device.cuh"
#include "internal.h"

namespace lp {
namespace {

// Largest matrix the static scratch serves: 2^24 rows (one 2 MiB bit vector).
constexpr int64_t kStaticMaxRows = int64_t(1) << 24;
constexpr size_t kCtlBytes = 256;  // control block, at the start of the array
constexpr size_t kStaticScratchBytes = kCtlBytes + kStaticMaxRows / 8;
static_assert(sizeof(DeviceCtl) <= kCtlBytes, "control block must fit its slot");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kStaticBlock = 256;
constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_static_scratch
  int max_grid = 0;                  // co-resident blocks of the kernel
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Rows r >= n_rows of the last word are empty (never true).
__device__ __forceinline__ uint32_t static_theta_word(int n_rows, const int32_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col,
                                                      const int32_t* __restrict__ threshold, const uint32_t* src,
                                                      int w, int lane, bool* bad) {
  const int r = (w << 5) + lane;
  const int rr = min(r, n_rows);
  const int beg = __ldg(row_ptr + rr);
  const int end = r < n_rows ? __ldg(row_ptr + rr + 1) : beg;
  const int base = __shfl_sync(FULL, beg, 0);
  const int stop = __shfl_sync(FULL, end, 31);
  int cnt = 0;
  for (int c = base; c < stop; c += 32) {
    const int e = c + lane;
    uint32_t bit = 0;
    if (e < stop) {
      const int j = __ldg(col + e);
      if ((unsigned)j < (unsigned)n_rows) bit = (src[j >> 5] >> (j & 31)) & 1u;
      else *bad = true;  // column outside the matrix: reported, never read
    }
    const uint32_t m = __ballot_sync(FULL, bit);
    const int lo = max(beg - c, 0), hi = min(end - c, 32);
    if (hi > lo) {
      const uint32_t sel = (hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo);
      cnt += __popc(m & sel);
    }
  }
  const int thr = r < n_rows ? max(__ldg(threshold + r), 1) : 1;
  return __ballot_sync(FULL, cnt >= thr);
}

struct StaticArgs {
  int32_t n_rows;
  int32_t n_words;  // 2 * ceil(n_rows / 64): the caller's vectors viewed as 32-bit words
  const int32_t* row_ptr;
  const int32_t* col;
  const int32_t* threshold;
  const uint32_t* v0;
  uint32_t* out;  // iterate buffer 0, and the result
  uint32_t* x1;   // iterate buffer 1 (static scratch)
  DeviceCtl* ctl; // control block (static scratch, zeroed before the launch)
  int32_t max_iters;
};

__global__ void __launch_bounds__(kStaticBlock) static_fixpoint_kernel(StaticArgs a) {
  __shared__ int s_flag;
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;

  // v0 -> out (a no-op when they are the same buffer); padding rows read as 0
  for (int w = gtid; w < a.n_words; w += nthreads) {
    uint32_t word = a.v0[w];
    const int64_t first = (int64_t)w * 32;
    if (first + 32 > a.n_rows) word = first >= a.n_rows ? 0u : (word & ((1u << (a.n_rows - first)) - 1u));
    a.out[w] = word;
  }
  if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) return;

  const uint32_t* fin = a.out;
  int it = 0;
  bool converged = false;
  for (; it < a.max_iters; ++it) {
    const uint32_t* src = (it & 1) ? a.x1 : a.out;
    uint32_t* dst = (it & 1) ? a.out : a.x1;
    bool changed = false, bad = false;
    for (int w = gwarp; w < a.n_words; w += nwarps) {
      const uint32_t u = static_theta_word(a.n_rows, a.row_ptr, a.col, a.threshold, src, w, lane, &bad);
      if (lane == 0) {
        dst[w] = u;
        changed |= (u != src[w]);
      }
    }
    if (bad) atomicCAS(&ctl->status, 0, LP_ERR_INVALID);
    const int any_changed = __syncthreads_or(changed);
    if (threadIdx.x == 0) {
      if (any_changed) atomicOr(&ctl->flag[it % 3], 1u);
      if (blockIdx.x == 0) ctl->flag[(it + 1) % 3] = 0u;
    }
    if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) return;
    if (threadIdx.x == 0) s_flag = (int)ld_volatile(&ctl->flag[it % 3]);
    __syncthreads();
    fin = dst;
    if (!s_flag) {
      converged = true;
      ++it;
      break;
    }
  }
  if (gtid == 0) {
    ctl->iters = it;
    if (!converged) atomicCAS(&ctl->status, 0, LP_ERR_NO_FIXPOINT);
  }
  if (fin != a.out)  // the last iterate is in the scratch vector: copy it to the caller
    for (int w = gtid; w < a.n_words; w += nthreads) a.out[w] = fin[w];
}

lp_status static_fail(lp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

// Once per device, with that device current: the device address of the static array and the
// kernel's co-resident grid size.
lp_status static_setup(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= kMaxDevices) return static_fail(LP_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return static_fail(LP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, static_fixpoint_kernel, kStaticBlock, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return static_fail(LP_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
    if (per_sm < 1) return static_fail(LP_ERR_CUDA, "static fixpoint kernel cannot be resident");
    s.scratch = static_cast<unsigned char*>(ptr);
    s.max_grid = per_sm * sms;
    s.ready = true;
  }
  *out = &s;
  return LP_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace lp

using namespace lp;

extern "C" lp_status lp_least_model_static(int32_t n_rows, const int32_t* row_ptr, const int32_t* col,
                                           const int32_t* threshold, const uint64_t* v0, uint64_t* out,
                                           int32_t max_iters, int32_t* iters_out, void* cuda_stream) {
  if (n_rows < 0) return static_fail(LP_ERR_INVALID, "n_rows must be >= 0");
  if (n_rows > kStaticMaxRows)
    return static_fail(LP_ERR_INVALID, "n_rows " + std::to_string(n_rows) + " exceeds the static scratch limit of " +
                                           std::to_string(kStaticMaxRows) + " rows");
  if (max_iters < 1) return static_fail(LP_ERR_INVALID, "max_iters must be >= 1");
  if (n_rows > 0 && (!row_ptr || !col || !threshold || !v0 || !out))
    return static_fail(LP_ERR_INVALID, "row_ptr, col, threshold, v0 and out must not be NULL");
  if (n_rows > 0 && !(on_device(row_ptr) && on_device(col) && on_device(threshold) && on_device(v0) && on_device(out)))
    return static_fail(LP_ERR_INVALID, "every buffer must be device memory (this entry point stages nothing)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(LP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  DeviceSetup* setup = nullptr;
  lp_status st = static_setup(dev, &setup);
  if (st != LP_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DeviceCtl* ctl = reinterpret_cast<DeviceCtl*>(setup->scratch);
  // The array keeps the previous call's contents: the control block must start at zero.
  e = cudaMemsetAsync(ctl, 0, kCtlBytes, s);
  if (e != cudaSuccess) return static_fail(LP_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  StaticArgs a{};
  a.n_rows = n_rows;
  a.n_words = 2 * ((n_rows + 63) / 64);
  a.row_ptr = row_ptr;
  a.col = col;
  a.threshold = threshold;
  a.v0 = reinterpret_cast<const uint32_t*>(v0);
  a.out = reinterpret_cast<uint32_t*>(out);
  a.x1 = reinterpret_cast<uint32_t*>(setup->scratch + kCtlBytes);
  a.ctl = ctl;
  a.max_iters = max_iters;
  const int warps_per_block = kStaticBlock / 32;
  const int grid = std::max(1, std::min(setup->max_grid, (a.n_words + warps_per_block - 1) / warps_per_block));
  void* params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)static_fixpoint_kernel, dim3(grid), dim3(kStaticBlock), params, 0, s);
  if (e != cudaSuccess) return static_fail(LP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (iters_out) {
    DeviceCtl h;
    std::memset(&h, 0, sizeof(h));
    e = cudaMemcpyAsync(&h, ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return static_fail(LP_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    *iters_out = h.iters;
    if (h.status == LP_ERR_INVALID) return static_fail(LP_ERR_INVALID, "a column index is outside [0, n_rows)");
    if (h.status == LP_ERR_NO_FIXPOINT) return static_fail(LP_ERR_NO_FIXPOINT, "no fixpoint within max_iters");
    if (h.status == LP_ERR_TIMEOUT) return static_fail(LP_ERR_TIMEOUT, "a grid barrier wait timed out; kernel aborted");
    if (h.status != 0) return static_fail(LP_ERR_CUDA, "device reported status " + std::to_string(h.status));
  }
  return LP_OK;
}

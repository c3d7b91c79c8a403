// program.h -- liblp's program handle and the helpers its C ABI translation units share.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct lp_program {
  lp::HostMatrix hm;  // metadata (row_ptr/col host copies are dropped after upload)
  int device = 0;
  int sm_count = 0;
  // device copy of the matrix and its tables
  int32_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  uint32_t* any_mask = nullptr;
  int32_t* perm = nullptr;
  int32_t* inv = nullptr;  // internal -> canonical, uploaded on first LP_ROWS call
  int32_t* fact_row = nullptr;
  int32_t* fact_owner = nullptr;
  uint64_t* fact_mask = nullptr;
  int32_t* neg_row = nullptr;
  int32_t* bar_row = nullptr;
  int32_t* row_tag = nullptr;
  // a device compile keeps the canonical kinds and rules here until a host-side user downloads
  // them with perm (ensure_host_tables); a host compile has them in hm from the start
  int8_t* dc_kind = nullptr;
  int32_t* dc_rule = nullptr;
  bool host_tables = true;
  // streamed layout of the least-model kernel
  uint32_t* desc = nullptr;
  int32_t* word_hdr = nullptr;
  int32_t* and_col = nullptr;
  int32_t* groups = nullptr;
  // sliced layout of the least-model kernel 2 (built on the device on first use)
  int32_t* sl_q = nullptr;        // internal row -> slice row
  int32_t* sl_qinv = nullptr;     // slice row -> internal row
  int4* sl_hdr = nullptr;         // per slice
  int32_t* sl_col = nullptr;      // entries
  int32_t* sl_fact_row = nullptr;
  int32_t* sl_perm = nullptr;
  int64_t sl_entries = -1;        // stored entries; -1 = not built
  // frontier schedule of the stable models: transposed matrix and counters (built on first use),
  // and the buffers of one wave of fr_tiles tiles of fr_W words (iterates, stamps, lists, bitmap)
  int32_t* fr_tptr = nullptr;
  int32_t* fr_seed = nullptr;  // fact rows, then guessed rows (the first list's sources)
  int32_t fr_nseed = 0;
  int32_t* fr_tidx = nullptr;
  unsigned* fr_cnt = nullptr;
  unsigned* fr_long = nullptr;  // rows the frontier evaluates a warp at a time
  bool fr_any_long = false;
  uint32_t* fr_F = nullptr;     // the guess-independent fixpoint (stable_frontier 2), internal rows
  DevBuf fr_buf;
  int32_t fr_W = 0, fr_tiles = 0;
  // scratch
  uint32_t* x[2] = {nullptr, nullptr};
  lp::DeviceCtl* ctl = nullptr;
  lp::DeviceCtl* h_ctl = nullptr;  // pinned mirror of ctl
  DevBuf tiles;                // stable-model iterate buffers
  DevBuf stage_in, stage_out, stage_out2;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  lp_schedule sched{};         // schedule of the solves (lp_set_schedule / lp_autotune)
  DevBuf tune_out, tune_in;    // autotuner result and guess buffers
  int64_t last_launches = 0;
  int64_t tile_words = 0;
  int64_t device_bytes = 0;
  int64_t upload_bytes = 0;
  double compile_ms = 0.0;
  bool host_only = false;  // LP_COMPILE_HOST_ONLY: host arrays kept, nothing on the device
  // relaxed (differentiable) path, built on first use
  bool rx_ready = false;
  int32_t* rx_info = nullptr;    // per internal row: kind << 30 | entries
  int32_t* rx_rule = nullptr;    // per internal row: original rule of a rule row, else -1
  int32_t* rx_colptr = nullptr;  // transpose (CSC) of the rule and OR rows
  int32_t* rx_rowidx = nullptr;
  DevBuf rx_dw;                  // per-row weight-gradient accumulators (double)
  void* rx_units = nullptr;      // fixed reduction tree of the transpose (RxUnit records, by level)
  std::vector<int64_t> rx_level_off;   // first unit of each level (+ end)
  std::vector<int64_t> rx_part_off;    // first partial row of each level's output (+ end)
  DevBuf rx_part;                // partial sums of the tree, rx_part_off.back() x batch floats
};

namespace lp {

lp_status fail(lp_status st, const std::string& msg);
lp_status cuda_fail(cudaError_t e, const char* what);
lp_status ensure(lp_program* p, DevBuf& b, size_t bytes);
bool is_device_ptr(const void* ptr);
lp_status launch_count_and_check(cudaError_t e, const char* what, lp_program* p);
void count_launches(int64_t n);  // add to lp_launch_count()

#define LP_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// cudaMalloc behind the allocation-failure hook (lp_debug_fail_alloc): every device allocation
// of liblp's handles goes through here, and small ones are reused across handles (api.cu).
cudaError_t device_malloc(void** ptr, size_t bytes);
// Frees what device_malloc returned (NULL entries are skipped); waits for the device first, as
// cudaFree does.
void device_free_all(void* const* ptrs, size_t n);
void device_free(void* ptr);
// The standardization of lp_compile on the device (compile_device.cu): fills the device arrays
// of the handle and hm's sizes and small tables; perm, canon_kind and canon_rule reach hm on
// demand through ensure_host_tables.
lp_status compile_on_device(lp_program* p, int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                            const int32_t* body_atom, const uint8_t* body_neg, cudaStream_t s);
lp_status ensure_host_tables(lp_program* p, cudaStream_t s);
// Stream-ordered allocation (freed with cudaFreeAsync on the same stream), with the same
// injected failures as device_malloc.
cudaError_t device_malloc_async(void** ptr, size_t bytes, cudaStream_t s);

// Least-model kernel 2 (sliced layout): whether the program fits its index widths, and the
// message of LP_ERR_INVALID when it does not.
bool sliced_supported(const lp_program* p);
extern const char* const sliced_unsupported_msg;
// Shared memory that kernel 2 uses at most for the staged vector prefix (the rest of the
// unified L1 / shared array stays L1).
constexpr int kSlicedStageBytesMax = 160 * 1024;
// Least-model kernel 3 (one block, sliced layout in shared memory): whether the program's layout
// fits (builds the sliced layout on stream s if it is not built yet).
lp_status block_kernel_fits(lp_program* p, cudaStream_t s, bool* fits);
lp_status ensure_sliced_layout(lp_program* p, cudaStream_t s);

// NVTX range for the duration of a scope (shows liblp's calls in a profiler's timeline; free
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

template <typename T>
lp_status dalloc(lp_program* p, T** ptr, size_t count) {
  size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = device_malloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  p->device_bytes += (int64_t)bytes;
  return LP_OK;
}

template <typename T, typename A>
lp_status upload(lp_program* p, T** ptr, const std::vector<T, A>& v, cudaStream_t s) {
  lp_status st = dalloc(p, ptr, v.size());
  if (st != LP_OK) return st;
  if (!v.empty()) {
    LP_CUDA(cudaMemcpyAsync(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    p->upload_bytes += (int64_t)(v.size() * sizeof(T));
  }
  return LP_OK;
}

}  // namespace lp

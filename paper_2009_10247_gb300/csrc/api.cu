// api.cu -- the extern "C" entry points of liblp (declared and documented in include/lp.h).
//
// Owns the program handle: the device copy of M_P in the internal layout built by
// compile_host, the per-handle solver scratch (iterate vectors, tile buffers, control block),
// and the staging buffers used when a caller passes host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "kernels.h"
#include "program.h"

namespace lp {

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }

}  // namespace lp

using namespace lp;

namespace lp {

lp_status fail(lp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

lp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(LP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}


namespace {
std::atomic<int64_t> g_fail_alloc_after{-1};  // lp_debug_fail_alloc: -1 = off
}

namespace {
// Small device buffers of the handles are kept for reuse instead of freed: a small program
// compiled, solved and freed in a loop would otherwise spend most of its time in cudaMalloc and
// cudaFree (each a driver call; cudaFree waits for the device). Requests up to 256 KiB are
// rounded up to a power of two and served from per-device free lists; freed blocks go back to
// those lists while they hold at most 16 MiB in all, and are never returned to the driver before
// the process exits. Larger buffers come from the driver each time: with the iterate vectors and
// group headers of a large program in reused blocks, the large least-model solve took 22.6 ms
// against 20.2 ms in fresh ones. LP_ALLOC_CACHE=0 turns the cache off.
constexpr int kCacheMinLog2 = 9;   // 512 B
constexpr int kCacheMaxLog2 = 18;  // 256 KiB
constexpr size_t kCacheCapBytes = 16ull << 20;
struct AllocCache {
  std::mutex mu;
  std::map<void*, std::pair<int, int>> live;           // cached-size blocks in use: (device, log2 size)
  std::map<std::pair<int, int>, std::vector<void*>> free;  // (device, log2 size) -> blocks
  size_t held = 0;                                      // bytes on the free lists
  std::vector<DeviceCtl*> pinned;                       // host control blocks (pinned)
};
AllocCache& alloc_cache() {
  static AllocCache* c = new AllocCache;  // outlives every handle, never destroyed
  return *c;
}
bool alloc_cache_on() {
  static const bool on = [] {
    const char* env = std::getenv("LP_ALLOC_CACHE");
    return !(env && env[0] == '0');
  }();
  return on;
}
int ceil_log2(size_t x) {
  int l = 0;
  while ((size_t(1) << l) < x) l++;
  return l;
}
}  // namespace

cudaError_t device_malloc(void** ptr, size_t bytes) {
  int64_t left = g_fail_alloc_after.load();
  while (left >= 0) {
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {  // this allocation is the one that fails (once)
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  if (!alloc_cache_on() || bytes > (size_t(1) << kCacheMaxLog2)) return cudaMalloc(ptr, bytes);
  const int l = std::max(kCacheMinLog2, ceil_log2(bytes));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  AllocCache& c = alloc_cache();
  {
    std::lock_guard<std::mutex> g(c.mu);
    auto it = c.free.find({dev, l});
    if (it != c.free.end() && !it->second.empty()) {
      *ptr = it->second.back();
      it->second.pop_back();
      c.held -= size_t(1) << l;
      c.live[*ptr] = {dev, l};
      return cudaSuccess;
    }
  }
  e = cudaMalloc(ptr, size_t(1) << l);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(c.mu);
  c.live[*ptr] = {dev, l};
  return cudaSuccess;
}

// Frees device_malloc's buffers: once the device is idle (what cudaFree would wait for), cached
// sizes go back to the free lists, the rest to the driver.
void device_free_all(void* const* ptrs, size_t n) {
  AllocCache& c = alloc_cache();
  std::vector<std::pair<void*, std::pair<int, int>>> keep;
  std::vector<void*> release;
  {
    std::lock_guard<std::mutex> g(c.mu);
    for (size_t i = 0; i < n; i++) {
      if (!ptrs[i]) continue;
      auto it = c.live.find(ptrs[i]);
      if (it == c.live.end()) {
        release.push_back(ptrs[i]);
      } else {
        keep.push_back({ptrs[i], it->second});
        c.live.erase(it);
      }
    }
  }
  if (!keep.empty()) {
    // the blocks' devices finish their work (all blocks of a handle share its device)
    int cur = 0;
    bool ok = cudaGetDevice(&cur) == cudaSuccess;
    const int dev = keep[0].second.first;
    if (ok && dev != cur) ok = cudaSetDevice(dev) == cudaSuccess;
    ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    if (dev != cur) cudaSetDevice(cur);
    cudaGetLastError();
    std::lock_guard<std::mutex> g(c.mu);
    for (auto& [q, dl] : keep) {
      const size_t sz = size_t(1) << dl.second;
      if (ok && dl.first == dev && c.held + sz <= kCacheCapBytes) {
        c.free[dl].push_back(q);
        c.held += sz;
      } else {
        release.push_back(q);
      }
    }
  }
  for (void* q : release) cudaFree(q);
}
void device_free(void* ptr) { device_free_all(&ptr, 1); }

// Pinned host control block of a handle (reused across handles like the device buffers).
cudaError_t pinned_ctl_alloc(DeviceCtl** out) {
  if (alloc_cache_on()) {
    AllocCache& c = alloc_cache();
    std::lock_guard<std::mutex> g(c.mu);
    if (!c.pinned.empty()) {
      *out = c.pinned.back();
      c.pinned.pop_back();
      return cudaSuccess;
    }
  }
  return cudaMallocHost((void**)out, sizeof(DeviceCtl));
}
void pinned_ctl_free(DeviceCtl* q) {
  if (!q) return;
  if (alloc_cache_on()) {
    AllocCache& c = alloc_cache();
    std::lock_guard<std::mutex> g(c.mu);
    if (c.pinned.size() < 64) {
      c.pinned.push_back(q);
      return;
    }
  }
  cudaFreeHost(q);
}

cudaError_t device_malloc_async(void** ptr, size_t bytes, cudaStream_t s) {
  int64_t left = g_fail_alloc_after.load();
  while (left >= 0) {
    if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
      if (left == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  static std::mutex mu;
  static std::vector<int> pools_set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(pools_set.begin(), pools_set.end(), dev) == pools_set.end()) {
      // this process's stream-ordered pool keeps up to 8 GiB between compiles instead of
      // returning it at every synchronization
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = 8ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      cudaGetLastError();
      pools_set.push_back(dev);
    }
  }
  return cudaMallocAsync(ptr, bytes, s);
}

lp_status ensure(lp_program* p, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return LP_OK;
  if (b.p) {
    device_free(b.p);
    p->device_bytes -= (int64_t)b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = device_malloc(&b.p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  b.bytes = std::max<size_t>(bytes, 16);
  p->device_bytes += (int64_t)b.bytes;
  return LP_OK;
}

// true if ptr is device-accessible memory (device or managed), false for host memory.
bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

lp_status ensure_scratch(lp_program* p) {
  if (!p->ctl) {
    lp_status st = dalloc(p, &p->ctl, 1);
    if (st != LP_OK) return st;
    LP_CUDA(pinned_ctl_alloc(&p->h_ctl));
    std::memset(p->h_ctl, 0, sizeof(DeviceCtl));
  }
  if (!p->ev0) {
    LP_CUDA(cudaEventCreate(&p->ev0));
    LP_CUDA(cudaEventCreate(&p->ev1));
  }
  return LP_OK;
}

void release(lp_program* p) {
  void* ptrs[] = {p->row_ptr, p->col, p->any_mask, p->perm, p->inv, p->fact_row, p->fact_owner, p->fact_mask,
                  p->neg_row, p->bar_row, p->row_tag, p->x[0], p->x[1], p->ctl, p->tiles.p, p->stage_in.p,
                  p->stage_out.p, p->stage_out2.p, p->desc, p->word_hdr, p->and_col, p->groups,
                  p->sl_q, p->sl_qinv, p->sl_hdr, p->sl_col, p->sl_fact_row, p->sl_perm,
                  p->fr_tptr, p->fr_tidx, p->fr_cnt, p->fr_long, p->fr_F, p->fr_buf.p, p->dc_kind, p->dc_rule, p->fr_seed,
                  p->rx_info, p->rx_rule, p->rx_colptr, p->rx_rowidx, p->rx_dw.p, p->rx_units, p->rx_part.p,
                  p->tune_out.p, p->tune_in.p};
  device_free_all(ptrs, sizeof(ptrs) / sizeof(ptrs[0]));
  pinned_ctl_free(p->h_ctl);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
}

void count_launches(int64_t n) { g_launches.fetch_add(n); }

lp_status launch_count_and_check(cudaError_t e, const char* what, lp_program* p) {
  if (e != cudaSuccess) return cuda_fail(e, what);
  g_launches.fetch_add(1);
  p->last_launches++;
  return LP_OK;
}

// Waits for the stream and turns the device status into the call's status.
lp_status finish_sync(lp_program* p, cudaStream_t s) {
  LP_CUDA(cudaStreamSynchronize(s));
  const int st = p->h_ctl->status;
  if (st == LP_ERR_INVALID) return fail(LP_ERR_INVALID, "initial vector selects an atom without a fact rule");
  if (st == LP_ERR_NO_FIXPOINT) return fail(LP_ERR_NO_FIXPOINT, "no fixpoint within max_iters");
  if (st == LP_ERR_TIMEOUT) return fail(LP_ERR_TIMEOUT, "a grid barrier wait timed out; kernel aborted");
  if (st != 0) return fail(LP_ERR_CUDA, "device reported status " + std::to_string(st));
  return LP_OK;
}

int max_coresident(lp_program* p, int per_sm) { return std::max(1, per_sm) * p->sm_count; }

cudaError_t set_kernel_smem(const void* kernel, int dyn_bytes, int carveout) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, std::pair<int, int>> last;  // (device, kernel) -> set values
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(dev, kernel);
  auto it = last.find(key);
  // a limit at least as large serves the launch as well
  if (it != last.end() && it->second.first >= dyn_bytes && it->second.second == carveout) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
  if (e != cudaSuccess) return e;
  last[key] = std::make_pair(dyn_bytes, carveout);
  return cudaSuccess;
}

// Kernel 2 indexes its padded entries with int32.
bool sliced_supported(const lp_program* p) { return p->hm.nnz <= (int64_t)INT32_MAX / 4; }
// The sliced layout of kernel 2, built on the device from the CSR on its first use: pass 1
// (renumbering, slice headers, prefix sum), the entry count to the host, pass 2.
lp_status ensure_sliced_layout(lp_program* p, cudaStream_t s) {
  if (p->sl_entries >= 0) return LP_OK;
  const HostMatrix& hm = p->hm;
  const int32_t n_words = hm.n_pad / 32;
  lp_status st;
  int32_t* cnt = nullptr;
  auto fail_clean = [&](lp_status code) {
    if (cnt) device_free(cnt);
    void** ptrs[] = {(void**)&p->sl_q, (void**)&p->sl_qinv, (void**)&p->sl_hdr, (void**)&p->sl_col,
                     (void**)&p->sl_fact_row, (void**)&p->sl_perm};
    for (void** q : ptrs)
      if (*q) {
        device_free(*q);
        *q = nullptr;
      }
    return code;
  };
  if ((st = dalloc(p, &p->sl_q, (size_t)hm.n_pad)) != LP_OK) return fail_clean(st);
  if ((st = dalloc(p, &p->sl_qinv, (size_t)hm.n_pad)) != LP_OK) return fail_clean(st);
  const int32_t n_groups = sliced_groups(hm.n_pad);
  if ((st = dalloc(p, &p->sl_hdr, 3 * (size_t)n_groups + 3)) != LP_OK) return fail_clean(st);
  if ((st = dalloc(p, &p->sl_fact_row, (size_t)hm.n_fact_rows)) != LP_OK) return fail_clean(st);
  if ((st = dalloc(p, &p->sl_perm, (size_t)hm.n_prime)) != LP_OK) return fail_clean(st);
  // scratch: per-group counts, then the total (8-byte aligned after the counts)
  const size_t cnt_ints = ((size_t)n_groups + 2) & ~(size_t)1;
  if (device_malloc((void**)&cnt, (cnt_ints + 2) * 4) != cudaSuccess) {
    cnt = nullptr;
    cudaGetLastError();
    return fail_clean(fail(LP_ERR_OOM, "sliced layout scratch"));
  }
  long long* total_dev = reinterpret_cast<long long*>(cnt + cnt_ints);
  cudaError_t e = build_sliced_pass1(p->row_ptr, p->col, p->any_mask, hm.n_sec_a, hm.n_pad, p->sl_q, p->sl_qinv,
                                     p->sl_hdr, cnt, total_dev, s);
  long long total = 0;
  if (e == cudaSuccess && n_words > 0) e = cudaMemcpyAsync(&total, total_dev, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_clean(cuda_fail(e, "sliced layout pass 1"));
  if (total > (long long)INT32_MAX - 256) return fail_clean(fail(LP_ERR_INVALID, sliced_unsupported_msg));
  if ((st = dalloc(p, &p->sl_col, (size_t)total)) != LP_OK) return fail_clean(st);
  e = build_sliced_pass2(p->row_ptr, p->col, p->sl_q, p->sl_qinv, p->sl_hdr, hm.n_pad, p->sl_col, p->fact_row,
                         hm.n_fact_rows, p->sl_fact_row, p->perm, hm.n_prime, p->sl_perm, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  device_free(cnt);
  cnt = nullptr;
  if (e != cudaSuccess) return fail_clean(cuda_fail(e, "sliced layout pass 2"));
  count_launches(n_words > 0 ? 6 : 0);
  p->sl_entries = total;
  return LP_OK;
}

lp_status block_kernel_fits(lp_program* p, cudaStream_t s, bool* fits) {
  *fits = false;
  if (!sliced_supported(p)) return LP_OK;
  static int optin = -1;
  if (optin < 0) LP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
  // a cheap bound first: the layout holds at least nnz entries
  const long long lower = block_kernel_smem_bytes(p->hm.n_pad / 32, sliced_groups(p->hm.n_pad), p->hm.nnz);
  if (lower + 1024 > (long long)optin) return LP_OK;
  lp_status st = ensure_sliced_layout(p, s);
  if (st != LP_OK) return st;
  *fits = block_kernel_smem_bytes(p->hm.n_pad / 32, sliced_groups(p->hm.n_pad), p->sl_entries) + 1024 <= (long long)optin;
  return LP_OK;
}
const char* const sliced_unsupported_msg = "fixpoint_kernel 2 needs fewer than 2^29 entries (padded below 2^31)";

}  // namespace lp

// What every device handle gets after its matrix is on the device: the iterate vectors, the
// scratch, the default schedule. Frees the handle on failure.
lp_status finish_handle(lp_program* p, cudaStream_t s, std::chrono::steady_clock::time_point t0,
                        std::chrono::steady_clock::time_point t_host, std::chrono::steady_clock::time_point t_upload,
                        lp_program** out) {
  auto cleanup = [&](lp_status code) {
    release(p);
    delete p;
    return code;
  };
  const HostMatrix& hm = p->hm;
  lp_status st;
  // iterate vectors, padded so 16-byte vector loads of a staged prefix stay inside
  if ((st = dalloc(p, &p->x[0], (size_t)hm.n_pad / 32 + 4)) != LP_OK) return cleanup(st);
  if ((st = dalloc(p, &p->x[1], (size_t)hm.n_pad / 32 + 4)) != LP_OK) return cleanup(st);
  if ((st = ensure_scratch(p)) != LP_OK) return cleanup(st);
  // default least-model schedule: the one-block kernel 3 where the program fits one block's
  // shared memory, else the sliced kernel 2 with the vector gathered through L1 (the autotuner's
  // picks on small and on large programs); kernel 0 where the sliced layout's indices overflow
  if (p->sched.fixpoint_kernel == 0 && sliced_supported(p)) {
    bool fits = false;
    if ((st = block_kernel_fits(p, s, &fits)) != LP_OK) return cleanup(st);
    p->sched.fixpoint_kernel = fits ? 3 : 2;
    p->sched.fixpoint_stage = fits ? 0 : 1;
  }
  p->sched.stable_frontier = 2;  // stable models: the frontier over all tiles, from F
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "lp_compile"));
  const auto t_end = std::chrono::steady_clock::now();
  p->compile_ms = std::chrono::duration<double, std::milli>(t_end - t0).count();
  if (std::getenv("LP_COMPILE_TRACE")) {
    auto ms = [](auto a, auto b) { return std::chrono::duration<double, std::milli>(b - a).count(); };
    std::fprintf(stderr, "lp_compile (ms): standardize=%.2f upload=%.2f schedule=%.2f total=%.2f\n", ms(t0, t_host),
                 ms(t_host, t_upload), ms(t_upload, t_end), p->compile_ms);
  }
  *out = p;
  return LP_OK;
}

// lp_compile without LP_COMPILE_ON_HOST: the rules go to the device and are standardized there.
lp_status compile_device_handle(lp_program* p, int32_t n_atoms, int64_t n_rules, const int32_t* head,
                                const int64_t* body_off, const int32_t* body_atom, const uint8_t* body_neg,
                                cudaStream_t s, std::chrono::steady_clock::time_point t0, lp_program** out) {
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice/attribute");
  }
  lp_status st;
  {
    NvtxRange nvtx_dev("lp_compile: standardize on the device");
    st = compile_on_device(p, n_atoms, n_rules, head, body_off, body_atom, body_neg, s);
  }
  if (st != LP_OK) {
    const std::string msg = g_err;  // release() may not touch it, but keep the compile's message
    cudaStreamSynchronize(s);       // the scratch frees are stream-ordered
    release(p);
    delete p;
    return fail(st, msg);
  }
  const auto t = std::chrono::steady_clock::now();
  return finish_handle(p, s, t0, t, t, out);
}

extern "C" {

const char* lp_last_error(void) { return g_err.c_str(); }

void lp_debug_fail_alloc(int64_t after) { g_fail_alloc_after.store(after < 0 ? -1 : after); }

int64_t lp_launch_count(void) { return g_launches.load(); }

lp_status lp_compile(int32_t n_atoms, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                     const int32_t* body_atom, const uint8_t* body_neg, uint32_t flags, void* cuda_stream,
                     lp_program** out) {
  NvtxRange nvtx("lp_compile");
  if (!out) return fail(LP_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  if (flags & ~(LP_COMPILE_HOST_ONLY | LP_COMPILE_ON_HOST | LP_COMPILE_ON_DEVICE))
    return fail(LP_ERR_INVALID, "unknown flags");
  if ((flags & LP_COMPILE_ON_DEVICE) && (flags & (LP_COMPILE_HOST_ONLY | LP_COMPILE_ON_HOST)))
    return fail(LP_ERR_INVALID, "LP_COMPILE_ON_DEVICE excludes the host flags");
  auto t0 = std::chrono::steady_clock::now();
  lp_program* p = new (std::nothrow) lp_program();
  if (p) {
    const char* env = std::getenv("LP_FIXPOINT");  // A/B switch for the least-model kernel
    p->sched.fixpoint_kernel = (env && std::strcmp(env, "stream") == 0) ? 1 : 0;
  }
  if (!p) return fail(LP_ERR_OOM, "host allocation failed");
  std::string err;
  lp_status st;
  // rules plus body literals (a malformed body_off is left to the compilers to reject)
  const int64_t size = n_rules > 0 && body_off ? n_rules + body_off[n_rules] : std::max<int64_t>(n_rules, 0);
  const bool small = size >= 0 && size <= kSmallCompile;
  const bool on_host = (flags & (LP_COMPILE_HOST_ONLY | LP_COMPILE_ON_HOST)) != 0 ||
                       (small && !(flags & LP_COMPILE_ON_DEVICE));
  if (!on_host) return compile_device_handle(p, n_atoms, n_rules, head, body_off, body_atom, body_neg,
                                             (cudaStream_t)cuda_stream, t0, out);
  {
    NvtxRange nvtx_host("lp_compile: standardize");
    st = small ? compile_host_serial(n_atoms, n_rules, head, body_off, body_atom, body_neg, p->hm, err)
               : compile_host(n_atoms, n_rules, head, body_off, body_atom, body_neg, p->hm, err);
  }
  if (st != LP_OK) {
    delete p;
    return fail(st, err);
  }
  if (flags & LP_COMPILE_HOST_ONLY) {
    p->host_only = true;
    p->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return LP_OK;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t_host = std::chrono::steady_clock::now();
  auto cleanup = [&](lp_status code) {
    release(p);
    delete p;
    return code;
  };
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGetDevice/attribute"));
  HostMatrix& hm = p->hm;
  if ((st = upload(p, &p->row_ptr, hm.row_ptr, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->col, hm.col, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->any_mask, hm.any_mask, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->perm, hm.perm, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->fact_row, hm.fact_row, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->fact_owner, hm.fact_owner, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->fact_mask, hm.fact_mask, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->neg_row, hm.neg_row, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->bar_row, hm.bar_row, s)) != LP_OK) return cleanup(st);
  if ((st = upload(p, &p->row_tag, hm.row_tag, s)) != LP_OK) return cleanup(st);
  e = cudaStreamSynchronize(s);  // host vectors are pageable and about to be released
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "upload"));
  free_vec(hm.row_ptr);
  free_vec(hm.col);
  free_vec(hm.row_tag);
  p->host_tables = true;
  return finish_handle(p, s, t0, t_host, std::chrono::steady_clock::now(), out);
}

lp_status lp_program_info(const lp_program* p, lp_info* out) {
  if (!p || !out) return fail(LP_ERR_INVALID, "NULL argument");
  const HostMatrix& hm = p->hm;
  out->n_atoms = hm.n;
  out->n_rules = hm.n_rules;
  out->n_prime = hm.n_prime;
  out->nnz = hm.nnz;
  out->n_barred = hm.n_barred;
  out->n_aux = hm.n_aux;
  out->k = hm.k;
  out->n_fact_rows = hm.n_fact_rows;
  out->n_and_rows = hm.n_rule_rows;
  out->n_or_rows = hm.n_or_rows;
  out->device_bytes = p->device_bytes;
  out->upload_bytes = p->upload_bytes;
  out->compile_ms = p->compile_ms;
  return LP_OK;
}

namespace {

// The frontier schedule's transposed matrix and counters, built on the device on first use.
lp_status ensure_frontier(lp_program* p, cudaStream_t s) {
  if (p->fr_cnt) return LP_OK;
  const HostMatrix& hm = p->hm;
  lp_status st;
  int32_t* cnt = nullptr;
  unsigned* counters = nullptr;
  auto fail_clean = [&](lp_status code) {
    if (cnt) device_free(cnt);
    void* ptrs[] = {p->fr_tptr, p->fr_tidx, p->fr_seed, p->fr_long, counters};
    device_free_all(ptrs, 5);
    p->fr_tptr = p->fr_tidx = p->fr_seed = nullptr;
    p->fr_long = nullptr;
    return code;
  };
  const int32_t n_seed = hm.n_fact_rows + (int32_t)hm.guess_row.size();
  if ((st = dalloc(p, &p->fr_seed, (size_t)n_seed)) != LP_OK) return fail_clean(st);
  if (hm.n_fact_rows > 0 &&
      cudaMemcpyAsync(p->fr_seed, p->fact_row, (size_t)hm.n_fact_rows * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail_clean(cuda_fail(cudaGetLastError(), "frontier seed rows"));
  if (!hm.guess_row.empty() && cudaMemcpyAsync(p->fr_seed + hm.n_fact_rows, hm.guess_row.data(),
                                               hm.guess_row.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail_clean(cuda_fail(cudaGetLastError(), "frontier seed rows"));
  if ((st = dalloc(p, &p->fr_tptr, (size_t)hm.n_pad + 1)) != LP_OK) return fail_clean(st);
  if ((st = dalloc(p, &p->fr_tidx, (size_t)std::max<int64_t>(hm.nnz, 1))) != LP_OK) return fail_clean(st);
  if ((st = dalloc(p, &p->fr_long, (size_t)hm.n_pad / 32 + 1)) != LP_OK) return fail_clean(st);
  if ((st = dalloc(p, &counters, kFrontierCounters)) != LP_OK) return fail_clean(st);
  if (device_malloc((void**)&cnt, ((size_t)hm.n_pad + 1) * 4) != cudaSuccess) {
    cnt = nullptr;
    cudaGetLastError();
    return fail_clean(fail(LP_ERR_OOM, "frontier scratch"));
  }
  cudaError_t e = cudaMemsetAsync(counters, 0, kFrontierCounters * sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, ((size_t)hm.n_pad + 1) * 4, s);
  if (e == cudaSuccess) e = build_transpose(p->row_ptr, p->col, hm.n_pad, p->fr_tptr, p->fr_tidx, cnt, s);
  // counters[kFrontierCounters - 1] (zeroed above, unused by the kernel): whether a row is long
  unsigned any_long = 0;
  if (e == cudaSuccess) e = build_long_rows(p->row_ptr, hm.n_pad, p->fr_long, counters + kFrontierCounters - 1, s);
  if (e == cudaSuccess && hm.n_pad > 0)
    e = cudaMemcpyAsync(&any_long, counters + kFrontierCounters - 1, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  device_free(cnt);
  cnt = nullptr;
  if (e != cudaSuccess) return fail_clean(cuda_fail(e, "frontier transpose"));
  count_launches(hm.n_pad > 0 ? 4 : 0);
  p->fr_nseed = n_seed;
  p->fr_any_long = any_long != 0;
  p->fr_cnt = counters;
  return LP_OK;
}

// Room for wide items (more dependents than the grid-push threshold) per wave of `items`; past it
// the warps push the rest themselves.
int64_t frontier_wide_cap(int64_t items) { return items / 16 + 64; }

// F for the frontier from F (stable_frontier 2): Algorithm 1 on the internal matrix from every
// fact row with every barred row zero (kernel 0; its loop ends when an iteration changes
// nothing, so both iterate vectors hold the fixpoint), kept per handle.
lp_status ensure_frontier_F(lp_program* p, cudaStream_t s) {
  if (p->fr_F) return LP_OK;
  const HostMatrix& hm = p->hm;
  lp_status st = ensure_scratch(p);
  if (st != LP_OK) return st;
  uint32_t* F = nullptr;
  if ((st = dalloc(p, &F, (size_t)hm.n_pad / 32 + 1)) != LP_OK) return st;
  auto fail_clean = [&](lp_status code) {
    device_free(F);
    return code;
  };
  FixArgs a{};
  a.row_ptr = p->row_ptr;
  a.col = p->col;
  a.any_mask = p->any_mask;
  a.x0 = p->x[0];
  a.x1 = p->x[1];
  a.n_words = hm.n_pad / 32;
  a.max_iters = (int32_t)std::min<int64_t>(INT32_MAX, (int64_t)hm.n_prime + 2);
  a.ctl = p->ctl;
  a.fact_row = p->fact_row;
  a.fact_owner = p->fact_owner;
  a.n_facts = hm.n_fact_rows;
  a.fact_mask = p->fact_mask;
  a.n_atom_words = (hm.n + 63) / 64;
  a.n_prime = hm.n_prime;
  a.perm = p->perm;
  a.n_sec_a = hm.n_sec_a;
  static int occ = -1;
  if (occ < 0) occ = fixpoint_blocks_per_sm(1, 1, 0);
  if (occ <= 0) return fail_clean(fail(LP_ERR_CUDA, "fixpoint kernel cannot be resident"));
  const int words_per_block = fix_block(0) / 32;
  const int grid = std::min(max_coresident(p, occ), std::max(1, (a.n_words + words_per_block - 1) / words_per_block));
  cudaError_t e = cudaMemsetAsync(p->ctl, 0, sizeof(DeviceCtl), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->x[0], 0, (size_t)hm.n_pad / 8, s);
  if (e == cudaSuccess) e = launch_fixpoint(a, grid, 1, 1, 0, s);
  if (e == cudaSuccess) count_launches(1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F, p->x[0], (size_t)hm.n_pad / 8, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_clean(cuda_fail(e, "guess-independent fixpoint"));
  if (p->h_ctl->status != 0)
    return fail_clean(fail((lp_status)p->h_ctl->status, "guess-independent fixpoint: the solve did not finish"));
  p->fr_F = F;
  return LP_OK;
}

// Bytes of the frontier buffers for `tiles` tiles of W words: two iterate buffers, a stamp and two
// list slots per item, the changed-item bitmap, a counter per tile, the wide-item list.
int64_t frontier_bytes(int64_t n_pad, int W, int64_t tiles) {
  const int64_t items = tiles * n_pad;
  return 2 * items * W * 8 + items * 4 + 2 * items * 4 + ((items + 31) / 32) * 4 + tiles * 4 +
         frontier_wide_cap(items) * 4 + 64;
}

// The wave buffers for `tiles` tiles of W words; a new allocation voids the rest-state record.
lp_status ensure_frontier_buffers(lp_program* p, int W, int32_t tiles, cudaStream_t s) {
  if (p->fr_buf.p && p->fr_W == W && p->fr_tiles == tiles) return LP_OK;
  const size_t bytes = (size_t)frontier_bytes(p->hm.n_pad, W, tiles);
  if (p->fr_buf.p && p->fr_buf.bytes < bytes) {
    device_free(p->fr_buf.p);
    p->device_bytes -= (int64_t)p->fr_buf.bytes;
    p->fr_buf = DevBuf{};
  }
  lp_status st = ensure(p, p->fr_buf, bytes);
  if (st != LP_OK) return st;
  p->fr_W = W;
  p->fr_tiles = tiles;
  LP_CUDA(cudaMemsetAsync(p->fr_cnt, 0, kFrontierCounters * sizeof(unsigned), s));
  return LP_OK;
}

// The streamed kernel's layout, built on its first use from the device CSR.
lp_status ensure_stream_layout(lp_program* p, cudaStream_t s) {
  if (p->desc) return LP_OK;
  lp_status ht = ensure_host_tables(p, s);  // the layout is built on the host from perm and kinds
  if (ht != LP_OK) return ht;
  HostMatrix& hm = p->hm;
  hm.row_ptr.resize((size_t)hm.n_pad + 1);
  hm.col.resize((size_t)std::max<int64_t>(hm.nnz, 1));
  LP_CUDA(cudaMemcpyAsync(hm.row_ptr.data(), p->row_ptr, hm.row_ptr.size() * 4, cudaMemcpyDeviceToHost, s));
  if (hm.nnz) LP_CUDA(cudaMemcpyAsync(hm.col.data(), p->col, (size_t)hm.nnz * 4, cudaMemcpyDeviceToHost, s));
  LP_CUDA(cudaStreamSynchronize(s));
  std::string err;
  lp_status st = build_stream_layout(hm, err);
  if (st == LP_OK && (st = upload(p, &p->desc, hm.desc, s)) == LP_OK && (st = upload(p, &p->word_hdr, hm.word_hdr, s)) == LP_OK &&
      (st = upload(p, &p->and_col, hm.and_col, s)) == LP_OK && (st = upload(p, &p->groups, hm.groups, s)) == LP_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "upload of the streamed layout");
  } else if (!err.empty()) {
    st = fail(st, err);
  }
  free_vec(hm.row_ptr);
  free_vec(hm.col);
  std::vector<uint32_t>().swap(hm.desc);
  std::vector<int32_t>().swap(hm.word_hdr);
  std::vector<int32_t>().swap(hm.and_col);
  return st;
}

}  // namespace

lp_status lp_least_model(lp_program* p, const uint64_t* init, uint64_t* out, int32_t max_iters, uint32_t flags,
                         int32_t* iters_out, void* cuda_stream) {
  NvtxRange nvtx("lp_least_model");
  if (!p || !out) return fail(LP_ERR_INVALID, "program and out must not be NULL");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  if (max_iters < 1) return fail(LP_ERR_INVALID, "max_iters must be >= 1");
  if (flags & ~(LP_ROWS | LP_TIMING)) return fail(LP_ERR_INVALID, "unknown flags");
  const bool rows = flags & LP_ROWS;
  if (rows && !init) return fail(LP_ERR_INVALID, "LP_ROWS needs an initial vector");
  const HostMatrix& hm = p->hm;
  // From a vector of facts the iterates only grow, so n' + 1 applications always suffice.
  if (!rows) max_iters = (int32_t)std::min<int64_t>(max_iters, (int64_t)hm.n_prime + 2);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  p->last_launches = 0;
  p->timed = flags & LP_TIMING;
  lp_status st = ensure_scratch(p);
  if (st != LP_OK) return st;
  const int32_t n_in = rows ? hm.n_prime : hm.n;
  const size_t in_words = ((size_t)n_in + 63) / 64;
  const size_t out_words = in_words;

  if (rows && !p->inv) {
    if ((st = ensure_host_tables(p, s)) != LP_OK) return st;
    std::vector<int32_t> inv(std::max(hm.n_pad, 1), 0);
    for (int32_t c = 0; c < hm.n_prime; c++) inv[hm.perm[c]] = c;
    if ((st = upload(p, &p->inv, inv, s)) != LP_OK) return st;
    LP_CUDA(cudaStreamSynchronize(s));
  }
  const bool host_in = init && !is_device_ptr(init);
  const bool host_out = !is_device_ptr(out);
  const uint64_t* d_init = init;
  uint64_t* d_out = out;
  if (host_in) {
    if ((st = ensure(p, p->stage_in, in_words * 8)) != LP_OK) return st;
    LP_CUDA(cudaMemcpyAsync(p->stage_in.p, init, in_words * 8, cudaMemcpyHostToDevice, s));
    d_init = (const uint64_t*)p->stage_in.p;
  }
  if (host_out) {
    if ((st = ensure(p, p->stage_out, out_words * 8)) != LP_OK) return st;
    d_out = (uint64_t*)p->stage_out.p;
  }

  LP_CUDA(cudaMemsetAsync(p->ctl, 0, sizeof(DeviceCtl), s));
  if (!rows) LP_CUDA(cudaMemsetAsync(p->x[0], 0, (size_t)hm.n_pad / 8, s));

  FixArgs a{};
  a.row_ptr = p->row_ptr;
  a.col = p->col;
  a.any_mask = p->any_mask;
  a.x0 = p->x[0];
  a.x1 = p->x[1];
  a.n_words = hm.n_pad / 32;
  a.max_iters = max_iters;
  a.ctl = p->ctl;
  a.init = rows ? nullptr : d_init;
  a.fact_row = p->fact_row;
  a.fact_owner = p->fact_owner;
  a.n_facts = hm.n_fact_rows;
  a.fact_mask = p->fact_mask;
  a.n_atom_words = (hm.n + 63) / 64;
  a.rows_init = rows ? d_init : nullptr;
  a.inv = p->inv;
  a.n_prime = hm.n_prime;
  a.out = d_out;
  a.perm = p->perm;
  a.n_out = n_in;
  a.n_sec_a = hm.n_sec_a;

  // Kernel and residency from the handle's schedule (both kernels are exact).
  cudaError_t le;
  if (p->sched.fixpoint_kernel == 3) {
    bool fits = false;
    if ((st = block_kernel_fits(p, s, &fits)) != LP_OK) return st;
    if (!fits) return fail(LP_ERR_INVALID, "fixpoint_kernel 3 needs the program's sliced layout to fit in one block's shared memory");
    if (rows) LP_CUDA(cudaMemsetAsync(p->x[0], 0, (size_t)hm.n_pad / 8, s));
    SlicedLayout L{p->sl_hdr, p->sl_col, p->sl_q, p->sl_fact_row, p->sl_perm, sliced_groups(hm.n_pad), p->sl_entries, 0};
    if (p->timed) LP_CUDA(cudaEventRecord(p->ev0, s));
    le = launch_fixpoint_block(a, L, s);
  } else if (p->sched.fixpoint_kernel == 2) {
    if (!sliced_supported(p)) return fail(LP_ERR_INVALID, sliced_unsupported_msg);
    if ((st = ensure_sliced_layout(p, s)) != LP_OK) return st;
    static int optin = -1;
    if (optin < 0) LP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    // leave the rest of the unified L1/shared array to L1 (the OR rows' vector words);
    // LP_SLICED_STAGE_BYTES lowers the cap (tests of the unstaged fallback)
    int cap = kSlicedStageBytesMax;
    if (const char* env = std::getenv("LP_SLICED_STAGE_BYTES")) cap = std::min(cap, std::max(0, std::atoi(env)));
    const int max_stage_words = std::max(0, std::min(optin - 1024, cap)) / 16 * 4;
    const int32_t need = (std::min(hm.n_sec_a, hm.n_pad) + 127) / 128 * 4;  // whole 16-byte units
    const bool stage = p->sched.fixpoint_stage == 0 && need > 0 && need <= max_stage_words;
    const int32_t stage_words = stage ? need : 0;
    static std::map<std::pair<int, int>, int> occ_cache;  // (stage, staged words) -> CTAs per SM
    static std::mutex occ_mu;
    int occ_c;
    {
      std::lock_guard<std::mutex> lock(occ_mu);
      auto key = std::make_pair((int)stage, (int)stage_words);
      auto f = occ_cache.find(key);
      occ_c = f != occ_cache.end() ? f->second : (occ_cache[key] = fixpoint_sliced_blocks_per_sm(stage, stage_words));
    }
    if (occ_c <= 0) return fail(LP_ERR_CUDA, "sliced fixpoint kernel cannot be resident");
    const int32_t n_groups = sliced_groups(hm.n_pad);
    SlicedLayout L{p->sl_hdr, p->sl_col, p->sl_q, p->sl_fact_row, p->sl_perm, n_groups, p->sl_entries, stage_words};
    if (rows) LP_CUDA(cudaMemsetAsync(p->x[0], 0, (size_t)hm.n_pad / 8, s));  // v0 is built with atomics
    const int grid = std::min(max_coresident(p, occ_c), std::max(1, (n_groups + kSlicedBlock / 32 - 1) / (kSlicedBlock / 32)));
    if (p->timed) LP_CUDA(cudaEventRecord(p->ev0, s));
    le = launch_fixpoint_sliced(a, L, stage, grid, s);
  } else if (p->sched.fixpoint_kernel == 1) {
    if ((st = ensure_stream_layout(p, s)) != LP_OK) return st;
    static int occ_s = -1;
    if (occ_s < 0) occ_s = fixpoint_stream_blocks_per_sm();
    if (occ_s <= 0) return fail(LP_ERR_CUDA, "streamed fixpoint kernel cannot be resident");
    const int per_sm_s = p->sched.fixpoint_blocks_per_sm > 0 ? std::min(occ_s, p->sched.fixpoint_blocks_per_sm) : occ_s;
    StreamLayout L{p->desc, p->word_hdr, p->and_col, p->groups, hm.n_groups, hm.n_sec_a, hm.groups.data()};
    int grid = std::max(1, std::min(max_coresident(p, per_sm_s), hm.n_groups));
    if (p->timed) LP_CUDA(cudaEventRecord(p->ev0, s));
    le = launch_fixpoint_stream(a, L, grid, s);
  } else {
    const int split = std::max(1, p->sched.fixpoint_row_split);
    const int xn = p->sched.fixpoint_chunk_batch == 4 ? 4 : 1;
    const int map = p->sched.fixpoint_row_map;
    static int occ_by_variant[4][2][9];
    static bool occ_init = false;
    if (!occ_init) {
      for (auto& m : occ_by_variant)
        for (auto& x : m)
          for (int& v : x) v = -1;
      occ_init = true;
    }
    int& occ = occ_by_variant[map][xn == 4][split];
    if (occ < 0) occ = fixpoint_blocks_per_sm(split, xn, map);
    if (occ <= 0) return fail(LP_ERR_CUDA, "fixpoint kernel cannot be resident");
    const int per_sm = p->sched.fixpoint_blocks_per_sm > 0 ? std::min(occ, p->sched.fixpoint_blocks_per_sm) : occ;
    const int words_per_block = fix_block(map) / 32 / split;
    int grid = std::min(max_coresident(p, per_sm), std::max(1, (a.n_words + words_per_block - 1) / words_per_block));
    if (p->timed) LP_CUDA(cudaEventRecord(p->ev0, s));
    le = launch_fixpoint(a, grid, split, xn, map, s);
  }
  if ((st = launch_count_and_check(le, "launch fixpoint kernel", p)) != LP_OK) return st;
  if (p->timed) LP_CUDA(cudaEventRecord(p->ev1, s));
  LP_CUDA(cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s));
  if (host_out) LP_CUDA(cudaMemcpyAsync(out, d_out, out_words * 8, cudaMemcpyDeviceToHost, s));
  if (iters_out || host_out || host_in) {
    st = finish_sync(p, s);
    if (iters_out) *iters_out = p->h_ctl->iters;
    return st;
  }
  return LP_OK;
}

lp_status lp_stable_models(lp_program* p, const uint64_t* guesses, int64_t n_guesses, uint64_t* stable_mask,
                           uint64_t* models, int64_t max_models, int64_t* n_stable_out, int32_t max_iters,
                           void* cuda_stream) {
  NvtxRange nvtx("lp_stable_models");
  if (!p) return fail(LP_ERR_INVALID, "program must not be NULL");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  if (max_iters < 1) return fail(LP_ERR_INVALID, "max_iters must be >= 1");
  if (n_guesses < 0 || max_models < 0) return fail(LP_ERR_INVALID, "negative count");
  const HostMatrix& hm = p->hm;
  if (guesses) {
    if (hm.k > 64) return fail(LP_ERR_TOO_MANY_GUESSES, "k > 64 guessed atoms do not fit a guess word");
  } else {
    if (hm.k > 40) return fail(LP_ERR_TOO_MANY_GUESSES, "enumerating all 2^k guesses needs k <= 40");
    if (n_guesses != (int64_t(1) << hm.k)) return fail(LP_ERR_INVALID, "n_guesses must be 2^k when guesses is NULL");
  }
  if (n_guesses > 0 && !stable_mask) return fail(LP_ERR_INVALID, "stable_mask must not be NULL");
  if (max_models > 0 && !models) return fail(LP_ERR_INVALID, "models must not be NULL when max_models > 0");
  // M_0 holds only self-loop rows (facts, barred atoms), so every column's iterates grow.
  max_iters = (int32_t)std::min<int64_t>(max_iters, (int64_t)hm.n_prime + 2);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  p->last_launches = 0;
  p->timed = false;
  lp_status st = ensure_scratch(p);
  if (st != LP_OK) return st;
  if (n_guesses == 0) {
    LP_CUDA(cudaMemsetAsync(p->ctl, 0, sizeof(DeviceCtl), s));
    LP_CUDA(cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s));
    if (n_stable_out) {
      LP_CUDA(cudaStreamSynchronize(s));
      *n_stable_out = 0;
    }
    return LP_OK;
  }
  const int64_t n_gwords = (n_guesses + 63) / 64;
  const int32_t atom_words = (hm.n + 63) / 64;
  // tile width: largest power of two <= 32 words whose two iterate buffers fit the budget
  // (wider tiles mean fewer tile iterations and grid barriers; 1 GiB covers 32-word tiles for
  // programs up to ~2M rows)
  int64_t budget = 1ll << 30;
  if (const char* env = std::getenv("LP_TILE_BYTES")) budget = std::max<int64_t>(1, std::atoll(env));
  int log2W = 0;
  if (p->sched.stable_tile_words > 0) {  // the schedule's width, capped at the guesses' words
    while ((1 << log2W) < p->sched.stable_tile_words && (int64_t(1) << log2W) < n_gwords) log2W++;
  } else {
    while (log2W < 5 && (int64_t(1) << (log2W + 1)) <= n_gwords &&
           2ll * hm.n_pad * 8 * (int64_t(1) << (log2W + 1)) <= budget)
      log2W++;
  }
  const int W = 1 << log2W;
  const int64_t n_tiles = (n_gwords + W - 1) / W;
  const bool split = p->sched.stable_row_split == 1;
  const bool frontier = p->sched.stable_frontier >= 1 && !split;
  const bool from_F = frontier && p->sched.stable_frontier == 2;
  int32_t wave_tiles = 0;
  if (frontier) {
    // tiles in flight at once: as many as the budget holds (8 GiB by default), item ids in int32
    int64_t fr_budget = 8ll << 30;
    if (const char* env = std::getenv("LP_FRONTIER_BYTES")) fr_budget = std::max<int64_t>(1, std::atoll(env));
    int64_t c = std::min<int64_t>(n_tiles, fr_budget / frontier_bytes(hm.n_pad, W, 1));
    c = std::min<int64_t>(c, (int64_t)(INT32_MAX - 64) / std::max<int64_t>(hm.n_pad, 1));
    wave_tiles = (int32_t)std::max<int64_t>(c, 1);
    if ((st = ensure_frontier(p, s)) != LP_OK) return st;
    if (from_F && (st = ensure_frontier_F(p, s)) != LP_OK) return st;
    // a handle keeps the largest wave it has run unless a wider tile needs another layout
    const int32_t keep = p->fr_W == W ? std::max(p->fr_tiles, wave_tiles) : wave_tiles;
    if (frontier_bytes(hm.n_pad, W, keep) <= fr_budget) wave_tiles = keep;
    if ((st = ensure_frontier_buffers(p, W, wave_tiles, s)) != LP_OK) return st;
  } else if ((st = ensure(p, p->tiles, (size_t)2 * hm.n_pad * W * 8)) != LP_OK) {
    return st;
  }
  p->tile_words = W;

  const bool host_g = guesses && !is_device_ptr(guesses);
  const bool host_mask = !is_device_ptr(stable_mask);
  const bool host_models = models && max_models > 0 && !is_device_ptr(models);
  const uint64_t* d_g = guesses;
  uint64_t* d_mask = stable_mask;
  uint64_t* d_models = max_models > 0 ? models : nullptr;
  if (host_g) {
    if ((st = ensure(p, p->stage_in, (size_t)n_guesses * 8)) != LP_OK) return st;
    LP_CUDA(cudaMemcpyAsync(p->stage_in.p, guesses, (size_t)n_guesses * 8, cudaMemcpyHostToDevice, s));
    d_g = (const uint64_t*)p->stage_in.p;
  }
  if (host_mask) {
    if ((st = ensure(p, p->stage_out, (size_t)n_gwords * 8)) != LP_OK) return st;
    d_mask = (uint64_t*)p->stage_out.p;
  }
  if (host_models) {
    if ((st = ensure(p, p->stage_out2, (size_t)max_models * atom_words * 8)) != LP_OK) return st;
    d_models = (uint64_t*)p->stage_out2.p;
  }
  LP_CUDA(cudaMemsetAsync(p->ctl, 0, sizeof(DeviceCtl), s));

  StableArgs a{};
  a.row_ptr = p->row_ptr;
  a.col = p->col;
  a.any_mask = p->any_mask;
  a.row_tag = p->row_tag;
  a.n_pad = hm.n_pad;
  a.W = W;
  a.log2W = log2W;
  a.n_guesses = n_guesses;
  a.n_gwords = n_gwords;
  a.n_tiles = n_tiles;
  a.guesses = d_g;
  a.k = hm.k;
  a.neg_row = p->neg_row;
  a.bar_row = p->bar_row;
  a.n_barred = hm.n_barred;
  a.perm = p->perm;
  a.n = hm.n;
  a.stable_mask = d_mask;
  a.models = d_models;
  a.max_models = max_models;
  a.n_atom_words = atom_words;
  a.max_iters = max_iters;
  a.ctl = p->ctl;
  int grid = 0;
  if (frontier) {
    const int64_t items = (int64_t)wave_tiles * hm.n_pad;
    char* b = (char*)p->fr_buf.p;
    a.X0 = (uint64_t*)b;
    a.X1 = a.X0 + items * W;
    a.mark = (unsigned*)(a.X1 + items * W);
    a.fr_list = (int32_t*)(a.mark + items);
    a.fr_dirty = (unsigned*)(a.fr_list + 2 * items);
    a.fr_last = (int32_t*)(a.fr_dirty + (items + 31) / 32);
    // from F the fact rows and their consequences are already in place: the guessed rows seed
    a.fr_F = from_F ? p->fr_F : nullptr;
    a.guess_rows = p->fr_seed + hm.n_fact_rows;  // the seed list ends with the guessed rows
    a.n_guess_rows = (int32_t)hm.guess_row.size();
    a.fr_seed = from_F ? p->fr_seed + hm.n_fact_rows : p->fr_seed;
    a.n_seed = from_F ? p->fr_nseed - hm.n_fact_rows : p->fr_nseed;
    a.fr_wide = a.fr_last + wave_tiles;
    a.wide_cap = (int32_t)frontier_wide_cap(items);
    if (const char* env = std::getenv("LP_FRONTIER_WIDE_ITEMS"))  // a smaller wide list (tests its overflow)
      a.wide_cap = (int32_t)std::max<int64_t>(0, std::min<int64_t>(a.wide_cap, std::atoll(env)));
    a.long_mask = p->fr_any_long ? p->fr_long : nullptr;
    a.t_ptr = p->fr_tptr;
    a.t_idx = p->fr_tidx;
    a.fr_cnt = p->fr_cnt;
    a.fr_tiles = wave_tiles;
    a.fr_key = 1u | ((unsigned)W << 1) | (from_F ? 0x80u : 0u) | ((unsigned)wave_tiles << 8);
    static int occ_by_w[6] = {-1, -1, -1, -1, -1, -1};
    int& occ_frontier = occ_by_w[log2W];
    if (occ_frontier < 0) occ_frontier = stable_frontier_blocks_per_sm(W);
    if (occ_frontier <= 0) return fail(LP_ERR_CUDA, "stable frontier kernel cannot be resident");
    const int per_sm =
        p->sched.stable_blocks_per_sm > 0 ? std::min(occ_frontier, p->sched.stable_blocks_per_sm) : occ_frontier;
    grid = (int)max_coresident(p, per_sm);
    if ((st = launch_count_and_check(launch_stable_frontier(a, grid, s), "launch stable frontier kernel", p)) != LP_OK)
      return st;
  } else {
    a.X0 = (uint64_t*)p->tiles.p;
    a.X1 = (uint64_t*)p->tiles.p + (size_t)hm.n_pad * W;
    static int occ_by_split[2] = {-1, -1};
    int& occ = occ_by_split[(int)split];
    if (occ < 0) occ = stable_blocks_per_sm(split);
    if (occ <= 0) return fail(LP_ERR_CUDA, "stable kernel cannot be resident");
    const int per_sm = p->sched.stable_blocks_per_sm > 0 ? std::min(occ, p->sched.stable_blocks_per_sm) : occ;
    const int64_t rows_per_block = (int64_t)(kStableBlock / 32) * (32 / W);
    grid = (int)std::min<int64_t>(max_coresident(p, per_sm), std::max<int64_t>(1, hm.n_pad / rows_per_block));
    if ((st = launch_count_and_check(launch_stable(a, grid, split, s), "launch stable kernel", p)) != LP_OK) return st;
  }
  LP_CUDA(cudaMemcpyAsync(p->h_ctl, p->ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s));
  if (host_mask) LP_CUDA(cudaMemcpyAsync(stable_mask, d_mask, (size_t)n_gwords * 8, cudaMemcpyDeviceToHost, s));
  if (host_models) LP_CUDA(cudaMemcpyAsync(models, d_models, (size_t)max_models * atom_words * 8, cudaMemcpyDeviceToHost, s));
  if (n_stable_out || host_g || host_mask || host_models) {
    st = finish_sync(p, s);
    if (n_stable_out) *n_stable_out = p->h_ctl->n_stable;
    return st;
  }
  return LP_OK;
}

lp_status lp_get_schedule(const lp_program* p, lp_schedule* out) {
  if (!p || !out) return fail(LP_ERR_INVALID, "NULL argument");
  *out = p->sched;
  return LP_OK;
}

lp_status lp_set_schedule(lp_program* p, const lp_schedule* in) {
  if (!p || !in) return fail(LP_ERR_INVALID, "NULL argument");
  const int32_t W = in->stable_tile_words;
  if (in->fixpoint_kernel < 0 || in->fixpoint_kernel > 3) return fail(LP_ERR_INVALID, "fixpoint_kernel must be 0, 1, 2 or 3");
  if (in->fixpoint_kernel == 3 && !p->host_only) {
    bool fits = false;
    lp_status st = block_kernel_fits(p, nullptr, &fits);
    if (st != LP_OK) return st;
    if (!fits) return fail(LP_ERR_INVALID, "fixpoint_kernel 3 needs the program's sliced layout to fit in one block's shared memory");
  }
  if (in->fixpoint_stage != 0 && in->fixpoint_stage != 1) return fail(LP_ERR_INVALID, "fixpoint_stage must be 0 or 1");
  if (in->fixpoint_kernel == 2 && !sliced_supported(p)) return fail(LP_ERR_INVALID, sliced_unsupported_msg);
  if (in->fixpoint_blocks_per_sm < 0 || in->stable_blocks_per_sm < 0)
    return fail(LP_ERR_INVALID, "blocks per SM must be >= 0");
  const int32_t G = in->fixpoint_row_split;
  if (G != 0 && G != 1 && G != 2 && G != 4 && G != 8)
    return fail(LP_ERR_INVALID, "fixpoint_row_split must be 0, 1, 2, 4 or 8");
  if (G > 1 && in->fixpoint_kernel != 0) return fail(LP_ERR_INVALID, "a row split needs fixpoint_kernel 0");
  const int32_t X = in->fixpoint_chunk_batch;
  if (X != 0 && X != 1 && X != 4) return fail(LP_ERR_INVALID, "fixpoint_chunk_batch must be 0, 1 or 4");
  if (X == 4 && in->fixpoint_kernel != 0) return fail(LP_ERR_INVALID, "a chunk batch needs fixpoint_kernel 0");
  const int32_t R = in->fixpoint_row_map;
  if (R < 0 || R > 3) return fail(LP_ERR_INVALID, "fixpoint_row_map must be 0, 1, 2 or 3");
  if (R > 0 && (in->fixpoint_kernel != 0 || G > 1 || X == 4))
    return fail(LP_ERR_INVALID, "a thread-per-row map needs fixpoint_kernel 0, no row split and no chunk batch");
  if (in->stable_row_split != 0 && in->stable_row_split != 1) return fail(LP_ERR_INVALID, "stable_row_split must be 0 or 1");
  if (in->stable_frontier < 0 || in->stable_frontier > 2) return fail(LP_ERR_INVALID, "stable_frontier must be 0, 1 or 2");
  if (in->stable_frontier >= 1 && in->stable_row_split == 1)
    return fail(LP_ERR_INVALID, "the frontier schedule needs stable_row_split 0");
  if (W < 0 || W > 32 || (W & (W - 1)) != 0) return fail(LP_ERR_INVALID, "stable_tile_words must be 0 or 1, 2, 4, 8, 16, 32");
  p->sched = *in;
  return LP_OK;
}

lp_status lp_last_solve_stats(lp_program* p, lp_solve_stats* out, void* cuda_stream) {
  if (!p || !out) return fail(LP_ERR_INVALID, "NULL argument");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  lp_status st = ensure_scratch(p);
  if (st != LP_OK) return st;
  LP_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  out->iters = p->h_ctl->iters;
  out->status = p->h_ctl->status;
  out->kernel_ms = -1.0f;
  if (p->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev0, p->ev1) == cudaSuccess) out->kernel_ms = ms;
    else cudaGetLastError();
  }
  out->launches = p->last_launches;
  out->tiles = p->h_ctl->tiles;
  out->tile_words = p->tile_words;
  out->max_tile_iters = p->h_ctl->max_tile_iters;
  out->sum_tile_iters = p->h_ctl->sum_tile_iters;
  out->frontier_rows = (int64_t)p->h_ctl->fr_rows;
  out->frontier_entries = (int64_t)p->h_ctl->fr_entries;
  out->frontier_list = (int64_t)p->h_ctl->fr_list;
  out->frontier_deps = (int64_t)p->h_ctl->fr_deps;
  return LP_OK;
}

lp_status lp_export_matrix(const lp_program* p, int64_t* row_ptr, int64_t* col, int32_t* threshold, int8_t* kind,
                           void* cuda_stream) {
  if (!p || !row_ptr || !col || !threshold) return fail(LP_ERR_INVALID, "NULL argument");
  const HostMatrix& hm = p->hm;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  lp_status st = ensure_host_tables(const_cast<lp_program*>(p), s);
  if (st != LP_OK) return st;
  std::vector<int32_t> rp, cl;
  if (p->host_only) {
    rp.assign(hm.row_ptr.begin(), hm.row_ptr.end());
    cl.assign(hm.col.begin(), hm.col.end());
    cl.resize(std::max<int64_t>(hm.nnz, 1));
  } else {
    rp.resize((size_t)hm.n_pad + 1);
    cl.resize(std::max<int64_t>(hm.nnz, 1));
    LP_CUDA(cudaMemcpyAsync(rp.data(), p->row_ptr, rp.size() * 4, cudaMemcpyDeviceToHost, s));
    if (hm.nnz) LP_CUDA(cudaMemcpyAsync(cl.data(), p->col, (size_t)hm.nnz * 4, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> inv(std::max(hm.n_prime, 1));
  for (int32_t c = 0; c < hm.n_prime; c++) inv[hm.perm[c]] = c;
  row_ptr[0] = 0;
  for (int32_t c = 0; c < hm.n_prime; c++) {
    const int32_t r = hm.perm[c];
    const int64_t b = row_ptr[c];
    int64_t m = 0;
    for (int32_t e = rp[r]; e < rp[r + 1]; e++) col[b + m++] = inv[cl[e]];
    std::sort(col + b, col + b + m);
    row_ptr[c + 1] = b + m;
    const int8_t kd = hm.canon_kind[c];
    threshold[c] = kd == K_RULE ? (int32_t)m : (kd == K_EMPTY ? 0 : 1);
    if (kind) kind[c] = kd;
  }
  return LP_OK;
}

void lp_free(lp_program* p) {
  if (!p) return;
  release(p);
  delete p;
}

}  // extern "C"

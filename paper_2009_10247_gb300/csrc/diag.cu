// diag.cu -- diagnostics (include/lp.h): lp_check_grid_barrier runs the bounded grid barrier
// that every persistent kernel of liblp uses alone, so that its failure path (a block that
// never arrives) can be exercised without faulting or hanging the GPU; lp_check_matrix checks
// the invariants of a compiled matrix on the device (the kernels rely on them and do not
// re-check them per access).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <string>

#include "device.cuh"
#include "program.h"

namespace lp {

constexpr int kDiagBlock = 128;

// Blocks [0, absent) return at once, like a rank that left; the others meet at one barrier.
__global__ void __launch_bounds__(kDiagBlock) barrier_check_kernel(DeviceCtl* ctl, int absent,
                                                                   unsigned long long limit_ns) {
  if ((int)blockIdx.x < absent) return;
  if (!grid_barrier(ctl, 1, LP_ERR_TIMEOUT, limit_ns)) return;
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) ctl->iters = 1;  // passed the barrier
}

}  // namespace lp

using namespace lp;

extern "C" lp_status lp_check_grid_barrier(int32_t blocks, int32_t absent, int32_t limit_us, int32_t* status_out,
                                           float* ms_out, void* cuda_stream) {
  if (blocks < 1 || absent < 0 || absent > blocks || limit_us < 1 || limit_us > 2000000 || !status_out)
    return fail(LP_ERR_INVALID, "bad arguments");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_check_kernel, kDiagBlock, 0);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (blocks > per_sm * sms) return fail(LP_ERR_INVALID, "more blocks than can be co-resident");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DeviceCtl* ctl = nullptr;
  DeviceCtl h{};
  if ((e = cudaMalloc((void**)&ctl, sizeof(DeviceCtl))) != cudaSuccess) return fail(LP_ERR_OOM, "cudaMalloc");
  cudaEvent_t a = nullptr, b = nullptr;
  lp_status st = LP_OK;
  if ((e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&b)) == cudaSuccess &&
      (e = cudaMemsetAsync(ctl, 0, sizeof(DeviceCtl), s)) == cudaSuccess &&
      (e = cudaEventRecord(a, s)) == cudaSuccess) {
    unsigned long long limit_ns = 1000ull * (unsigned long long)limit_us;
    int ab = absent;
    void* params[] = {&ctl, &ab, &limit_ns};
    e = cudaLaunchCooperativeKernel((const void*)barrier_check_kernel, dim3(blocks), dim3(kDiagBlock), params, 0, s);
    if (e == cudaSuccess) {
      count_launches(1);
      if ((e = cudaEventRecord(b, s)) == cudaSuccess &&
          (e = cudaMemcpyAsync(&h, ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s)) == cudaSuccess)
        e = cudaStreamSynchronize(s);
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    st = fail(LP_ERR_CUDA, cudaGetErrorString(e));
  } else {
    *status_out = h.status != 0 ? h.status : (h.iters == 1 ? LP_OK : LP_ERR_CUDA);
    if (ms_out) cudaEventElapsedTime(ms_out, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(ctl);
  return st;
}

namespace lp {

// Invariants of a compiled matrix: row_ptr starts at 0, never decreases and ends at nnz;
// every column is a row of the matrix; every fact row is a self-loop (one entry, its own row).
__global__ void matrix_check_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                    int32_t n_pad, int64_t nnz, const int32_t* __restrict__ fact_row,
                                    int32_t n_facts, unsigned long long* bad) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long b = 0;
  if (tid == 0) b += (row_ptr[0] != 0) + ((long long)row_ptr[n_pad] != nnz);
  for (long long r = tid; r < n_pad; r += nth) b += row_ptr[r + 1] < row_ptr[r];
  for (long long e = tid; e < nnz; e += nth) b += (unsigned)col[e] >= (unsigned)n_pad;
  for (long long f = tid; f < n_facts; f += nth) {
    const int32_t r = fact_row[f];
    const bool ok = r >= 0 && r < n_pad && row_ptr[r + 1] - row_ptr[r] == 1 && col[row_ptr[r]] == r;
    b += !ok;
  }
  if (b) atomicAdd(bad, b);
}

}  // namespace lp

extern "C" lp_status lp_check_matrix(const lp_program* p, int64_t* n_bad, void* cuda_stream) {
  if (!p || !n_bad) return fail(LP_ERR_INVALID, "NULL argument");
  const HostMatrix& hm = p->hm;
  if (p->host_only) {  // the host copy is kept: check it on the host
    int64_t bad = (hm.row_ptr.empty() || hm.row_ptr[0] != 0) + ((int64_t)hm.row_ptr.back() != hm.nnz);
    for (int32_t r = 0; r < hm.n_pad; r++) bad += hm.row_ptr[r + 1] < hm.row_ptr[r];
    for (int64_t e = 0; e < hm.nnz; e++) bad += (unsigned)hm.col[e] >= (unsigned)hm.n_pad;
    for (int32_t r : hm.fact_row)
      bad += !(r >= 0 && r < hm.n_pad && hm.row_ptr[r + 1] - hm.row_ptr[r] == 1 && hm.col[hm.row_ptr[r]] == r);
    *n_bad = bad;
    return LP_OK;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned long long* d_bad = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_bad, sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(LP_ERR_OOM, "cudaMalloc");
  unsigned long long h_bad = 0;
  if ((e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), s)) == cudaSuccess) {
    const int blocks = (int)std::min<long long>(1024, std::max<long long>(1, (hm.nnz + 255) / 256));
    matrix_check_kernel<<<blocks, 256, 0, s>>>(p->row_ptr, p->col, hm.n_pad, hm.nnz, p->fact_row, hm.n_fact_rows,
                                                d_bad);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      count_launches(1);
      if ((e = cudaMemcpyAsync(&h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s)) == cudaSuccess)
        e = cudaStreamSynchronize(s);
    }
  }
  cudaFree(d_bad);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, cudaGetErrorString(e));
  *n_bad = (int64_t)h_bad;
  return LP_OK;
}

extern "C" lp_status lp_debug_internal(const lp_program* p, int32_t which, void* out, int64_t* bytes,
                                       void* cuda_stream) {
  if (!p || !bytes) return fail(LP_ERR_INVALID, "NULL argument");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  const HostMatrix& hm = p->hm;
  const void* src = nullptr;
  int64_t size = 0;
  switch (which) {
    case 0: src = p->row_ptr; size = 4 * ((int64_t)hm.n_pad + 1); break;
    case 1: src = p->col; size = 4 * hm.nnz; break;
    case 2: src = p->perm; size = 4 * (int64_t)hm.n_prime; break;
    case 3: src = p->any_mask; size = 4 * ((int64_t)hm.n_pad / 32); break;
    case 4: src = p->row_tag; size = 4 * (int64_t)hm.n_pad; break;
    case 5: src = p->fact_row; size = 4 * (int64_t)hm.n_fact_rows; break;
    case 6: src = p->fact_owner; size = 4 * (int64_t)hm.n_fact_rows; break;
    case 7: src = p->fact_mask; size = 8 * (((int64_t)hm.n + 63) / 64); break;
    case 8: src = p->neg_row; size = 4 * (int64_t)hm.n_barred; break;
    case 9: src = p->bar_row; size = 4 * (int64_t)hm.n_barred; break;
    default: return fail(LP_ERR_INVALID, "unknown internal array");
  }
  *bytes = size;
  if (!out || size == 0) return LP_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaMemcpyAsync(out, src, (size_t)size, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, cudaGetErrorString(e));
  return LP_OK;
}

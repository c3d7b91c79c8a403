// diag.cu -- lp_check_grid_barrier (include/lp.h): the bounded grid barrier that every
// persistent kernel of liblp uses, run alone, so that its failure path (a block that never
// arrives) can be exercised without faulting or hanging the GPU.
#include <cuda_runtime.h>

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

// fixpoint_block.cu -- Algorithm 1 for small programs in one thread block (kernel 3 of the
// least-model schedule).
//
// A small program's solve is bound by latency, not bandwidth: its whole matrix is a few tens of
// kilobytes, and every theta application of a multi-block persistent kernel pays a grid-wide
// barrier through global memory (microseconds). Here one block of 1024 threads copies the CSR
// (row pointers, column ids, OR-row mask) into shared memory once, keeps both iterate vectors
// there, and meets at a block barrier per iteration, so the loop touches global memory only to
// load the matrix, read the initial facts and write the projected fixpoint.
//
// theta(M_P v) per 32-row word, one warp per word as in kernel 0: the word's entries are walked
// 32 at a time, each lane gathers one entry's bit from the shared vector, a ballot makes the
// chunk's mask, and each lane counts the bits of its own row's entries; the row fires when the
// count reaches its threshold (all m body atoms of a rule row, one entry of an OR row or a
// self-loop) -- theta of Def. 5 in exact integers.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace lp {

namespace {

// Shared-memory layout (32-bit words): row_ptr (n_pad + 1), col (nnz), OR-row mask, x0, x1;
// every part padded to a multiple of 4 words.
struct BlockLayout {
  int rp, col, any, x0, x1, total;
};

__host__ __device__ inline int pad4(long long n) { return (int)((n + 3) & ~3ll); }

__host__ __device__ inline BlockLayout block_layout(int n_words, long long nnz) {
  BlockLayout L;
  L.rp = 0;
  L.col = L.rp + pad4(32ll * n_words + 1);
  L.any = L.col + pad4(nnz);
  L.x0 = L.any + pad4(n_words);
  L.x1 = L.x0 + pad4(n_words);
  L.total = L.x1 + pad4(n_words);
  return L;
}

__device__ __forceinline__ uint32_t block_theta_word(const int* s_rp, const int* s_col, const uint32_t* s_any,
                                                     const uint32_t* src, int w, int lane) {
  const int r = (w << 5) + lane;
  const int beg = s_rp[r], end = s_rp[r + 1];
  const int base = __shfl_sync(FULL, beg, 0), stop = __shfl_sync(FULL, end, 31);
  int cnt = 0;
  for (int c = base; c < stop; c += 32) {
    const int e = c + lane;
    uint32_t bit = 0u;
    if (e < stop) {
      const int j = s_col[e];
      bit = (src[j >> 5] >> (j & 31)) & 1u;
    }
    const uint32_t m = __ballot_sync(FULL, bit);
    const int lo = max(beg - c, 0), hi = min(end - c, 32);
    if (hi > lo) cnt += __popc(m & ((hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo)));
  }
  const bool any = (s_any[w] >> lane) & 1u;
  return __ballot_sync(FULL, cnt >= (any ? 1 : max(end - beg, 1)));  // an empty row never fires
}

__global__ void __launch_bounds__(kBlockThreads, 1) fixpoint_block_kernel(FixArgs a, long long nnz) {
  extern __shared__ uint4 s_raw[];
  __shared__ int s_bad;
  uint32_t* sm = reinterpret_cast<uint32_t*>(s_raw);
  const BlockLayout L = block_layout(a.n_words, nnz);
  int* s_rp = reinterpret_cast<int*>(sm + L.rp);
  int* s_col = reinterpret_cast<int*>(sm + L.col);
  uint32_t* s_any = sm + L.any;
  uint32_t* const s_x0 = sm + L.x0;
  uint32_t* const s_x1 = sm + L.x1;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
  const int n_rp = 32 * a.n_words + 1;

  // ---- the matrix into shared memory; x0 = 0
  for (int i = t; i < n_rp; i += blockDim.x) s_rp[i] = __ldg(a.row_ptr + i);
  for (long long i = t; i < nnz; i += blockDim.x) s_col[i] = __ldg(a.col + i);
  for (int i = t; i < a.n_words; i += blockDim.x) {
    s_any[i] = __ldg(a.any_mask + i);
    s_x0[i] = 0u;
  }
  if (t == 0) s_bad = 0;
  __syncthreads();

  // ---- initial vector v0 (Def. 4, or the caller's row vector in LP_ROWS mode)
  if (a.rows_init) {
    for (int w = warp; w < a.n_words; w += nwarp) {
      const int r = (w << 5) + lane;
      uint32_t bit = 0u;
      if (r < a.n_prime) {
        const int c = a.inv[r];
        bit = (uint32_t)(a.rows_init[c >> 6] >> (c & 63)) & 1u;
      }
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) s_x0[w] = word;
    }
  } else {
    for (int i = t; i < a.n_facts; i += blockDim.x) {
      const int own = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own >> 6] >> (own & 63)) & 1ull) : true;
      if (sel) atomicOr(&s_x0[a.fact_row[i] >> 5], 1u << (a.fact_row[i] & 31));
    }
    if (a.init)
      for (int i = t; i < a.n_atom_words; i += blockDim.x)
        if (a.init[i] & ~a.fact_mask[i]) s_bad = 1;
  }
  __syncthreads();
  if (s_bad) {
    if (t == 0) atomicCAS(&a.ctl->status, 0, 1 /* LP_ERR_INVALID */);
    return;
  }

  // ---- Algorithm 1 loop, one block barrier per theta application
  int it = 0;
  const uint32_t* fin = s_x0;
  bool converged = false;
  for (; it < a.max_iters; ++it) {
    const uint32_t* src = (it & 1) ? s_x1 : s_x0;
    uint32_t* dst = (it & 1) ? s_x0 : s_x1;
    bool changed = false;
    for (int w = warp; w < a.n_words; w += nwarp) {
      const uint32_t u = block_theta_word(s_rp, s_col, s_any, src, w, lane);
      if (lane == 0) {
        dst[w] = u;
        changed |= u != src[w];
      }
    }
    fin = dst;
    if (!__syncthreads_or(changed)) {
      converged = true;
      ++it;
      break;
    }
  }
  if (t == 0) {
    a.ctl->iters = it;
    if (!converged) atomicCAS(&a.ctl->status, 0, 4 /* LP_ERR_NO_FIXPOINT */);
  }

  // ---- output: bit a of out = fixpoint bit of internal row perm[a]
  if (a.out) {
    const uint32_t* x = fin;
    uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
    const int n32 = 2 * ((a.n_out + 63) >> 6);
    for (int u = warp; u < n32; u += nwarp) {
      const int i = (u << 5) + lane;
      uint32_t bit = 0u;
      if (i < a.n_out) {
        const int r = a.perm[i];
        bit = (x[r >> 5] >> (r & 31)) & 1u;
      }
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) out32[u] = word;
    }
  }
}

}  // namespace

long long block_kernel_smem_bytes(int n_words, long long nnz) { return 4ll * block_layout(n_words, nnz).total; }

cudaError_t launch_fixpoint_block(const FixArgs& a, long long nnz, cudaStream_t s) {
  const long long bytes = block_kernel_smem_bytes(a.n_words, nnz);
  cudaError_t e = set_kernel_smem((const void*)fixpoint_block_kernel, (int)bytes, -1);
  if (e != cudaSuccess) return e;
  fixpoint_block_kernel<<<1, kBlockThreads, (size_t)bytes, s>>>(a, nnz);
  return cudaGetLastError();
}

}  // namespace lp

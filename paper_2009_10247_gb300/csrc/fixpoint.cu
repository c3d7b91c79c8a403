// fixpoint.cu -- Algorithm 1 (matrix computation of the least model) as one persistent kernel.
//
// One launch runs the whole loop: build v0 (Def. 4), then repeat u = theta(M_P v) until u = v
// (Def. 5 thresholding fused in), then write the fixpoint back in the caller's atom order.
// Blocks stay resident (cooperative launch) and meet at a bounded grid barrier once per
// iteration; a rotating device flag records whether any row changed.
//
// theta(M_P v) for one row: the entries of a rule row are 1/m over its m body atoms, so the
// row sum reaches 1 iff all m are true; an OR-rule row or a self-loop has entries 1, so it
// reaches 1 iff one entry is true. The kernel counts true entries and compares the count
// with m (rule rows) or 1 (OR rows): the exact value of theta, with no floating point.
//
// Work mapping: a warp owns one 32-bit output word = 32 consecutive rows. It walks the rows'
// contiguous column range 32 entries at a time with coalesced loads, gathers one bit per
// entry from the bit-packed vector (L1/L2 resident), and a ballot turns the 32 bits into a
// mask; every lane then pops the bits of its own row's sub-range. Row lengths never cause
// divergence; the cost is one gather per stored entry. With a row split G > 1 (programs whose
// words hold thousands of entries), G warps of a block share a word: each counts a contiguous
// share of its chunks and the partial counts meet in shared memory.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace lp {

// u bits of the 32 rows of word w, given the bit vector src.
__device__ __forceinline__ uint32_t theta_word(const int32_t* __restrict__ row_ptr,
                                               const int32_t* __restrict__ col,
                                               const uint32_t* __restrict__ any_mask,
                                               const uint32_t* src, int w, int lane) {
  const int r = (w << 5) + lane;
  const int beg = __ldg(row_ptr + r);
  int end = __shfl_down_sync(FULL, beg, 1);
  if (lane == 31) end = __ldg(row_ptr + r + 1);
  const int base = __shfl_sync(FULL, beg, 0);
  const int stop = __shfl_sync(FULL, end, 31);
  int cnt = 0;
  for (int c = base; c < stop; c += 32) {
    const int e = c + lane;
    uint32_t bit = 0;
    if (e < stop) {
      const int j = __ldg(col + e);
      bit = (src[j >> 5] >> (j & 31)) & 1u;
    }
    const uint32_t m = __ballot_sync(FULL, bit);
    const int lo = max(beg - c, 0), hi = min(end - c, 32);
    if (hi > lo) {
      const uint32_t sel = (hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo);
      cnt += __popc(m & sel);
    }
  }
  const int len = end - beg;
  const bool any = (__ldg(any_mask + w) >> lane) & 1u;
  const int thr = any ? 1 : max(len, 1);  // an empty row never fires
  return __ballot_sync(FULL, cnt >= thr);
}

// Row split (G > 1 warps per word, for long rows): part `part` of G counts the true entries of
// every row of word w within its share of the word's 32-entry chunks; the G partial counts are
// summed in shared memory before the threshold. Returns this lane's partial count; *len_out is
// the lane's row length.
__device__ __forceinline__ int theta_word_part(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                               const uint32_t* src, int w, int lane, int part, int G,
                                               int* len_out) {
  const int r = (w << 5) + lane;
  const int beg = __ldg(row_ptr + r);
  int end = __shfl_down_sync(FULL, beg, 1);
  if (lane == 31) end = __ldg(row_ptr + r + 1);
  const int base = __shfl_sync(FULL, beg, 0);
  const int stop = __shfl_sync(FULL, end, 31);
  const int n_chunks = (stop - base + 31) >> 5;
  const int c_lo = base + 32 * (n_chunks * part / G), c_hi = min(stop, base + 32 * (n_chunks * (part + 1) / G));
  int cnt = 0;
  for (int c = c_lo; c < c_hi; c += 32) {
    const int e = c + lane;
    uint32_t bit = 0;
    if (e < c_hi) {
      const int j = __ldg(col + e);
      bit = (src[j >> 5] >> (j & 31)) & 1u;
    }
    const uint32_t m = __ballot_sync(FULL, bit);
    const int lo = max(beg - c, 0), hi = min(end - c, 32);
    if (hi > lo) {
      const uint32_t sel = (hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo);
      cnt += __popc(m & sel);
    }
  }
  *len_out = end - beg;
  return cnt;
}

__device__ __forceinline__ uint32_t get_bit(const uint32_t* v, int i) { return (v[i >> 5] >> (i & 31)) & 1u; }

template <int G>
__global__ void __launch_bounds__(kFixBlock) fixpoint_kernel(FixArgs a) {
  __shared__ int s_flag;
  __shared__ int s_cnt[G > 1 ? kFixBlock : 1];
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;

  // ---- initial vector v0
  if (a.rows_init) {
    // LP_ROWS: internal row r takes bit inv[r] of the caller's canonical vector.
    for (int w = gwarp; w < a.n_words; w += nwarps) {
      const int r = (w << 5) + lane;
      uint32_t bit = 0;
      if (r < a.n_prime) {
        const int c = a.inv[r];
        bit = (uint32_t)(a.rows_init[c >> 6] >> (c & 63)) & 1u;
      }
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) a.x0[w] = word;
    }
  } else {
    // Def. 4: a fact row is 1 (when its atom is selected); x0 was zeroed by the caller.
    for (int i = gtid; i < a.n_facts; i += nthreads) {
      const int own = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own >> 6] >> (own & 63)) & 1ull) : true;
      if (sel) atomicOr(a.x0 + (a.fact_row[i] >> 5), 1u << (a.fact_row[i] & 31));
    }
    if (a.init)
      for (int i = gtid; i < a.n_atom_words; i += nthreads)
        if (a.init[i] & ~a.fact_mask[i]) atomicCAS(&ctl->status, 0, 1 /* LP_ERR_INVALID */);
  }
  if (!grid_barrier(ctl, ++round, 6)) return;
  if (ld_volatile((const unsigned*)&ctl->status) != 0) return;

  // ---- Algorithm 1 loop
  const uint32_t* fin = a.x0;
  int it = 0;
  bool converged = false;
  for (; it < a.max_iters; ++it) {
    const uint32_t* src = (it & 1) ? a.x1 : a.x0;
    uint32_t* dst = (it & 1) ? a.x0 : a.x1;
    bool changed = false;
    if (G == 1) {
      for (int w = gwarp; w < a.n_words; w += nwarps) {
        const uint32_t u = theta_word(a.row_ptr, a.col, a.any_mask, src, w, lane);
        if (lane == 0) {
          dst[w] = u;
          changed |= (u != src[w]);
        }
      }
    } else {
      // kFixBlock / 32 / G words per block and round; the loop bound is uniform in the block
      const int warp = threadIdx.x >> 5, slot = warp / G, part = warp % G;
      const int per_block = (kFixBlock / 32) / G;
      for (int wb = blockIdx.x * per_block; wb < a.n_words; wb += gridDim.x * per_block) {
        const int w = wb + slot;
        int len = 0, cnt = 0;
        if (w < a.n_words) cnt = theta_word_part(a.row_ptr, a.col, src, w, lane, part, G, &len);
        s_cnt[threadIdx.x] = cnt;
        __syncthreads();
        if (part == 0 && w < a.n_words) {
          int total = 0;
#pragma unroll
          for (int q = 0; q < G; q++) total += s_cnt[threadIdx.x + 32 * q];
          const bool any = (__ldg(a.any_mask + w) >> lane) & 1u;
          const uint32_t u = __ballot_sync(FULL, total >= (any ? 1 : max(len, 1)));
          if (lane == 0) {
            dst[w] = u;
            changed |= (u != src[w]);
          }
        }
        __syncthreads();
      }
    }
    const int any_changed = __syncthreads_or(changed);
    if (threadIdx.x == 0) {
      if (any_changed) atomicOr(&ctl->flag[it % 3], 1u);
      if (blockIdx.x == 0) ctl->flag[(it + 1) % 3] = 0u;  // nobody reads or writes it now
    }
    if (!grid_barrier(ctl, ++round, 6)) return;
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
    if (!converged) atomicCAS(&ctl->status, 0, 4 /* LP_ERR_NO_FIXPOINT */);
  }

  // ---- output: bit a = fixpoint bit of internal row perm[a]
  if (a.out) {
    uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
    const int n32 = 2 * ((a.n_out + 63) >> 6);
    for (int u = gwarp; u < n32; u += nwarps) {
      const int i = (u << 5) + lane;
      const uint32_t bit = i < a.n_out ? get_bit(fin, a.perm[i]) : 0u;
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) out32[u] = word;
    }
  }
}

static const void* fixpoint_entry(int G) {
  switch (G) {
    case 2: return (const void*)fixpoint_kernel<2>;
    case 4: return (const void*)fixpoint_kernel<4>;
    case 8: return (const void*)fixpoint_kernel<8>;
    default: return (const void*)fixpoint_kernel<1>;
  }
}

cudaError_t launch_fixpoint(const FixArgs& a, int grid, int row_split, cudaStream_t s) {
  FixArgs copy = a;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(fixpoint_entry(row_split), dim3(grid), dim3(kFixBlock), params, 0, s);
}

int fixpoint_blocks_per_sm(int row_split) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fixpoint_entry(row_split), kFixBlock, 0) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace lp

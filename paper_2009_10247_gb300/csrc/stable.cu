// stable.cu -- Algorithms 2 and 3 (stable models of a normal program) over batches of guesses.
//
// The initial matrix M_0 of Def. 8 has one column per guess. Columns are packed 64 to a
// 64-bit word, so a row of the iterate holds the row's truth value under 64 guesses, and a
// tile of W words (64W guesses) is iterated as one bit-packed sparse matrix x multi-vector
// product: for a rule row the new word is the AND of the words of its body atoms (all m
// entries 1/m true), for an OR-rule row or a self-loop the OR (one entry true) -- theta of
// Def. 5 applied to M_P M_k exactly, for 64 columns per instruction.
//
// One persistent cooperative launch walks the tiles. Per tile:
//   1. M_0 words (Def. 8): fact rows all ones; guessed barred rows carry bit j of each guess
//      (for the full enumeration, a fixed pattern for j < 6 and the guess-word index bits
//      above); every other row zero;
//   2. M_{k+1} = theta(M_P M_k) until no word changes (per-tile early exit). The columns only
//      gain true bits from one iterate to the next (theta is monotone and M_1 >= M_0), so the
//      number of true bits of the tile decides it, and a row's old words are never read;
//   3. Algorithm 3: a column is stable iff a_q XOR a_q-bar = 1 for every negated atom q, so the
//      stable bits of a word are the AND over q of (word of q) XOR (word of q-bar);
//   4. the stable columns of the tile are numbered in guess order and their models (the
//      column over the original atoms) are written out.
// The iterate buffers of a tile are sized by the host to stay L2 resident.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"
#include "stable_common.cuh"

namespace lp {

// SPLIT: a warp takes one row at a time and its 32 / W lane groups split the row's entries
// (each group one word per lane), combining their partial AND / OR with shuffles; for long rows
// (dense programs) this replaces one lane walking a whole row. With W = 32 both are the same.
template <bool SPLIT>
__global__ void __launch_bounds__(kStableBlock) stable_kernel(StableArgs a) {
  __shared__ unsigned long long s_cnt;
  __shared__ long long s_base;
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;
  const int W = a.W;
  const int rows_per_warp = 32 >> a.log2W;  // W <= 32 lanes per row
  const int sub = lane >> a.log2W;          // row within the warp's group
  const int wl = lane & (W - 1);            // word within the tile
  const int n_groups = a.n_pad / rows_per_warp;
  const long long tile_words = (long long)a.n_pad * W;

  for (long long t = 0; t < a.n_tiles; ++t) {
    const long long gw0 = t * W;  // first guess word of the tile
    // The previous tile's readers of the change flags are all past its last barrier.
    if (threadIdx.x == 0) s_cnt = 0ull;
    __syncthreads();
    // ---- 1. M_0
    unsigned cnt0 = 0;
    for (long long e = gtid; e < tile_words; e += nthreads) {
      const int row = (int)(e >> a.log2W);
      const int w = (int)(e & (W - 1));
      const uint64_t m0 = m0_word(__ldg(a.row_tag + row), gw0 + w, a);
      a.X0[e] = m0;
      cnt0 += __popcll(m0);
    }
    cnt0 = __reduce_add_sync(FULL, cnt0);
    if (lane == 0 && cnt0) atomicAdd(&s_cnt, (unsigned long long)cnt0);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_cnt) atomicAdd(&ctl->init_count, s_cnt);
      s_cnt = 0ull;
    }
    if (!grid_barrier(ctl, ++round, 6)) return;
    unsigned long long prev_count = ld_volatile64(&ctl->init_count);

    // ---- 2. M_{k+1} = theta(M_P M_k) until unchanged
    const uint64_t* fin = a.X0;
    int it = 0;
    bool converged = false;
    for (; it < a.max_iters; ++it) {
      const uint64_t* src = (it & 1) ? a.X1 : a.X0;
      uint64_t* dst = (it & 1) ? a.X0 : a.X1;
      unsigned cnt = 0;  // true bits this thread wrote
      if (SPLIT) {
        const int S = 32 >> a.log2W;  // entry slots per warp
        const int slot = lane >> a.log2W;
        for (int row = gwarp; row < a.n_pad; row += nwarps) {
          const int beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
          const bool any = (__ldg(a.any_mask + (row >> 5)) >> (row & 31)) & 1u;
          const uint64_t ident = any ? 0ull : ~0ull;
          uint64_t acc = ident;
          for (int e = beg + slot; e < end; e += 4 * S) {
            int cc[4];
#pragma unroll
            for (int j = 0; j < 4; j++) cc[j] = e + j * S < end ? __ldg(a.col + e + j * S) : -1;
            uint64_t vv[4];
#pragma unroll
            for (int j = 0; j < 4; j++) vv[j] = cc[j] >= 0 ? src[((long long)cc[j] << a.log2W) + wl] : ident;
            acc = any ? (acc | vv[0] | vv[1] | vv[2] | vv[3]) : (acc & vv[0] & vv[1] & vv[2] & vv[3]);
          }
          for (int o = W; o < 32; o <<= 1) {  // combine the slots (lanes with the same word)
            const uint64_t other = __shfl_xor_sync(FULL, acc, o);
            acc = any ? (acc | other) : (acc & other);
          }
          if (end == beg) acc = 0ull;  // an empty row never fires
          if (slot == 0) {
            const long long o = ((long long)row << a.log2W) + wl;
            cnt += __popcll(acc);
            dst[o] = acc;
          }
        }
      } else
      for (int g = gwarp; g < n_groups; g += nwarps) {
        const int row = g * rows_per_warp + sub;
        const int beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
        const bool any = (__ldg(a.any_mask + (row >> 5)) >> (row & 31)) & 1u;
        const uint64_t ident = any ? 0ull : ~0ull;
        uint64_t acc = (end > beg) ? ident : 0ull;
        const long long o = ((long long)row << a.log2W) + wl;
        // four entries per step: their column loads, then their gathers, so that a row costs
        // two dependent memory latencies per four body atoms
        for (int e = beg; e < end; e += 4) {
          int cc[4];
#pragma unroll
          for (int j = 0; j < 4; j++) cc[j] = e + j < end ? __ldg(a.col + e + j) : -1;
          uint64_t vv[4];
#pragma unroll
          for (int j = 0; j < 4; j++) vv[j] = cc[j] >= 0 ? src[((long long)cc[j] << a.log2W) + wl] : ident;
          const uint64_t orv = vv[0] | vv[1] | vv[2] | vv[3], andv = vv[0] & vv[1] & vv[2] & vv[3];
          acc = any ? (acc | orv) : (acc & andv);
        }
        cnt += __popcll(acc);
        dst[o] = acc;
      }
      // the iterates only grow (Def. 8 columns under a monotone theta), so the same number of
      // true bits means the same iterate
      cnt = __reduce_add_sync(FULL, cnt);
      if (lane == 0 && cnt) atomicAdd(&s_cnt, (unsigned long long)cnt);
      __syncthreads();
      if (threadIdx.x == 0) {
        if (s_cnt) atomicAdd(&ctl->count[it % 3], s_cnt);
        s_cnt = 0ull;
        if (blockIdx.x == 0) ctl->count[(it + 1) % 3] = 0ull;  // nobody reads or adds to it now
      }
      if (!grid_barrier(ctl, ++round, 6)) return;
      const unsigned long long now = ld_volatile64(&ctl->count[it % 3]);
      const bool again = now != prev_count;
      prev_count = now;
      fin = dst;
      if (!again) {
        converged = true;
        ++it;
        break;
      }
    }
    if (!converged) {
      if (gtid == 0) {
        ctl->iters = it;
        atomicCAS(&ctl->status, 0, 4 /* LP_ERR_NO_FIXPOINT */);
      }
      return;  // every block takes this branch: the count it read is the same for all
    }

    // ---- 3. Algorithm 3 on the W words of the tile
    if (gtid < W) {
      const long long gw = gw0 + gtid;
      if (gw < a.n_gwords) {
        const long long rem = a.n_guesses - gw * 64;
        uint64_t st = rem >= 64 ? ~0ull : ((1ull << rem) - 1ull);
        for (int j = 0; j < a.n_barred; j++)
          st &= fin[((long long)a.neg_row[j] << a.log2W) + gtid] ^ fin[((long long)a.bar_row[j] << a.log2W) + gtid];
        a.stable_mask[gw] = st;
      }
    }
    if (gtid == 0) {
      ctl->iters = it;
      ctl->max_tile_iters = max(ctl->max_tile_iters, it);
      ctl->sum_tile_iters += it;
      ctl->tiles = t + 1;
    }
    if (!grid_barrier(ctl, ++round, 6)) return;

    // ---- 4. models of the stable columns, numbered in guess order
    if (threadIdx.x == 0) s_base = *reinterpret_cast<volatile long long*>(&ctl->n_stable);
    __syncthreads();
    const long long base = s_base;
    // words of this tile: lane w holds popc(stable word w) (W <= 32)
    const long long gwl = gw0 + lane;
    const uint64_t myword = (lane < W && gwl < a.n_gwords) ? a.stable_mask[gwl] : 0ull;
    const int mycnt = __popcll(myword);
    int incl = mycnt;  // inclusive prefix over lanes
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += v;
    }
    const int tile_count = __shfl_sync(FULL, incl, 31);
    if (a.models) {
      for (int m = gwarp; m < tile_count && base + m < a.max_models; m += nwarps) {
        // word holding the m-th stable column, and its bit
        const unsigned ballot = __ballot_sync(FULL, incl > m);
        const int wsel = __ffs(ballot) - 1;
        const int before = __shfl_sync(FULL, incl - mycnt, wsel);
        uint64_t word = __shfl_sync(FULL, myword, wsel);
        for (int q = 0; q < m - before; q++) word &= word - 1;  // drop lower set bits
        const int b = __ffsll((long long)word) - 1;
        uint32_t* dst = reinterpret_cast<uint32_t*>(a.models + (base + m) * a.n_atom_words);
        const int n32 = 2 * a.n_atom_words;
        for (int u = 0; u < n32; u++) {
          const int atom = (u << 5) + lane;
          uint32_t bit = 0;
          if (atom < a.n) bit = (uint32_t)(fin[((long long)a.perm[atom] << a.log2W) + wsel] >> b) & 1u;
          const uint32_t word32 = __ballot_sync(FULL, bit);
          if (lane == 0) dst[u] = word32;
        }
      }
    }
    if (gtid == 0) {  // every block is past this tile's convergence checks
      ctl->init_count = 0ull;
      ctl->count[0] = ctl->count[1] = ctl->count[2] = 0ull;
    }
    if (!grid_barrier(ctl, ++round, 6)) return;
    if (gtid == 0) ctl->n_stable = base + tile_count;  // everyone read base before the barrier
  }
}

namespace {
const void* stable_entry(bool row_split) {
  return row_split ? (const void*)stable_kernel<true> : (const void*)stable_kernel<false>;
}

// Transposed matrix: per column the rows that refer to it (order within a column is arbitrary).
__global__ void transpose_count_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                       int32_t n_pad, int32_t* __restrict__ cnt) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_pad) return;
  for (int e = row_ptr[r]; e < row_ptr[r + 1]; e++) atomicAdd(cnt + col[e], 1);
}

constexpr int kScanThreads = 1024;
// Exclusive prefix sum of cnt[0 .. n) into out[0 .. n] (one block); cnt is then reset to out.
__global__ void __launch_bounds__(kScanThreads) transpose_scan_kernel(int32_t* __restrict__ cnt, int32_t n,
                                                                     int32_t* __restrict__ out) {
  __shared__ long long s_sum[kScanThreads];
  const int t = threadIdx.x;
  const int per = (n + kScanThreads - 1) / kScanThreads;
  const int lo = min(n, t * per), hi = min(n, lo + per);
  long long sum = 0;
  for (int i = lo; i < hi; i++) sum += cnt[i];
  s_sum[t] = sum;
  __syncthreads();
  for (int d = 1; d < kScanThreads; d <<= 1) {
    const long long v = t >= d ? s_sum[t - d] : 0;
    __syncthreads();
    s_sum[t] += v;
    __syncthreads();
  }
  long long run = s_sum[t] - sum;
  for (int i = lo; i < hi; i++) {
    const int c = cnt[i];
    out[i] = (int)run;
    cnt[i] = (int)run;
    run += c;
  }
  if (t == kScanThreads - 1) out[n] = (int)s_sum[t];
}

__global__ void transpose_fill_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                      int32_t n_pad, int32_t* __restrict__ cursor, int32_t* __restrict__ t_idx) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_pad) return;
  for (int e = row_ptr[r]; e < row_ptr[r + 1]; e++) t_idx[atomicAdd(cursor + col[e], 1)] = r;
}
}  // namespace

cudaError_t build_transpose(const int32_t* row_ptr, const int32_t* col, int32_t n_pad, int32_t* t_ptr, int32_t* t_idx,
                            int32_t* cnt, cudaStream_t s) {
  if (n_pad <= 0) return cudaSuccess;
  const int threads = 256, blocks = (n_pad + threads - 1) / threads;
  transpose_count_kernel<<<blocks, threads, 0, s>>>(row_ptr, col, n_pad, cnt);
  transpose_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, n_pad, t_ptr);
  transpose_fill_kernel<<<blocks, threads, 0, s>>>(row_ptr, col, n_pad, cnt, t_idx);
  return cudaGetLastError();
}

cudaError_t launch_stable(const StableArgs& a, int grid, bool row_split, cudaStream_t s) {
  StableArgs copy = a;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(stable_entry(row_split), dim3(grid), dim3(kStableBlock), params, 0, s);
}

int stable_blocks_per_sm(bool row_split) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stable_entry(row_split), kStableBlock, 0) !=
      cudaSuccess)
    return 0;
  return nb;
}

}  // namespace lp

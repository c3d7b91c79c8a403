// fixpoint_block.cu -- Algorithm 1 for small programs in one thread block (kernel 3 of the
// least-model schedule).
//
// A small program's solve is bound by latency, not bandwidth: its whole matrix is a few tens of
// kilobytes, and every theta application of a multi-block persistent kernel pays a grid-wide
// barrier through global memory (about 1.5 microseconds). Here one block of 1024 threads copies
// the sliced layout of kernel 2 (fixpoint_sliced.cu: rows renumbered by length, 128-row groups
// stored column-major at their width, a row's entries reduced as one AND with an XOR mask for OR
// rows) into shared memory once, keeps both iterate vectors there, and meets at a block barrier
// per iteration, so the loop touches global memory only to load the layout, read the initial
// facts and write the projected fixpoint. Warps take groups round-robin (the groups are
// ordered by width, so each warp gets a similar mix; a shared work counter cost one more block
// barrier and an atomic per iteration).
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace lp {

namespace {

constexpr int kGroupRows = 128;
constexpr uint32_t kStagedFlag = 0x80000000u;

// Shared-memory layout, in 16-byte units: x0 and x1 (n_pad / 32 words each, rounded up to whole
// units), the group headers (3 units per group), the entries.
struct BlockLayout {
  int x0, x1, hdr, col, total;
};

__host__ __device__ inline BlockLayout block_layout(int n_words, int n_groups, long long entries) {
  BlockLayout L;
  const int xu = (n_words + 3) / 4;
  L.x0 = 0;
  L.x1 = xu;
  L.hdr = 2 * xu;
  L.col = L.hdr + 3 * n_groups;
  L.total = L.col + (int)((entries + 3) / 4);
  return L;
}

__device__ __forceinline__ uint32_t rot(uint32_t x, int j) { return __funnelshift_r(x, x, (uint32_t)j); }

__global__ void __launch_bounds__(kBlockThreads, 1) fixpoint_block_kernel(FixArgs a, SlicedLayout S) {
  extern __shared__ int4 s_raw[];
  __shared__ int s_bad;
  const BlockLayout B = block_layout(a.n_words, S.n_groups, S.total_entries);
  uint32_t* const s_x0 = reinterpret_cast<uint32_t*>(s_raw + B.x0);
  uint32_t* const s_x1 = reinterpret_cast<uint32_t*>(s_raw + B.x1);
  int4* const s_hdr = s_raw + B.hdr;
  int4* const s_col = s_raw + B.col;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;

  // ---- the layout into shared memory; x0 = 0
  for (int i = t; i < 3 * S.n_groups; i += blockDim.x) s_hdr[i] = __ldg(S.hdr + i);
  const int4* gcol = reinterpret_cast<const int4*>(S.col);
  for (int i = t; i < (int)(S.total_entries / 4); i += blockDim.x) s_col[i] = __ldg(gcol + i);
  for (int i = t; i < a.n_words; i += blockDim.x) s_x0[i] = 0u;
  if (t == 0) s_bad = 0;
  __syncthreads();

  // ---- initial vector v0 in the new numbering (Def. 4, or the caller's row vector)
  if (a.rows_init) {
    for (int r = t; r < a.n_prime; r += blockDim.x) {
      const int c = a.inv[r];
      if ((a.rows_init[c >> 6] >> (c & 63)) & 1ull) {
        const int q = S.q[r];
        atomicOr(&s_x0[q >> 5], 1u << (q & 31));
      }
    }
  } else {
    for (int i = t; i < a.n_facts; i += blockDim.x) {
      const int own = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own >> 6] >> (own & 63)) & 1ull) : true;
      if (sel) atomicOr(&s_x0[S.fact_row[i] >> 5], 1u << (S.fact_row[i] & 31));
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
    // warp w takes groups w, w + nwarp, ...
    bool changed = false;
    int g = warp;
    while (g < S.n_groups) {  // uniform in the warp
      const int4 h0 = s_hdr[3 * g], h1 = s_hdr[3 * g + 1], h2 = s_hdr[3 * g + 2];
      const int K = h0.y & ~(int)kStagedFlag;
      const uint32_t inv0 = ((uint32_t)h1.x >> lane) & 1u ? FULL : 0u, inv1 = ((uint32_t)h1.y >> lane) & 1u ? FULL : 0u;
      const uint32_t inv2 = ((uint32_t)h1.z >> lane) & 1u ? FULL : 0u, inv3 = ((uint32_t)h1.w >> lane) & 1u ? FULL : 0u;
      uint32_t a0 = FULL, a1 = FULL, a2 = FULL, a3 = FULL;
      const int4* e = s_col + h0.x / 4 + lane;
#pragma unroll 4  // the entries' loads of four steps in flight at once
      for (int k = 0; k < K; k++) {
        const int4 c = e[32 * k];
        a0 &= rot(src[c.x >> 5], c.x) ^ inv0;
        a1 &= rot(src[c.y >> 5], c.y) ^ inv1;
        a2 &= rot(src[c.z >> 5], c.z) ^ inv2;
        a3 &= rot(src[c.w >> 5], c.w) ^ inv3;
      }
      const uint32_t u0 = __ballot_sync(FULL, ((a0 ^ inv0) & ~((uint32_t)h2.x >> lane)) & 1u);
      const uint32_t u1 = __ballot_sync(FULL, ((a1 ^ inv1) & ~((uint32_t)h2.y >> lane)) & 1u);
      const uint32_t u2 = __ballot_sync(FULL, ((a2 ^ inv2) & ~((uint32_t)h2.z >> lane)) & 1u);
      const uint32_t u3 = __ballot_sync(FULL, ((a3 ^ inv3) & ~((uint32_t)h2.w >> lane)) & 1u);
      const int w0 = g * (kGroupRows / 32);
      if (lane < 4 && w0 + lane < a.n_words) {
        const uint32_t word = lane == 0 ? u0 : lane == 1 ? u1 : lane == 2 ? u2 : u3;
        changed |= word != src[w0 + lane];
        dst[w0 + lane] = word;
      }
      g += nwarp;
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

  // ---- output: bit a of out = fixpoint bit of row q[perm[a]]
  if (a.out) {
    uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
    const int n32 = 2 * ((a.n_out + 63) >> 6);
    for (int u = warp; u < n32; u += nwarp) {
      const int i = (u << 5) + lane;
      uint32_t bit = 0u;
      if (i < a.n_out) {
        const int r = S.perm[i];
        bit = (fin[r >> 5] >> (r & 31)) & 1u;
      }
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) out32[u] = word;
    }
  }
}

}  // namespace

long long block_kernel_smem_bytes(int n_words, int n_groups, long long entries) {
  return 16ll * block_layout(n_words, n_groups, entries).total;
}

cudaError_t launch_fixpoint_block(const FixArgs& a, const SlicedLayout& S, cudaStream_t s) {
  const long long bytes = block_kernel_smem_bytes(a.n_words, S.n_groups, S.total_entries);
  cudaError_t e = set_kernel_smem((const void*)fixpoint_block_kernel, (int)bytes, -1);
  if (e != cudaSuccess) return e;
  fixpoint_block_kernel<<<1, kBlockThreads, (size_t)bytes, s>>>(a, S);
  return cudaGetLastError();
}

}  // namespace lp

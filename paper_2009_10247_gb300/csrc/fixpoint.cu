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
// mask; each lane then counts its own row's bits. Row lengths never cause divergence; the
// cost is one gather per stored entry. A warp takes two words per step (their loads overlap)
// and counts a word's rows from a prefix sum of its chunk ballots (prefix_count). With a row
// split G > 1 (programs whose words hold thousands of entries), G warps of a block share a
// word: each counts a contiguous share of its chunks and the partial counts meet in shared
// memory. That is row map 0. Row maps 1-3 give each lane one row of the word instead (a thread
// per row; see theta_pair_rows below), which suits programs whose rows hold a few entries.
#include <cuda_runtime.h>

#include "device.cuh"
#include "fixpoint_phases.cuh"
#include "kernels.h"

namespace lp {

// True entries of this lane's row [beg, end) among the word's entries [c_lo, c_hi), walked 32
// at a time (XN chunks per step: all their column loads, then all their gathers, then the
// ballots, which shortens the dependent-load chain of words with many chunks).
template <int XN>
__device__ __forceinline__ int count_chunks(const int32_t* __restrict__ col, const uint32_t* src, int beg, int end,
                                            int c_lo, int c_hi, int lane) {
  int cnt = 0;
  for (int c0 = c_lo; c0 < c_hi; c0 += 32 * XN) {
    int j[XN];
#pragma unroll
    for (int q = 0; q < XN; q++) {
      const int e = c0 + 32 * q + lane;
      j[q] = e < c_hi ? __ldg(col + e) : -1;
    }
    uint32_t bit[XN];
#pragma unroll
    for (int q = 0; q < XN; q++) bit[q] = j[q] >= 0 ? (src[j[q] >> 5] >> (j[q] & 31)) & 1u : 0u;
#pragma unroll
    for (int q = 0; q < XN; q++) {
      const int c = c0 + 32 * q;
      const uint32_t m = __ballot_sync(FULL, bit[q]);
      const int lo = max(beg - c, 0), hi = min(end - c, 32);
      if (hi > lo) {
        const uint32_t sel = (hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo);
        cnt += __popc(m & sel);
      }
    }
  }
  return cnt;
}

// u bits of the 32 rows of word w, given the bit vector src.
template <int XN>
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
  const int cnt = count_chunks<XN>(col, src, beg, end, base, stop, lane);
  const int len = end - beg;
  const bool any = (__ldg(any_mask + w) >> lane) & 1u;
  const int thr = any ? 1 : max(len, 1);  // an empty row never fires
  return __ballot_sync(FULL, cnt >= thr);
}

// Row split (G > 1 warps per word, for long rows): part `part` of G counts the true entries of
// every row of word w within its share of the word's 32-entry chunks; the G partial counts are
// summed in shared memory before the threshold. Returns this lane's partial count; *len_out is
// the lane's row length.
template <int XN>
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
  *len_out = end - beg;
  return count_chunks<XN>(col, src, beg, end, c_lo, c_hi, lane);
}

// Count of this lane's row [beg, end) from a word's per-chunk ballots (word of at most 32
// chunks): lane q holds the ballot of chunk q. An exclusive warp scan of their popcounts gives
// P(x), the true entries before offset x of the word's entry range; the row's count is
// P(end) - P(beg) (offsets relative to the word's first entry).
__device__ __forceinline__ int prefix_count(uint32_t mine, int lane, int xb, int xe) {
  const int pc = __popc(mine);
  int incl = pc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += t;
  }
  const int excl = incl - pc;
  const int qb = xb >> 5, qe = xe >> 5;  // chunk of each offset (32 = just past chunk 31)
  const int qb2 = qb > 31 ? 31 : qb, qe2 = qe > 31 ? 31 : qe;
  const uint32_t lb = qb > 31 ? FULL : ((1u << (xb & 31)) - 1u), le = qe > 31 ? FULL : ((1u << (xe & 31)) - 1u);
  const int pb = __shfl_sync(FULL, excl, qb2) + __popc(__shfl_sync(FULL, mine, qb2) & lb);
  const int pe = __shfl_sync(FULL, excl, qe2) + __popc(__shfl_sync(FULL, mine, qe2) & le);
  return pe - pb;
}

// Two words per warp step (w1, w2): their loads interleave, so each warp keeps twice the
// memory requests in flight. Words of at most 32 chunks use prefix_count; longer ones the
// chunk-by-chunk count.
template <int XN>
__device__ __forceinline__ void theta_word_pair(const FixArgs& a, const uint32_t* src, int w1, int w2, int lane,
                                                uint32_t* u1, uint32_t* u2) {
  const int r1 = (w1 << 5) + lane, r2 = (w2 << 5) + lane;
  const int b1 = __ldg(a.row_ptr + r1), b2 = __ldg(a.row_ptr + r2);
  int e1 = __shfl_down_sync(FULL, b1, 1), e2 = __shfl_down_sync(FULL, b2, 1);
  if (lane == 31) {
    e1 = __ldg(a.row_ptr + r1 + 1);
    e2 = __ldg(a.row_ptr + r2 + 1);
  }
  const int s1 = __shfl_sync(FULL, b1, 0), t1 = __shfl_sync(FULL, e1, 31);
  const int s2 = __shfl_sync(FULL, b2, 0), t2 = __shfl_sync(FULL, e2, 31);
  const int n1 = (t1 - s1 + 31) >> 5, n2 = (t2 - s2 + 31) >> 5;
  int c1, c2;
  if (n1 <= 32 && n2 <= 32) {
    uint32_t m1 = 0, m2 = 0;
    const int nmax = max(n1, n2);
    for (int q = 0; q < nmax; q++) {
      const int ea = s1 + 32 * q + lane, eb = s2 + 32 * q + lane;
      const int ja = ea < t1 ? __ldg(a.col + ea) : -1, jb = eb < t2 ? __ldg(a.col + eb) : -1;
      const uint32_t ba = ja >= 0 ? (src[ja >> 5] >> (ja & 31)) & 1u : 0u;
      const uint32_t bb = jb >= 0 ? (src[jb >> 5] >> (jb & 31)) & 1u : 0u;
      const uint32_t ma = __ballot_sync(FULL, ba), mb = __ballot_sync(FULL, bb);
      if (lane == q) {
        m1 = ma;
        m2 = mb;
      }
    }
    c1 = prefix_count(m1, lane, b1 - s1, e1 - s1);
    c2 = prefix_count(m2, lane, b2 - s2, e2 - s2);
  } else {
    c1 = count_chunks<XN>(a.col, src, b1, e1, s1, t1, lane);
    c2 = count_chunks<XN>(a.col, src, b2, e2, s2, t2, lane);
  }
  const bool any1 = (__ldg(a.any_mask + w1) >> lane) & 1u, any2 = (__ldg(a.any_mask + w2) >> lane) & 1u;
  *u1 = __ballot_sync(FULL, c1 >= (any1 ? 1 : max(e1 - b1, 1)));  // an empty row never fires
  *u2 = __ballot_sync(FULL, c2 >= (any2 ? 1 : max(e2 - b2, 1)));
}

// ---- Thread-per-row maps (row maps 1-3). Lane l owns row 32w + l of word w and walks its own
// entries: U column ids are loaded together, then their U bits are gathered, so a row of at
// most U entries costs one dependent load pair; longer rows continue U at a time. No ballot or
// scan per chunk, so a short-row program issues fewer instructions per word than the chunked
// map, at the price of lanes idling on the word's longest row.

// Two words per warp step (w1, w2), their loads interleaved.
template <int U>
__device__ __forceinline__ void theta_pair_rows(const FixArgs& a, const uint32_t* src, int w1, int w2, int lane,
                                                uint32_t* u1, uint32_t* u2) {
  const int r1 = (w1 << 5) + lane, r2 = (w2 << 5) + lane;
  const int b1 = __ldg(a.row_ptr + r1), b2 = __ldg(a.row_ptr + r2);
  int e1 = __shfl_down_sync(FULL, b1, 1), e2 = __shfl_down_sync(FULL, b2, 1);
  if (lane == 31) {
    e1 = __ldg(a.row_ptr + r1 + 1);
    e2 = __ldg(a.row_ptr + r2 + 1);
  }
  const int l1 = e1 - b1, l2 = e2 - b2;
  const int lm = max(l1, l2);
  int c1 = 0, c2 = 0;
  for (int q = 0; q < lm; q += U) {
    int j1[U], j2[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      j1[k] = q + k < l1 ? __ldg(a.col + b1 + q + k) : -1;
      j2[k] = q + k < l2 ? __ldg(a.col + b2 + q + k) : -1;
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      c1 += j1[k] >= 0 ? (src[j1[k] >> 5] >> (j1[k] & 31)) & 1 : 0;
      c2 += j2[k] >= 0 ? (src[j2[k] >> 5] >> (j2[k] & 31)) & 1 : 0;
    }
  }
  const bool any1 = (__ldg(a.any_mask + w1) >> lane) & 1u, any2 = (__ldg(a.any_mask + w2) >> lane) & 1u;
  *u1 = __ballot_sync(FULL, c1 >= (any1 ? 1 : max(l1, 1)));  // an empty row never fires
  *u2 = __ballot_sync(FULL, c2 >= (any2 ? 1 : max(l2, 1)));
}

// NW words per warp step (w0 + q * stride, q < NW).
template <int NW, int U>
__device__ __forceinline__ void theta_words_rows(const FixArgs& a, const uint32_t* src, int w0, int stride, int lane,
                                                 uint32_t* u) {
  int b[NW], l[NW];
#pragma unroll
  for (int q = 0; q < NW; q++) b[q] = __ldg(a.row_ptr + ((w0 + q * stride) << 5) + lane);
  int lm = 0;
#pragma unroll
  for (int q = 0; q < NW; q++) {
    int e = __shfl_down_sync(FULL, b[q], 1);
    if (lane == 31) e = __ldg(a.row_ptr + ((w0 + q * stride) << 5) + 32);
    l[q] = e - b[q];
    lm = max(lm, l[q]);
  }
  int c[NW];
#pragma unroll
  for (int q = 0; q < NW; q++) c[q] = 0;
  for (int k0 = 0; k0 < lm; k0 += U) {
    int j[NW][U];
#pragma unroll
    for (int q = 0; q < NW; q++)
#pragma unroll
      for (int k = 0; k < U; k++) j[q][k] = k0 + k < l[q] ? __ldg(a.col + b[q] + k0 + k) : -1;
#pragma unroll
    for (int q = 0; q < NW; q++)
#pragma unroll
      for (int k = 0; k < U; k++) c[q] += j[q][k] >= 0 ? (src[j[q][k] >> 5] >> (j[q][k] & 31)) & 1 : 0;
  }
#pragma unroll
  for (int q = 0; q < NW; q++) {
    const bool any = (__ldg(a.any_mask + w0 + q * stride) >> lane) & 1u;
    u[q] = __ballot_sync(FULL, c[q] >= (any ? 1 : max(l[q], 1)));
  }
}

// Row bounds of word w for the pipelined map: this lane's row begin, lane 31's row end, and
// the word's OR-row mask (zeros past the last word).
__device__ __forceinline__ void word_bounds(const FixArgs& a, int w, int lane, int* b, int* e31, uint32_t* anyw) {
  if (w < a.n_words) {
    const int r = (w << 5) + lane;
    *b = __ldg(a.row_ptr + r);
    *e31 = lane == 31 ? __ldg(a.row_ptr + r + 1) : 0;
    *anyw = __ldg(a.any_mask + w);
  } else {
    *b = 0;
    *e31 = 0;
    *anyw = 0;
  }
}

// One theta application over the warp's words gwarp, gwarp + nwarps, ..., software pipelined:
// while the bits of word w are gathered, the column ids of the next word and the row bounds
// of the one after are already in flight. U column ids per row are staged; the rest of a longer
// row is read in a plain loop. Returns whether any of the warp's words changed (lane 0).
template <int U>
__device__ __forceinline__ bool theta_rows_pipelined(const FixArgs& a, const uint32_t* src, uint32_t* dst, int gwarp,
                                                     int nwarps, int lane) {
  bool changed = false;
  int w = gwarp;
  int b1, e1x, b2, e2x;
  uint32_t any1, any2;
  word_bounds(a, w, lane, &b1, &e1x, &any1);
  int j0[U];
  int l0, bb0;
  uint32_t any0;
  {
    int e = __shfl_down_sync(FULL, b1, 1);
    if (lane == 31) e = e1x;
    l0 = w < a.n_words ? e - b1 : 0;
    bb0 = b1;
    any0 = any1;
#pragma unroll
    for (int k = 0; k < U; k++) j0[k] = k < l0 ? __ldg(a.col + b1 + k) : -1;
  }
  word_bounds(a, w + nwarps, lane, &b1, &e1x, &any1);
  for (; w < a.n_words; w += nwarps) {  // w is uniform in the warp
    word_bounds(a, w + 2 * nwarps, lane, &b2, &e2x, &any2);
    int e = __shfl_down_sync(FULL, b1, 1);
    if (lane == 31) e = e1x;
    const int l1 = w + nwarps < a.n_words ? e - b1 : 0;
    int j1[U];
#pragma unroll
    for (int k = 0; k < U; k++) j1[k] = k < l1 ? __ldg(a.col + b1 + k) : -1;
    int c = 0;
#pragma unroll
    for (int k = 0; k < U; k++) c += j0[k] >= 0 ? (src[j0[k] >> 5] >> (j0[k] & 31)) & 1 : 0;
    for (int k = U; k < l0; k++) {
      const int j = __ldg(a.col + bb0 + k);
      c += (src[j >> 5] >> (j & 31)) & 1;
    }
    const uint32_t u = __ballot_sync(FULL, c >= (((any0 >> lane) & 1u) ? 1 : max(l0, 1)));
    if (lane == 0) {
      dst[w] = u;
      changed |= (u != src[w]);
    }
#pragma unroll
    for (int k = 0; k < U; k++) j0[k] = j1[k];
    l0 = l1;
    bb0 = b1;
    any0 = any1;
    b1 = b2;
    e1x = e2x;
    any1 = any2;
  }
  return changed;
}

template <int G, int XN, int MAP>
__global__ void __launch_bounds__(MAP == 0 ? kFixBlockMap0 : kFixBlockRows) fixpoint_kernel(FixArgs a) {
  constexpr int kBlock = MAP == 0 ? kFixBlockMap0 : kFixBlockRows;
  __shared__ int s_flag;
  __shared__ int s_cnt[G > 1 ? kBlock : 1];
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;

  // ---- initial vector v0
  fix_init_phase(a, gwarp, nwarps, gtid, nthreads, lane);
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
    if constexpr (MAP == 1) {
      int w = gwarp;
      for (; w + nwarps < a.n_words; w += 2 * nwarps) {
        uint32_t u1, u2;
        theta_pair_rows<8>(a, src, w, w + nwarps, lane, &u1, &u2);
        if (lane == 0) {
          dst[w] = u1;
          dst[w + nwarps] = u2;
          changed |= (u1 != src[w]) | (u2 != src[w + nwarps]);
        }
      }
      for (; w < a.n_words; w += nwarps) {
        uint32_t u[1];
        theta_words_rows<1, 8>(a, src, w, nwarps, lane, u);
        if (lane == 0) {
          dst[w] = u[0];
          changed |= (u[0] != src[w]);
        }
      }
    } else if constexpr (MAP == 2) {
      int w = gwarp;
      for (; w + 3 * nwarps < a.n_words; w += 4 * nwarps) {
        uint32_t u[4];
        theta_words_rows<4, 8>(a, src, w, nwarps, lane, u);
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            dst[w + q * nwarps] = u[q];
            changed |= (u[q] != src[w + q * nwarps]);
          }
        }
      }
      for (; w < a.n_words; w += nwarps) {
        uint32_t u[1];
        theta_words_rows<1, 8>(a, src, w, nwarps, lane, u);
        if (lane == 0) {
          dst[w] = u[0];
          changed |= (u[0] != src[w]);
        }
      }
    } else if constexpr (MAP == 3) {
      changed = theta_rows_pipelined<5>(a, src, dst, gwarp, nwarps, lane);
    } else if (G == 1) {
      int w = gwarp;
      for (; w + nwarps < a.n_words; w += 2 * nwarps) {
        uint32_t u1, u2;
        theta_word_pair<XN>(a, src, w, w + nwarps, lane, &u1, &u2);
        if (lane == 0) {
          dst[w] = u1;
          dst[w + nwarps] = u2;
          changed |= (u1 != src[w]) | (u2 != src[w + nwarps]);
        }
      }
      for (; w < a.n_words; w += nwarps) {  // a last single word
        const uint32_t u = theta_word<XN>(a.row_ptr, a.col, a.any_mask, src, w, lane);
        if (lane == 0) {
          dst[w] = u;
          changed |= (u != src[w]);
        }
      }
    } else {
      // kBlock / 32 / G words per block and round; the loop bound is uniform in the block
      const int warp = threadIdx.x >> 5, slot = warp / G, part = warp % G;
      const int per_block = (kBlock / 32) / G;
      for (int wb = blockIdx.x * per_block; wb < a.n_words; wb += gridDim.x * per_block) {
        const int w = wb + slot;
        int len = 0, cnt = 0;
        if (w < a.n_words) cnt = theta_word_part<XN>(a.row_ptr, a.col, src, w, lane, part, G, &len);
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
  fix_output_phase(a, fin, gwarp, nwarps, lane);
}

static const void* fixpoint_entry(int G, int XN, int MAP) {
  switch (MAP) {  // the thread-per-row maps have no row split or chunk batch
    case 1: return (const void*)fixpoint_kernel<1, 1, 1>;
    case 2: return (const void*)fixpoint_kernel<1, 1, 2>;
    case 3: return (const void*)fixpoint_kernel<1, 1, 3>;
    default: break;
  }
  if (XN == 4) {
    switch (G) {
      case 2: return (const void*)fixpoint_kernel<2, 4, 0>;
      case 4: return (const void*)fixpoint_kernel<4, 4, 0>;
      case 8: return (const void*)fixpoint_kernel<8, 4, 0>;
      default: return (const void*)fixpoint_kernel<1, 4, 0>;
    }
  }
  switch (G) {
    case 2: return (const void*)fixpoint_kernel<2, 1, 0>;
    case 4: return (const void*)fixpoint_kernel<4, 1, 0>;
    case 8: return (const void*)fixpoint_kernel<8, 1, 0>;
    default: return (const void*)fixpoint_kernel<1, 1, 0>;
  }
}

cudaError_t launch_fixpoint(const FixArgs& a, int grid, int row_split, int chunk_batch, int row_map, cudaStream_t s) {
  FixArgs copy = a;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(fixpoint_entry(row_split, chunk_batch, row_map), dim3(grid),
                                     dim3(fix_block(row_map)), params, 0, s);
}

int fixpoint_blocks_per_sm(int row_split, int chunk_batch, int row_map) {
  int nb = 0;
  const void* k = fixpoint_entry(row_split, chunk_batch, row_map);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, fix_block(row_map), 0) != cudaSuccess) return 0;
  return nb;
}

}  // namespace lp

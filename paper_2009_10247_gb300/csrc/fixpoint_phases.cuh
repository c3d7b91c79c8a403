// fixpoint_phases.cuh -- the phases of a least-model launch that every row map shares: the
// initial vector v0 (Def. 4, or a caller's row vector) and the projection of the fixpoint on
// the original atoms in the caller's order.
#pragma once

#include "device.cuh"
#include "kernels.h"

namespace lp {

__device__ __forceinline__ uint32_t get_bit(const uint32_t* v, int i) { return (v[i >> 5] >> (i & 31)) & 1u; }

// v0 into a.x0. LP_ROWS: internal row r takes bit inv[r] of the caller's canonical vector.
// Default: a fact row is 1 when its atom is selected (x0 was zeroed by the caller), and a
// selected atom without a fact rule raises LP_ERR_INVALID.
__device__ __forceinline__ void fix_init_phase(const FixArgs& a, int gwarp, int nwarps, int gtid, int nthreads,
                                               int lane) {
  if (a.rows_init) {
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
    for (int i = gtid; i < a.n_facts; i += nthreads) {
      const int own = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own >> 6] >> (own & 63)) & 1ull) : true;
      if (sel) atomicOr(a.x0 + (a.fact_row[i] >> 5), 1u << (a.fact_row[i] & 31));
    }
    if (a.init)
      for (int i = gtid; i < a.n_atom_words; i += nthreads)
        if (a.init[i] & ~a.fact_mask[i]) atomicCAS(&a.ctl->status, 0, 1 /* LP_ERR_INVALID */);
  }
}

// Bit a of a.out = fixpoint bit of internal row perm[a], a < n_out.
__device__ __forceinline__ void fix_output_phase(const FixArgs& a, const uint32_t* fin, int gwarp, int nwarps,
                                                 int lane) {
  if (!a.out) return;
  uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
  const int n32 = 2 * ((a.n_out + 63) >> 6);
  for (int u = gwarp; u < n32; u += nwarps) {
    const int i = (u << 5) + lane;
    const uint32_t bit = i < a.n_out ? get_bit(fin, a.perm[i]) : 0u;
    const uint32_t word = __ballot_sync(FULL, bit);
    if (lane == 0) out32[u] = word;
  }
}

}  // namespace lp

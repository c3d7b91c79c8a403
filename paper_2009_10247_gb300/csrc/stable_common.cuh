// stable_common.cuh -- device helpers shared by the two stable-model kernels (the full sweep of
// stable.cu and the frontier schedule of stable_frontier.cu): the words of the initial matrix
// M_0 (Def. 8), one row of theta(M_P M_k) over a tile of guess words (Def. 5), and a warp-wide
// append to a work list.
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace lp {

// Word gw of M_0 in a row with tag `tag` (row_tag values): bit b of the word is the row's value
// under guess 64 gw + b.
__device__ __forceinline__ uint64_t m0_word(int tag, long long gw, const StableArgs& a) {
  if (tag == -2) return ~0ull;  // fact row (Def. 8 item 2)
  if (tag < 0) return 0ull;     // other original rows, barred atoms of facts (item 3)
  if (a.guesses == nullptr) {
    // guess g = 64*gw + b, bit tag of g
    switch (tag) {  // bit b of the word is bit tag of b
      case 0: return 0xAAAAAAAAAAAAAAAAull;
      case 1: return 0xCCCCCCCCCCCCCCCCull;
      case 2: return 0xF0F0F0F0F0F0F0F0ull;
      case 3: return 0xFF00FF00FF00FF00ull;
      case 4: return 0xFFFF0000FFFF0000ull;
      case 5: return 0xFFFFFFFF00000000ull;
      default: break;
    }
    return ((gw >> (tag - 6)) & 1ll) ? ~0ull : 0ull;
  }
  uint64_t w = 0;
  const long long g0 = gw * 64;
  for (int b = 0; b < 64; b++) {
    const long long g = g0 + b;
    if (g < a.n_guesses) w |= ((a.guesses[g] >> tag) & 1ull) << b;
  }
  return w;
}

// The words of `row` in a tile of W words (lane word wl; src is the tile's buffer): AND of its
// entries' words for a rule row, OR for an OR row or a self-loop, 0 for an empty row. Four
// entries per step: their column loads, then their gathers. *n_entries grows by the row's length.
__device__ __forceinline__ uint64_t eval_row(const StableArgs& a, const uint64_t* src, int row, int wl,
                                             unsigned* n_entries) {
  const int beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
  const bool any = (__ldg(a.any_mask + (row >> 5)) >> (row & 31)) & 1u;
  const uint64_t ident = any ? 0ull : ~0ull;
  uint64_t acc = (end > beg) ? ident : 0ull;
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
  *n_entries += (unsigned)(end - beg);
  return acc;
}

// Appends `value` of every lane whose flag is set to list[*cnt ...] (one atomic per warp; all
// lanes of the warp call it).
__device__ __forceinline__ void warp_append(int32_t* list, unsigned* cnt, bool flag, int value, int lane) {
  const unsigned m = __ballot_sync(FULL, flag);
  if (m == 0u) return;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (flag) list[base + __popc(m & ((1u << lane) - 1u))] = value;
}

}  // namespace lp

// stable_frontier.cu -- Algorithms 2 and 3 under the frontier schedule: all tiles of guesses are
// iterated together, and each iteration evaluates only the rows one of whose inputs changed.
//
// Algorithm 2 computes M_{t+1} = theta(M_P M_t) column by column. Row i of M_{t+1} depends only on
// the rows of M_t that row i of M_P refers to, so a row none of whose inputs changed in the last
// iteration keeps its value. With two buffers (src holds M_t, dst held M_{t-1}) a row that is not
// evaluated keeps the right value in dst, provided every row that changed in the last iteration is
// evaluated again too. An iteration therefore works from a list of items (tile, row): it evaluates
// them, and pushes each item that changed, with the rows referring to it in the same tile
// (transposed matrix, deduplicated by a per-item stamp), into the next iteration's list. The
// columns of a tile have reached their fixpoint when the tile has no item left; the launch ends an
// iteration after the last tile's. With T tiles of one wave in flight, one grid barrier serves T
// tiles, so a wave costs about as many barriers as its slowest tile has iterations.
//
// Iteration 0 needs no full sweep: M_0 is zero outside the fact rows and the guessed barred rows,
// and theta of a row whose inputs are all zero is zero (an AND row has an entry, an OR row fires on
// none, an empty row never fires). So with dst = M_0 on every other row, the first list is those
// rows and the rows referring to them.
//
// Starting from F (fr_F set): F is the least fixpoint reached from the fact rows with every
// guessed row zero -- the part of every column's fixpoint that no guess can change (theta of M_P
// is monotone and a guess only adds ones to M_0). The iteration may start from S = F with the
// guess's bits on the guessed rows instead of from M_0: M_0 <= S <= the column's least fixpoint
// and S <= theta(M_P S) (F is a fixpoint, a guessed row is a self-loop), so it climbs to the same
// fixpoint, the same stable bits and models, in fewer iterations (the iteration counts are then
// those from S, not Algorithm 2's from M_0). Rows other than the guessed rows and the rows
// referring to them keep F's value in iteration 0, so the first list is those rows alone, and the
// buffers rest at F.
//
// Between solves the buffers rest in that state -- fact rows all ones, every other row zero, in
// both buffers -- and a solve leaves them so: a bitmap records every item that changed, and after
// Algorithm 3 those items and the guessed rows are written back. The first solve on a handle (or
// after a launch that did not finish, or after the layout changed) writes the rest state in full.
// A record in fr_cnt tells the next launch whether it can trust the buffers: the layout tag, the
// grid size, and how many blocks of the last launch finished.
//
// Dense programs (rows of hundreds of entries, atoms in thousands of bodies) get two more paths.
// A row with at least kLongRow entries goes to a long list whose items a whole warp evaluates, its
// lane groups splitting the entries and combining their partial AND / OR with shuffles. An item
// whose row has more than kWideDeps dependents lists itself as wide, and after the iteration's
// barrier the whole grid pushes those dependents (one more barrier in such an iteration) instead
// of one lane group pushing them in sequence. Where an item takes fewer than eight lanes, a
// warp's pushes are numbered across its items and spread over all 32 lanes.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"
#include "stable_common.cuh"

namespace lp {

namespace {

// fr_cnt slots
constexpr int kCntGrid = 3;   // grid size of the last launch
constexpr int kCntKey = 4;    // layout tag of the rest state
constexpr int kCntStamp = 5;  // next unused stamp
constexpr int kCntClean = 6;  // tiles of the buffers in the rest state
constexpr int kCntDone = 7;   // blocks of the last launch that finished
// Three groups of four (16-byte aligned), rotating: group t % 3 holds what iteration t produces
// -- the sizes of the next short and long lists and the number of its wide items -- read by
// every thread with one load after the barrier that ends the iteration. The first list is
// iteration -1's (group 2).
constexpr int kCntGroups = 16;
constexpr unsigned kStampLimit = 0xF0000000u;
// an item whose row has more dependents than this has them pushed by the whole grid
constexpr int kWideDeps = 128;

// The words a row rests at between solves (in every tile): with fr_F, its bit of the
// guess-independent fixpoint F (all ones or all zeros across the guesses); else M_0 outside the
// guessed rows (ones on a fact row, zeros elsewhere).
__device__ __forceinline__ uint64_t rest_word(const StableArgs& a, int row) {
  if (a.fr_F) return ((__ldg(a.fr_F + (row >> 5)) >> (row & 31)) & 1u) ? ~0ull : 0ull;
  return __ldg(a.row_tag + row) == -2 ? ~0ull : 0ull;
}

__device__ __forceinline__ uint4 ld_volatile4(const unsigned* p) {
  uint4 v;
  asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

// Per-warp staging of list appends in shared memory: the winners of a step go to the warp's
// 64-slot buffer, and the list gets them 32 at a time with one atomic on its counter (all warps
// of the grid append to the same counter; one atomic per step serialized on it).
// one 1024-thread block per SM: a quarter of the blocks (and arrivals) at each grid barrier of
// the 256-thread blocks it replaced, with the same 32 warps per SM (2 % faster on the 2^16-guess
// normal program)
constexpr int kFrontierBlock = 1024;
__shared__ int s_stage[2][kFrontierBlock / 32][64];  // [short, long][warp of the block]

// The two lists an iteration appends to share one buffer of cap = fr_tiles * n_pad slots: the
// short list from the front, the long list from the back (slot cap - 1 - i holds entry i).
// Their sizes are cnt[0] and cnt[1]. Both never hold more than cap items together, as an item
// enters them at most once per stamp.
struct Lists {
  int32_t* list;
  unsigned* cnt;
  int n_s, n_l;  // entries staged in this warp's two buffers
};

__device__ __forceinline__ void stage_out(const StableArgs& a, int32_t* list, unsigned base, int i, int v, bool back) {
  const long long pos = (long long)base + i;
  list[back ? (long long)a.fr_tiles * a.n_pad - 1 - pos : pos] = v;
}
// One staged append; all lanes call it with the same state.
__device__ __forceinline__ void staged_append(const StableArgs& a, Lists& L, bool back, bool flag, int value,
                                              int lane) {
  const unsigned m = __ballot_sync(FULL, flag);
  if (m == 0u) return;
  int* buf = s_stage[back][threadIdx.x >> 5];
  int& n = back ? L.n_l : L.n_s;
  if (flag) buf[n + __popc(m & ((1u << lane) - 1u))] = value;
  n += __popc(m);
  __syncwarp();
  if (n >= 32) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(L.cnt + (back ? 1 : 0), 32u);
    base = __shfl_sync(FULL, base, 0);
    stage_out(a, L.list, base, lane, buf[lane], back);
    const int rest = n - 32;
    const int moved = lane < rest ? buf[32 + lane] : 0;
    __syncwarp();
    if (lane < rest) buf[lane] = moved;
    n = rest;
    __syncwarp();
  }
}
__device__ __forceinline__ void staged_flush(const StableArgs& a, Lists& L, int lane) {
#pragma unroll
  for (int back = 0; back < 2; back++) {
    int& n = back ? L.n_l : L.n_s;
    if (n > 0) {
      const int* buf = s_stage[back][threadIdx.x >> 5];
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(L.cnt + (back ? 1 : 0), (unsigned)n);
      base = __shfl_sync(FULL, base, 0);
      if (lane < n) stage_out(a, L.list, base, lane, buf[lane], back);
      n = 0;
    }
    __syncwarp();
  }
}

// One push of item (tile c, row): the first push under `stamp` wins, and the winner goes to the
// long list if the row is long, else to the short one (long_mask is NULL when no row is long).
// All lanes call it; `valid` marks a push.
__device__ __forceinline__ void push_item(const StableArgs& a, bool valid, int c, int row, unsigned stamp, Lists& L,
                                          int lane) {
  bool win = false, lg = false;
  int item = 0;
  if (valid) {
    item = c * a.n_pad + row;
    win = atomicExch(a.mark + item, stamp) != stamp;
    if (a.long_mask) lg = (__ldg(a.long_mask + (row >> 5)) >> (row & 31)) & 1u;
  }
  staged_append(a, L, false, win && !lg, item, lane);
  if (a.long_mask) staged_append(a, L, true, win && lg, item, lane);
}

// The dependents of the wide items (items whose rows have more than kWideDeps dependents, set
// aside while the grid evaluated): with n_wide <= nwarps each item gets a run of nwarps / n_wide
// warps whose lanes split its dependents, else each warp takes whole items.
__device__ __forceinline__ void expand_wide(const StableArgs& a, unsigned n_wide, unsigned stamp, Lists& L, int gwarp,
                                            int nwarps, int lane) {
  const long long nw = n_wide;
  long long i0, di, k, nk;
  if (nw <= nwarps) {
    i0 = (long long)gwarp * nw / nwarps;
    const long long f0 = (i0 * nwarps + nw - 1) / nw, f1 = ((i0 + 1) * nwarps + nw - 1) / nw;
    k = gwarp - f0;
    nk = f1 - f0;
    di = nw;  // one item
  } else {
    i0 = gwarp;
    di = nwarps;
    k = 0;
    nk = 1;
  }
  for (long long i = i0; i < nw; i += di) {
    const int item = a.fr_wide[i];
    const int c = item / a.n_pad, row = item - c * a.n_pad;
    const int tb = __ldg(a.t_ptr + row), nd = __ldg(a.t_ptr + row + 1) - tb;
    for (long long d0 = k * 32; d0 < nd; d0 += nk * 32) {
      const long long d = d0 + lane;
      const int dep = d < nd ? __ldg(a.t_idx + tb + d) : 0;
      push_item(a, d < nd, c, dep, stamp, L, lane);
    }
  }
}

// WPL consecutive 64-bit words at p (16-byte aligned when WPL > 1).
template <int WPL>
__device__ __forceinline__ void load_words(const uint64_t* p, uint64_t (&v)[WPL]) {
  if constexpr (WPL == 1) {
    v[0] = *p;
  } else {
#pragma unroll
    for (int j = 0; j < WPL; j += 2) {
      const ulonglong2 q = *reinterpret_cast<const ulonglong2*>(p + j);
      v[j] = q.x;
      v[j + 1] = q.y;
    }
  }
}

// Words w0 .. w0 + WPL - 1 of `row` in a tile (src is the tile's buffer), as eval_row: AND of the
// entries' words for a rule row, OR for an OR row or a self-loop, 0 for an empty row; over the
// entries beg + s0, beg + s0 + S, ... (S = 1: all of them; lane groups that split a long row
// take one residue each and combine afterwards), E per step (their column loads, then their
// gathers: four entries, two with four words per lane). Returns the row's length.
template <int WPL>
__device__ __forceinline__ int eval_row_words(const StableArgs& a, const uint64_t* src, int row, int w0, int s0,
                                              int S, uint64_t (&acc)[WPL]) {
  constexpr int E = WPL >= 4 ? 2 : 4;
  const int beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
  const bool any = (__ldg(a.any_mask + (row >> 5)) >> (row & 31)) & 1u;
  const uint64_t ident = any ? 0ull : ~0ull;
#pragma unroll
  for (int j = 0; j < WPL; j++) acc[j] = end > beg ? ident : 0ull;
  for (int e = beg + s0; e < end; e += E * S) {
    int cc[E];
#pragma unroll
    for (int q = 0; q < E; q++) cc[q] = e + q * S < end ? __ldg(a.col + e + q * S) : -1;
    uint64_t v[E][WPL];
#pragma unroll
    for (int q = 0; q < E; q++) {
      if (cc[q] >= 0) {
        load_words<WPL>(src + ((long long)cc[q] << a.log2W) + w0, v[q]);
      } else {
#pragma unroll
        for (int j = 0; j < WPL; j++) v[q][j] = ident;
      }
    }
#pragma unroll
    for (int j = 0; j < WPL; j++) {
      uint64_t orv = 0ull, andv = ~0ull;
#pragma unroll
      for (int q = 0; q < E; q++) {
        orv |= v[q][j];
        andv &= v[q][j];
      }
      acc[j] = any ? (acc[j] | orv) : (acc[j] & andv);
    }
  }
  return end - beg;
}

// WPL: words per lane in the iterations. An item (W words) takes W / WPL lanes, so a warp
// evaluates 32 WPL / W items at once: with W = 32, four items of eight lanes, four words each.
template <int WPL>
__global__ void __launch_bounds__(kFrontierBlock, 1) stable_frontier_kernel(StableArgs a) {
  __shared__ long long s_base;
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  DeviceCtl* ctl = a.ctl;
  unsigned* const st = a.fr_cnt;
  unsigned long long round = 0;
  const int W = a.W, log2W = a.log2W;
  const int rpw = 32 >> log2W;   // items per warp
  const int sub = lane >> log2W;  // item within the warp's group
  const int wl = lane & (W - 1);  // word within the tile
  const int lpi = W / WPL;           // lanes per item in the iterations
  const int ipw = 32 / lpi;          // items per warp
  const int isub = lane / lpi;       // item within the warp
  const int il = lane - isub * lpi;  // lane within the item
  const unsigned imask = lpi == 32 ? FULL : (((1u << lpi) - 1u) << (isub * lpi));
  const int n_pad = a.n_pad;
  const long long tile_words = (long long)n_pad * W;
  const int c_wave = (int)min((long long)a.fr_tiles, (long long)a.n_tiles);  // tiles per wave
  const long long cap_items = (long long)a.fr_tiles * n_pad;

  // ---- the buffers' state left by the last launch
  const bool known = ld_volatile(st + kCntKey) == a.fr_key && ld_volatile(st + kCntDone) == ld_volatile(st + kCntGrid);
  unsigned stamp = known ? ld_volatile(st + kCntStamp) : 1u;
  int clean = known ? (int)ld_volatile(st + kCntClean) : 0;
  if (!grid_barrier(ctl, ++round, 6)) return;
  if (gtid == 0) {  // everyone has read the record
    st[kCntKey] = a.fr_key;
    st[kCntGrid] = gridDim.x;
    st[kCntDone] = 0u;
    for (int q = kCntGroups; q < kCntGroups + 12; q++) st[q] = 0u;
  }
  for (long long c = gtid; c < a.fr_tiles; c += nthreads) a.fr_last[c] = -1;
  if (clean < c_wave) {  // tiles clean .. c_wave - 1 into the rest state
    const long long i0 = (long long)clean * n_pad, i1 = (long long)c_wave * n_pad;
    for (long long g = gwarp; i0 + g * rpw < i1; g += nwarps) {
      const long long item = i0 + g * rpw + sub;
      if (item < i1) {
        const uint64_t v = rest_word(a, (int)(item % n_pad));
        a.X0[item * W + wl] = v;
        a.X1[item * W + wl] = v;
        if (wl == 0) a.mark[item] = 0u;
      }
    }
    for (long long q = i0 / 32 + gtid; q < (i1 + 31) / 32; q += nthreads) a.fr_dirty[q] = 0u;
    clean = c_wave;  // tiles past c_wave that were clean stay so
  }
  if (!grid_barrier(ctl, ++round, 6)) return;

  unsigned n_rows = 0, n_ent = 0, n_list = 0, n_deps = 0;
  for (long long w0 = 0; w0 < a.n_tiles; w0 += c_wave) {
    const int cw = (int)min((long long)c_wave, (long long)(a.n_tiles - w0));  // tiles of this wave
    const long long gw0 = w0 * W;                                   // its first guess word
    if (stamp > kStampLimit - (unsigned)a.max_iters - 4u) {  // stamps start over
      for (long long i = gtid; i < (long long)c_wave * n_pad; i += nthreads) a.mark[i] = 0u;
      clean = c_wave;  // tiles past c_wave keep old stamps: no longer clean
      stamp = 1u;
      if (!grid_barrier(ctl, ++round, 6)) return;
    }

    uint4 cnt4;  // the sizes of the list an iteration works on (x: short, y: long)

    // ---- 1. M_0 of the guessed rows, and the first list: fact and guessed rows and the rows
    // referring to them, in every tile of the wave. A (seed row, tile) pair per eight lanes,
    // four pairs per warp; a seed row with many dependents has them pushed by the whole grid.
    {
      Lists L{a.fr_list, st + kCntGroups + 8, 0, 0};
      const int gsub = lane >> 3, gl = lane & 7;
      const long long n_pairs = (long long)a.n_seed * cw;
      for (long long base = (long long)gwarp * 4; base < n_pairs; base += (long long)nwarps * 4) {
        const long long pi = base + gsub;
        int row = 0, c = 0, tb = 0, per = 0, tg = -1;
        if (pi < n_pairs) {
          row = __ldg(a.fr_seed + (int)(pi % a.n_seed));
          c = (int)(pi / a.n_seed);
          tg = __ldg(a.row_tag + row);
          tb = __ldg(a.t_ptr + row);
          per = 1 + __ldg(a.t_ptr + row + 1) - tb;
          if (per - 1 > kWideDeps) {  // its dependents go to the grid (if the wide list has room)
            unsigned slot = 0;
            if (gl == 0) {
              slot = atomicAdd(L.cnt + 2, 1u);
              if (slot < (unsigned)a.wide_cap) a.fr_wide[slot] = c * n_pad + row;
            }
            slot = __shfl_sync(0xFFu << (8 * gsub), slot, 8 * gsub);
            if (slot < (unsigned)a.wide_cap) per = 1;
          }
        }
        if (tg >= 0)  // a guessed row: its words of M_0 in this tile
          for (int w = gl; w < W; w += 8)
            a.X0[((long long)c * n_pad + row) * W + w] = m0_word(tg, gw0 + (long long)c * W + w, a);
        const int steps = (int)__reduce_max_sync(FULL, (unsigned)((per + 7) >> 3));
        for (int s2 = 0; s2 < steps; s2++) {
          const int d = 8 * s2 + gl;
          const int dep = d < per ? (d == 0 ? row : __ldg(a.t_idx + tb + d - 1)) : 0;
          push_item(a, d < per, c, dep, stamp, L, lane);
        }
      }
      staged_flush(a, L, lane);
      if (!grid_barrier(ctl, ++round, 6)) return;  // the first list and its wide seeds are listed
      cnt4 = ld_volatile4(L.cnt);
      const unsigned n_wide = min(cnt4.z, (unsigned)a.wide_cap);
      if (n_wide > 0u) {
        expand_wide(a, n_wide, stamp, L, gwarp, nwarps, lane);
        staged_flush(a, L, lane);
        if (!grid_barrier(ctl, ++round, 6)) return;
        cnt4 = ld_volatile4(L.cnt);
      }
    }

    // ---- 2. the iterations: the long list (rows of at least kLongRow entries, a warp per item,
    // the warp's lane groups splitting the entries), then the short list (a lane group per item)
    const uint64_t* fin = a.X0;
    int t = 0;
    bool converged = false;
    for (; t < a.max_iters; ++t) {
      const uint64_t* src = (t & 1) ? a.X1 : a.X0;
      uint64_t* dst = (t & 1) ? a.X0 : a.X1;
      const int32_t* cur = a.fr_list + (size_t)(t & 1) * cap_items;
      int32_t* nxt = a.fr_list + (size_t)((t + 1) & 1) * cap_items;
      unsigned* const grp = st + kCntGroups + 4 * (t % 3);  // what this iteration produces
      unsigned* const wide_cnt = grp + 2;
      const unsigned nstamp = stamp + (unsigned)t + 1u;
      // group (t + 1) % 3 was last read after iteration t - 2, before the last barrier
      if (gtid == 0) {
        unsigned* g1 = st + kCntGroups + 4 * ((t + 1) % 3);
        g1[0] = g1[1] = g1[2] = 0u;
      }
      const long long n_cur = cnt4.x, n_long = cnt4.y;
      Lists L{nxt, grp, 0, 0};

      // (a) long items, one per warp
      for (long long g = gwarp; g < n_long; g += nwarps) {
        const int item = cur[cap_items - 1 - g];
        const int c = item / n_pad, row = item - c * n_pad;
        const long long o = (long long)item * W + il * WPL;
        uint64_t acc[WPL], old[WPL];
        load_words<WPL>(src + o, old);
        const int tb = __ldg(a.t_ptr + row), te = __ldg(a.t_ptr + row + 1);
        const bool any = (__ldg(a.any_mask + (row >> 5)) >> (row & 31)) & 1u;
        const int len = eval_row_words<WPL>(a, src + (size_t)c * tile_words, row, il * WPL, isub, ipw, acc);
        for (int off = lpi; off < 32; off <<= 1) {  // combine the lane groups
#pragma unroll
          for (int j = 0; j < WPL; j++) {
            const uint64_t other = __shfl_xor_sync(FULL, acc[j], off);
            acc[j] = any ? (acc[j] | other) : (acc[j] & other);
          }
        }
        bool differs = false;
#pragma unroll
        for (int j = 0; j < WPL; j++) differs |= acc[j] != old[j];
        if (isub == 0) {
#pragma unroll
          for (int j = 0; j < WPL; j++) dst[o + j] = acc[j];
        }
        if (lane == 0) {
          n_rows++;
          n_ent += (unsigned)len;
        }
        if (__ballot_sync(FULL, differs) == 0u) continue;
        int per = 1 + te - tb;
        if (lane == 0) {
          atomicOr(a.fr_dirty + (item >> 5), 1u << (item & 31));
          atomicMax(a.fr_last + c, t);
          n_list++;
          n_deps += (unsigned)(per - 1);
          if (per - 1 > kWideDeps) {
            const unsigned slot = atomicAdd(wide_cnt, 1u);
            if (slot < (unsigned)a.wide_cap) {
              a.fr_wide[slot] = item;
              per = 1;
            }
          }
        }
        per = __shfl_sync(FULL, per, 0);
        for (int d0 = 0; d0 < per; d0 += 32) {
          const int d = d0 + lane;
          const int dep = d < per ? (d == 0 ? row : __ldg(a.t_idx + tb + d - 1)) : 0;
          push_item(a, d < per, c, dep, nstamp, L, lane);
        }
      }

      // (b) short items, ipw per warp; the chunks start after the warps that took long items
      const long long g0 = ((gwarp - n_long) % nwarps + nwarps) % nwarps;
      for (long long g = g0; g * ipw < n_cur; g += nwarps) {
        const long long idx = g * ipw + isub;
        const int item = idx < n_cur ? cur[idx] : -1;
        uint64_t acc[WPL], old[WPL];
        bool differs = false;
        int c = 0, row = 0, tb = 0, te = 0;
        if (item >= 0) {
          c = item / n_pad;
          row = item - c * n_pad;
          const long long o = (long long)item * W + il * WPL;
          // loads that do not wait on the row's entries go first: the old words and the
          // transposed row's range (used if the row changes)
          load_words<WPL>(src + o, old);
          tb = __ldg(a.t_ptr + row);
          te = __ldg(a.t_ptr + row + 1);
          const int len = eval_row_words<WPL>(a, src + (size_t)c * tile_words, row, il * WPL, 0, 1, acc);
#pragma unroll
          for (int j = 0; j < WPL; j++) {
            dst[o + j] = acc[j];
            differs |= acc[j] != old[j];
          }
          if (il == 0) {
            n_rows++;
            n_ent += (unsigned)len;
          }
        }
        const unsigned diff = __ballot_sync(FULL, differs);
        const bool ch = item >= 0 && (diff & imask) != 0u;
        // pushes of the warp's changed items (each: itself and the rows referring to it), numbered
        // across the warp and spread over all 32 lanes
        int per = 0;
        if (ch && il == 0) {
          per = 1 + te - tb;
          atomicOr(a.fr_dirty + (item >> 5), 1u << (item & 31));
          atomicMax(a.fr_last + c, t);
          n_list++;
          n_deps += (unsigned)(per - 1);
          if (per - 1 > kWideDeps) {
            const unsigned slot = atomicAdd(wide_cnt, 1u);
            if (slot < (unsigned)a.wide_cap) {
              a.fr_wide[slot] = item;
              per = 1;
            }
          }
        }
        if (WPL >= 2 || lpi >= 8) {
          // eight lanes per item: each item pushes itself and its dependents, eight at a time
          per = __shfl_sync(FULL, per, isub * lpi);
          const int steps = __reduce_max_sync(FULL, (unsigned)((per + lpi - 1) / lpi));
          for (int s2 = 0; s2 < steps; s2++) {
            const int d = s2 * lpi + il;
            const int dep = d < per ? (d == 0 ? row : __ldg(a.t_idx + tb + d - 1)) : 0;
            push_item(a, d < per, c, dep, nstamp, L, lane);
          }
        } else {
          // one to four lanes per item: the warp's pushes are numbered across its items and
          // spread over all 32 lanes
          int incl = per;  // inclusive scan (only each item's first lane is nonzero)
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += u;
          }
          const int total = __shfl_sync(FULL, incl, 31);
          const int first = incl - per;  // this item's first push (valid on its first lane)
          for (int f0 = 0; f0 < total; f0 += 32) {
            const int f = f0 + lane;
            int pos = 0;  // the last item whose first push is <= f
            for (int step = ipw >> 1; step > 0; step >>= 1) {
              const int b = __shfl_sync(FULL, first, (pos + step) * lpi);
              if (b <= f) pos += step;
            }
            const int src_lane = pos * lpi;
            const int p_item = __shfl_sync(FULL, item, src_lane);
            const int p_tb = __shfl_sync(FULL, tb, src_lane);
            const int d = f - __shfl_sync(FULL, first, src_lane);
            const int pc = p_item / n_pad, prow = p_item - pc * n_pad;
            const int dep = f < total ? (d == 0 ? prow : __ldg(a.t_idx + p_tb + d - 1)) : 0;
            push_item(a, f < total, pc, dep, nstamp, L, lane);
          }
        }
      }
      staged_flush(a, L, lane);
      if (!grid_barrier(ctl, ++round, 6)) return;  // the next lists and this iteration's wide items
      cnt4 = ld_volatile4(grp);
      const unsigned n_wide = min(cnt4.z, (unsigned)a.wide_cap);
      if (n_wide > 0u) {  // the wide items' dependents join the next lists
        expand_wide(a, n_wide, nstamp, L, gwarp, nwarps, lane);
        staged_flush(a, L, lane);
        if (!grid_barrier(ctl, ++round, 6)) return;
        cnt4 = ld_volatile4(grp);
      }
      fin = dst;
      if (cnt4.x == 0u && cnt4.y == 0u) {
        converged = true;
        ++t;
        break;
      }
    }
    stamp += (unsigned)t + 1u;

    const int nw = cw * W;                 // guess words of the wave
    const int n_chunks = (nw + 31) / 32;   // 32 words per warp below
    int32_t* csum = a.fr_list;             // the lists are free now: chunk counts, then offsets
    if (converged) {
      // ---- 3. Algorithm 3 on the wave's words; per-tile iteration counts
      for (long long c = gtid; c < cw; c += nthreads) {
        const int its = a.fr_last[c] + 2;  // last changing iteration, then one that confirms
        atomicMax(&ctl->max_tile_iters, its);
        atomicAdd((unsigned long long*)&ctl->sum_tile_iters, (unsigned long long)its);
        if (c == cw - 1) {
          ctl->iters = its;
          ctl->tiles = w0 + cw;
        }
      }
      for (int q = gwarp; q < n_chunks; q += nwarps) {
        const int k = q * 32 + lane;
        const long long gw = gw0 + k;
        uint64_t sw = 0ull;
        if (k < nw && gw < a.n_gwords) {
          const uint64_t* fc = fin + (size_t)(k >> log2W) * tile_words;
          const int w = k & (W - 1);
          const long long rem = a.n_guesses - gw * 64;
          sw = rem >= 64 ? ~0ull : ((1ull << rem) - 1ull);
          for (int j = 0; j < a.n_barred; j++)
            sw &= fc[((long long)a.neg_row[j] << log2W) + w] ^ fc[((long long)a.bar_row[j] << log2W) + w];
          a.stable_mask[gw] = sw;
        }
        const int cnt = __reduce_add_sync(FULL, (unsigned)__popcll(sw));
        if (lane == 0) csum[q] = cnt;
      }
      if (!grid_barrier(ctl, ++round, 6)) return;
      // ---- 4. the chunks' offsets (one warp), then the models of the stable columns in guess order
      if (gtid < 32) {
        int run = 0;
        for (int q0 = 0; q0 < n_chunks; q0 += 32) {
          const int q = q0 + lane;
          const int v = q < n_chunks ? csum[q] : 0;
          int incl = v;
          for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += u;
          }
          if (q < n_chunks) csum[q] = run + incl - v;
          run += __shfl_sync(FULL, incl, 31);
        }
        if (lane == 0) csum[n_chunks] = run;
      }
      if (!grid_barrier(ctl, ++round, 6)) return;
      if (threadIdx.x == 0) s_base = *reinterpret_cast<volatile long long*>(&ctl->n_stable);
      __syncthreads();
      const long long base = s_base;
      const int wave_count = ((volatile int32_t*)csum)[n_chunks];
      if (a.models) {
        for (long long m = gwarp; m < wave_count && base + m < a.max_models; m += nwarps) {
          int lo = 0, hi = n_chunks - 1;  // last chunk whose offset is <= m
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (((volatile int32_t*)csum)[mid] <= m) lo = mid;
            else hi = mid - 1;
          }
          const int q = lo;
          const int k = q * 32 + lane;
          const long long gw = gw0 + k;
          const uint64_t myword = (k < nw && gw < a.n_gwords) ? a.stable_mask[gw] : 0ull;
          const int mycnt = __popcll(myword);
          int incl = mycnt;
          for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += u;
          }
          const int r = (int)(m - ((volatile int32_t*)csum)[q]);  // rank within the chunk
          const int wsel = __ffs(__ballot_sync(FULL, incl > r)) - 1;
          const int before = __shfl_sync(FULL, incl - mycnt, wsel);
          uint64_t word = __shfl_sync(FULL, myword, wsel);
          for (int z = 0; z < r - before; z++) word &= word - 1;  // drop lower set bits
          const int b = __ffsll((long long)word) - 1;
          const int kk = q * 32 + wsel;
          const uint64_t* fc = fin + (size_t)(kk >> log2W) * tile_words;
          const int w = kk & (W - 1);
          uint32_t* out = reinterpret_cast<uint32_t*>(a.models + (base + m) * a.n_atom_words);
          const int n32 = 2 * a.n_atom_words;
          for (int u = 0; u < n32; u++) {
            const int atom = (u << 5) + lane;
            uint32_t bit = 0;
            if (atom < a.n) bit = (uint32_t)(fc[((long long)a.perm[atom] << log2W) + w] >> b) & 1u;
            const uint32_t word32 = __ballot_sync(FULL, bit);
            if (lane == 0) out[u] = word32;
          }
        }
      }
      if (!grid_barrier(ctl, ++round, 6)) return;
      if (gtid == 0) ctl->n_stable = base + wave_count;  // everyone has read base
    } else {
      if (gtid == 0) {
        ctl->iters = t;
        atomicCAS(&ctl->status, 0, 4 /* LP_ERR_NO_FIXPOINT */);
      }
      // every block has read the last list size before the reset below clears it
      if (!grid_barrier(ctl, ++round, 6)) return;
    }

    // ---- 5. the wave's changed items and guessed rows back to the rest state
    // the bitmap wpw words per warp step, a word per lane, wpw the power of two (at most 32) that
    // spreads the words over all warps (a word per warp step made every warp wait on ~80
    // dependent loads on the 2^16-guess program: 55 us of a 137 us solve; 32 per step left most
    // warps idle where few tiles hold many changed rows)
    const long long n_dw = ((long long)cw * n_pad + 31) / 32;
    int wpw = 1;
    while (wpw < 32 && (long long)wpw * nwarps < n_dw) wpw <<= 1;
    for (long long qb = (long long)gwarp * wpw; qb < n_dw; qb += (long long)nwarps * wpw) {
      const long long q = qb + lane;
      unsigned bits = lane < wpw && q < n_dw ? a.fr_dirty[q] : 0u;
      if (bits) a.fr_dirty[q] = 0u;
      unsigned lanes = __ballot_sync(FULL, bits != 0u);
      while (lanes) {  // uniform: the warp restores the set bits of one lane's word at a time
        const int src = __ffs(lanes) - 1;
        lanes &= lanes - 1;
        unsigned wbits = __shfl_sync(FULL, bits, src);
        while (wbits) {
          const int b = __ffs(wbits) - 1;
          wbits &= wbits - 1;
          const long long item = (qb + src) * 32 + b;
          const uint64_t v = rest_word(a, (int)(item % n_pad));
          for (int w = lane; w < W; w += 32) {
            a.X0[item * W + w] = v;
            a.X1[item * W + w] = v;
          }
        }
      }
    }
    // the guessed rows back to zero in every tile of the wave
    for (long long u = gwarp; u < a.n_guess_rows; u += nwarps) {
      const int row = __ldg(a.guess_rows + (int)u);
      for (int k = lane; k < cw * W; k += 32) {
        const long long o = ((long long)(k >> log2W) * n_pad + row) * W + (k & (W - 1));
        a.X0[o] = 0ull;
        a.X1[o] = 0ull;
      }
    }
    // every read of the list sizes and wide counts was before the last barrier
    if (gtid < 12) st[kCntGroups + gtid] = 0u;
    for (long long c = gtid; c < cw; c += nthreads) a.fr_last[c] = -1;
    if (!converged) break;  // every block takes this branch
    if (w0 + c_wave < a.n_tiles && !grid_barrier(ctl, ++round, 6)) return;
  }

  n_rows = __reduce_add_sync(FULL, n_rows);
  n_ent = __reduce_add_sync(FULL, n_ent);
  n_list = __reduce_add_sync(FULL, n_list);
  n_deps = __reduce_add_sync(FULL, n_deps);
  if (lane == 0) {
    if (n_rows) atomicAdd(&ctl->fr_rows, (unsigned long long)n_rows);
    if (n_ent) atomicAdd(&ctl->fr_entries, (unsigned long long)n_ent);
    if (n_list) atomicAdd(&ctl->fr_list, (unsigned long long)n_list);
    if (n_deps) atomicAdd(&ctl->fr_deps, (unsigned long long)n_deps);
  }
  if (gtid == 0) {
    st[kCntStamp] = stamp;
    st[kCntClean] = (unsigned)clean;
  }
  __syncthreads();  // this block's writes are issued; the next launch reads the count
  if (threadIdx.x == 0) atomicAdd(st + kCntDone, 1u);
}

}  // namespace

namespace {
__global__ void long_rows_kernel(const int32_t* __restrict__ row_ptr, int32_t n_pad, unsigned* __restrict__ mask,
                                 unsigned* __restrict__ any) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool lg = r < n_pad && row_ptr[r + 1] - row_ptr[r] >= kLongRow;
  const unsigned m = __ballot_sync(FULL, lg);
  if ((threadIdx.x & 31) == 0 && r < n_pad) {
    mask[r >> 5] = m;
    if (m) atomicOr(any, 1u);
  }
}

// words per lane: W <= 8 one (W lanes per item), W = 16 two, W = 32 four (eight lanes per item)
const void* frontier_entry(int W) {
  if (W >= 32) return (const void*)stable_frontier_kernel<4>;
  if (W == 16) return (const void*)stable_frontier_kernel<2>;
  return (const void*)stable_frontier_kernel<1>;
}
}  // namespace

cudaError_t launch_stable_frontier(const StableArgs& a, int grid, cudaStream_t s) {
  StableArgs copy = a;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(frontier_entry(a.W), dim3(grid), dim3(kFrontierBlock), params, 0, s);
}

cudaError_t build_long_rows(const int32_t* row_ptr, int32_t n_pad, unsigned* mask, unsigned* any, cudaStream_t s) {
  if (n_pad <= 0) return cudaSuccess;
  long_rows_kernel<<<(n_pad + 255) / 256, 256, 0, s>>>(row_ptr, n_pad, mask, any);
  return cudaGetLastError();
}

int stable_frontier_blocks_per_sm(int W) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, frontier_entry(W), kFrontierBlock, 0) != cudaSuccess) return 0;
  return nb;
}

}  // namespace lp

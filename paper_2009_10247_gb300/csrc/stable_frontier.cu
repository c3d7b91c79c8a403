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
// Between solves the buffers rest in that state -- fact rows all ones, every other row zero, in
// both buffers -- and a solve leaves them so: a bitmap records every item that changed, and after
// Algorithm 3 those items and the guessed rows are written back. The first solve on a handle (or
// after a launch that did not finish, or after the layout changed) writes the rest state in full.
// A record in fr_cnt tells the next launch whether it can trust the buffers: the layout tag, the
// grid size, and how many blocks of the last launch finished.
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
constexpr unsigned kStampLimit = 0xF0000000u;

__device__ __forceinline__ uint64_t rest_word(int tag) { return tag == -2 ? ~0ull : 0ull; }

// Appends to a work list staged per warp in shared memory: the winners of a step go to the
// warp's 64-slot buffer, and the list gets them 32 at a time with one atomic on its counter (all
// warps of the grid append to the same counter; one atomic per step serialized on it). All lanes
// call both functions with the same n.
__device__ __forceinline__ void staged_append(int* buf, int& n, bool flag, int value, int32_t* list, unsigned* cnt,
                                              int lane) {
  const unsigned m = __ballot_sync(FULL, flag);
  if (flag) buf[n + __popc(m & ((1u << lane) - 1u))] = value;
  n += __popc(m);
  __syncwarp();
  if (n >= 32) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(cnt, 32u);
    base = __shfl_sync(FULL, base, 0);
    list[base + lane] = buf[lane];
    const int rest = n - 32;
    const int moved = lane < rest ? buf[32 + lane] : 0;
    __syncwarp();
    if (lane < rest) buf[lane] = moved;
    n = rest;
    __syncwarp();
  }
}
__device__ __forceinline__ void staged_flush(int* buf, int& n, int32_t* list, unsigned* cnt, int lane) {
  if (n > 0) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(cnt, (unsigned)n);
    base = __shfl_sync(FULL, base, 0);
    if (lane < n) list[base + lane] = buf[lane];
    n = 0;
  }
  __syncwarp();
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
// entries' words for a rule row, OR for an OR row or a self-loop, 0 for an empty row; E entries
// per step (their column loads, then their gathers: four entries, two with four words per lane).
// *n_entries grows by the row's length.
template <int WPL>
__device__ __forceinline__ void eval_row_words(const StableArgs& a, const uint64_t* src, int row, int w0,
                                               uint64_t (&acc)[WPL], unsigned* n_entries) {
  constexpr int E = WPL >= 4 ? 2 : 4;
  const int beg = __ldg(a.row_ptr + row), end = __ldg(a.row_ptr + row + 1);
  const bool any = (__ldg(a.any_mask + (row >> 5)) >> (row & 31)) & 1u;
  const uint64_t ident = any ? 0ull : ~0ull;
#pragma unroll
  for (int j = 0; j < WPL; j++) acc[j] = end > beg ? ident : 0ull;
  for (int e = beg; e < end; e += E) {
    int cc[E];
#pragma unroll
    for (int q = 0; q < E; q++) cc[q] = e + q < end ? __ldg(a.col + e + q) : -1;
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
  *n_entries += (unsigned)(end - beg);
}

// WPL: words per lane in the iterations. An item (W words) takes W / WPL lanes, so a warp
// evaluates 32 WPL / W items at once: with W = 32, four items of eight lanes, four words each.
template <int WPL>
__global__ void __launch_bounds__(kStableBlock, 4) stable_frontier_kernel(StableArgs a) {
  __shared__ long long s_base;
  __shared__ int s_stage[kStableBlock / 32][64];  // per-warp list staging
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
  const unsigned subm = W == 32 ? FULL : (((1u << W) - 1u) << (sub * W));
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
    st[0] = st[1] = st[2] = 0u;
  }
  for (long long c = gtid; c < a.fr_tiles; c += nthreads) a.fr_last[c] = -1;
  if (clean < c_wave) {  // tiles clean .. c_wave - 1 into the rest state
    const long long i0 = (long long)clean * n_pad, i1 = (long long)c_wave * n_pad;
    for (long long g = gwarp; i0 + g * rpw < i1; g += nwarps) {
      const long long item = i0 + g * rpw + sub;
      if (item < i1) {
        const uint64_t v = rest_word(__ldg(a.row_tag + (int)(item % n_pad)));
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

    // ---- 1. M_0 of the guessed rows, and the first list: fact and guessed rows and the rows
    // referring to them, in every tile of the wave. A (seed row, tile) pair per eight lanes,
    // four pairs per warp.
    {
      int* const buf = s_stage[threadIdx.x >> 5];
      int n_staged = 0;
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
        }
        if (tg >= 0)  // a guessed row: its words of M_0 in this tile
          for (int w = gl; w < W; w += 8)
            a.X0[((long long)c * n_pad + row) * W + w] = m0_word(tg, gw0 + (long long)c * W + w, a);
        const int steps = (int)__reduce_max_sync(FULL, (unsigned)((per + 7) >> 3));
        for (int s2 = 0; s2 < steps; s2++) {
          const int d = 8 * s2 + gl;
          bool win = false;
          int item = 0;
          if (d < per) {
            item = c * n_pad + (d == 0 ? row : __ldg(a.t_idx + tb + d - 1));
            win = atomicExch(a.mark + item, stamp) != stamp;
          }
          staged_append(buf, n_staged, win, item, a.fr_list, st + 0, lane);
        }
      }
      staged_flush(buf, n_staged, a.fr_list, st + 0, lane);
    }
    if (!grid_barrier(ctl, ++round, 6)) return;

    // ---- 2. the iterations
    const uint64_t* fin = a.X0;
    int t = 0;
    bool converged = false;
    for (; t < a.max_iters; ++t) {
      const uint64_t* src = (t & 1) ? a.X1 : a.X0;
      uint64_t* dst = (t & 1) ? a.X0 : a.X1;
      const int32_t* cur = a.fr_list + (size_t)(t & 1) * cap_items;
      int32_t* nxt = a.fr_list + (size_t)((t + 1) & 1) * cap_items;
      unsigned* nxt_cnt = st + (t + 1) % 3;
      const unsigned nstamp = stamp + (unsigned)t + 1u;
      // slot (t + 2) % 3 was last read as iteration t - 1's list size, before the last barrier
      if (gtid == 0) st[(t + 2) % 3] = 0u;
      const long long n_cur = ld_volatile(st + t % 3);
      int* const buf = s_stage[threadIdx.x >> 5];
      int n_staged = 0;
      for (long long g = gwarp; g * ipw < n_cur; g += nwarps) {
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
          unsigned ne = 0;
          eval_row_words<WPL>(a, src + (size_t)c * tile_words, row, il * WPL, acc, &ne);
#pragma unroll
          for (int j = 0; j < WPL; j++) {
            dst[o + j] = acc[j];
            differs |= acc[j] != old[j];
          }
          if (il == 0) {
            n_rows++;
            n_ent += ne;
          }
        }
        const unsigned diff = __ballot_sync(FULL, differs);
        const bool ch = item >= 0 && (diff & imask) != 0u;
        int per = 0;
        if (ch) {
          per = 1 + te - tb;
          if (il == 0) {
            atomicOr(a.fr_dirty + (item >> 5), 1u << (item & 31));
            atomicMax(a.fr_last + c, t);
            n_list++;
            n_deps += (unsigned)(per - 1);
          }
        }
        // the item and the rows referring to it, lpi lanes at a time
        const int steps = __reduce_max_sync(FULL, (unsigned)((per + lpi - 1) / lpi));
        for (int s = 0; s < steps; s++) {
          const int d = s * lpi + il;
          bool win = false;
          int it2 = 0;
          if (d < per) {
            it2 = c * n_pad + (d == 0 ? row : __ldg(a.t_idx + tb + d - 1));
            win = atomicExch(a.mark + it2, nstamp) != nstamp;
          }
          staged_append(buf, n_staged, win, it2, nxt, nxt_cnt, lane);
        }
      }
      staged_flush(buf, n_staged, nxt, nxt_cnt, lane);
      if (!grid_barrier(ctl, ++round, 6)) return;
      fin = dst;
      if (ld_volatile(nxt_cnt) == 0u) {
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
    const long long n_dw = ((long long)cw * n_pad + 31) / 32;
    for (long long q = gwarp; q < n_dw; q += nwarps) {
      unsigned bits = 0u;
      if (lane == 0) {
        bits = a.fr_dirty[q];
        if (bits) a.fr_dirty[q] = 0u;
      }
      bits = __shfl_sync(FULL, bits, 0);
      while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        const long long item = q * 32 + b;
        const uint64_t v = rest_word(__ldg(a.row_tag + (int)(item % n_pad)));
        for (int w = lane; w < W; w += 32) {
          a.X0[item * W + w] = v;
          a.X1[item * W + w] = v;
        }
      }
    }
    for (long long rb = (long long)gwarp * 32; rb < n_pad; rb += (long long)nwarps * 32) {
      const long long r = rb + lane;
      const int tag = r < n_pad ? __ldg(a.row_tag + r) : -1;
      unsigned m = __ballot_sync(FULL, tag >= 0);
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const long long row = rb + b;
        for (int k = lane; k < cw * W; k += 32) {
          const long long o = ((long long)(k >> log2W) * n_pad + row) * W + (k & (W - 1));
          a.X0[o] = 0ull;
          a.X1[o] = 0ull;
        }
      }
    }
    if (gtid < 3) st[gtid] = 0u;  // every read of the list sizes was before the last barrier
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
  return cudaLaunchCooperativeKernel(frontier_entry(a.W), dim3(grid), dim3(kStableBlock), params, 0, s);
}

int stable_frontier_blocks_per_sm(int W) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, frontier_entry(W), kStableBlock, 0) != cudaSuccess) return 0;
  return nb;
}

}  // namespace lp

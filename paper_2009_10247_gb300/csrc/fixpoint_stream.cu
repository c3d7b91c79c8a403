// fixpoint_stream.cu -- Algorithm 1 as a persistent kernel fed by bulk asynchronous copies.
//
// Same loop as fixpoint.cu (v0 of Def. 4, u = theta(M_P v) until u = v, projection), laid out
// for GB300 so that evaluating a 32-row word touches shared memory only:
//  * one 1024-thread CTA per SM owns a contiguous range of "groups" (<= 64 words of 32 rows).
//    A producer thread copies each group's word headers, row descriptors and rule entries
//    with cp.async.bulk into a ring of 32 KiB stages guarded by mbarriers; 31 consumer warps
//    evaluate the words. That part of a stage never changes, so the producer prefetches the
//    next iteration's first groups while the grid meets at its barrier. Each stage also gets
//    the slice of the current vector that holds the group's OR rows' new atoms, copied by the
//    producer after the barrier (a second arrival on the stage's mbarrier).
//  * every rule-row entry is an original or barred atom, and those atoms form the first rows
//    of the internal order, most referenced first. After each grid barrier every CTA copies
//    that prefix of the vector into shared memory (as much as fits), so rule rows' bit
//    gathers are shared-memory reads.
//  * each CTA keeps the words it writes in shared memory too; a self-loop reads its own bit
//    from there.
//  * in the default mode the iterates only grow (the initial vector holds self-loop rows only,
//    and theta is monotone), so u = v exactly when both have the same number of true rows:
//    the kernel counts true rows instead of comparing words. With an arbitrary initial vector
//    (LP_ROWS) it compares every word with its previous value.
//
// Rows (compile.cpp builds the layout):
//   rule row  (entries 1/m): true iff all m listed body atoms are true;
//   OR-rule row (entries 1): true iff one of its new atoms is true; those atoms are a
//             contiguous bit range (the OR rows' new atoms are laid out in OR-row order), so
//             the row stores only its length;
//   self-loop (a_ii = 1, facts and barred atoms): its own bit.
// That is theta(M_P v) of Def. 5 row by row, exactly.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "kernels.h"

namespace lp {

constexpr int kStreamThreads = 1024;
constexpr int kConsumerWarps = kStreamThreads / 32 - 1;
constexpr int kStages = 3;
constexpr int kStageRegion = kStages * kStageBytes;
constexpr int kStageXOff = kStageHdrBytes + kStageDescBytes;
constexpr int kStageColOff = kStageXOff + kStageXBytes;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Test the phase; a thread whose phase is not complete is suspended (not spinning, so it
// takes no issue slots) until the phase completes or the hint of kSuspendNs expires.
constexpr unsigned kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint32_t lds32(unsigned addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// Bounded wait on an mbarrier phase; false when the grid is aborting or the wait timed out
// (then the abort flag and LP_ERR_TIMEOUT are recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, DeviceCtl* ctl) {
  unsigned polls = 0;
  unsigned long long t0 = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++polls;
    if (polls == 1) t0 = global_ns();
    if (polls > 1) {
      if (ld_volatile(&ctl->abort)) return false;
      if (global_ns() - t0 > kWaitLimitNs) {
        atomicExch(&ctl->abort, 1u);
        atomicCAS(&ctl->status, 0, LP_ERR_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

struct StreamArgs {
  const uint32_t* desc;
  const int32_t* word_hdr;  // 2 per word
  const int32_t* and_col;
  const int32_t* groups;    // kGroupInts per group
  int32_t n_groups;
  int32_t xs_words;         // words of the vector staged in shared memory (multiple of 4)
  int32_t sec_a_words;      // words holding the rows rule rows refer to: ceil(n_sec_a / 32)
  int32_t own_words;        // shared-memory words for the CTA's own output words (multiple of 4)
  int32_t monotone;         // 1: convergence by true-row counts (default mode)
  uint32_t* x0;
  uint32_t* x1;
  int32_t n_words;
  int32_t max_iters;
  DeviceCtl* ctl;
  const uint64_t* init;
  const int32_t* fact_row;
  const int32_t* fact_owner;
  int32_t n_facts;
  const uint64_t* fact_mask;
  int32_t n_atom_words;
  const uint64_t* rows_init;
  const int32_t* inv;
  int32_t n_prime;
  uint64_t* out;
  const int32_t* perm;
  int32_t n_out;
};

// Word i of the current vector: from the shared-memory copy when staged there.
struct XView {
  const uint32_t* xs;   // shared
  const uint32_t* src;  // global
  int xs_words;
  __device__ __forceinline__ uint32_t operator[](int i) const { return i < xs_words ? xs[i] : src[i]; }
};

// Where a word finds what it reads besides the rule entries.
struct WordCtx {
  const uint32_t* or_src;  // vector words holding the OR rows' new atoms (stage slice or global)
  int or_shift;            // bit index of or_src[0] in the vector
  uint32_t self_word;      // the word's own previous value
  int zero_j;              // a gather index whose bit is always 0 (kAllSmem)
};

// theta of the 32 rows of a word whose rows all have <= 32 entries; each descriptor carries
// its row's offset. col points at the word's first rule entry, or_base is the word's first
// new atom. Rule entries are gathered 32 per ballot (lanes past the word's last entry read a
// bit that is always 0) and chunk c's ballot is kept in lane c; a rule row then reads its
// (at most 32) bits from two ballots with one funnel shift, an OR row tests its contiguous
// range of new atoms with one funnel shift, a self-loop reads its own bit.
// kAllSmem: every gathered atom lies in the shared-memory copy of the vector.
template <bool kAllSmem>
__device__ __noinline__ uint32_t stream_word_fast(int lane, uint32_t d, uint32_t hflags, int or_base,
                                                  const int32_t* col, const XView& x, const WordCtx& ctx) {
  const uint32_t kind = d >> 30;
  const int off = (int)((d >> 6) & 0xffffffu);
  const int len = (int)(d & 63u);
  const bool rule = kind == SK_RULE;
  const int a_total = (int)__reduce_max_sync(FULL, rule ? (unsigned)(off + len) : 0u);
  const uint32_t want = __funnelshift_rc(FULL, 0u, 32 - len);  // len low bits set (len <= 32)
  bool val = false;
  if (a_total > 0) {  // warp-uniform
    uint32_t mymask = 0;
    const int nch = (a_total + 31) >> 5;
    for (int c = 0; c < nch; c += 2) {
      const int e0 = (c << 5) + lane, e1 = e0 + 32;
      uint32_t b0, b1;
      if (kAllSmem) {
        const int j0 = e0 < a_total ? col[e0] : ctx.zero_j;
        const int j1 = e1 < a_total ? col[e1] : ctx.zero_j;
        const uint32_t w0 = x.xs[j0 >> 5], w1 = x.xs[j1 >> 5];
        b0 = __funnelshift_r(w0, w0, j0) & 1u;
        b1 = __funnelshift_r(w1, w1, j1) & 1u;
      } else {
        b0 = b1 = 0u;
        if (e0 < a_total) {
          const int j0 = col[e0];
          const uint32_t w0 = x[j0 >> 5];
          b0 = __funnelshift_r(w0, w0, j0) & 1u;
        }
        if (e1 < a_total) {
          const int j1 = col[e1];
          const uint32_t w1 = x[j1 >> 5];
          b1 = __funnelshift_r(w1, w1, j1) & 1u;
        }
      }
      const uint32_t m0 = __ballot_sync(FULL, b0);
      const uint32_t m1 = __ballot_sync(FULL, b1);
      if (lane == c) mymask = m0;
      if (lane == c + 1) mymask = m1;
    }
    const uint32_t lo = __shfl_sync(FULL, mymask, (off >> 5) & 31);
    const uint32_t hi = __shfl_sync(FULL, mymask, ((off >> 5) + 1) & 31);
    val = rule && len > 0 && (__funnelshift_r(lo, hi, off) & want) == want;
  }
  if ((hflags & kHasOr) && kind == SK_OR) {
    const int p = or_base + off - ctx.or_shift;
    const uint32_t lo = ctx.or_src[p >> 5], hi = ctx.or_src[(p + len - 1) >> 5];
    val = (__funnelshift_r(lo, hi, p) & want) != 0u;
  }
  if ((hflags & kHasSelf) && kind == SK_SELF) val = (ctx.self_word >> lane) & 1u;
  return __ballot_sync(FULL, val);
}

// The same evaluation when everything the word reads is in shared memory (the common case):
// 32-bit shared addresses and explicit shared loads. col_a: the word's first rule entry in the
// stage; xs_a: the staged vector prefix; or_a: the group's vector slice, whose first bit is
// bit or_shift of the vector.
__device__ __forceinline__ uint32_t stream_word_smem(int lane, uint32_t d, uint32_t hflags, int or_base,
                                                     unsigned col_a, unsigned xs_a, unsigned or_a, int or_shift,
                                                     uint32_t self_word, int zero_j) {
  const uint32_t kind = d >> 30;
  const int off = (int)((d >> 6) & 0xffffffu);
  const int len = (int)(d & 63u);
  const bool rule = kind == SK_RULE;
  const int a_total = (int)__reduce_max_sync(FULL, rule ? (unsigned)(off + len) : 0u);
  const uint32_t want = __funnelshift_rc(FULL, 0u, 32 - len);  // len low bits set (len <= 32)
  bool val = false;
  if (a_total > 0) {  // warp-uniform
    uint32_t mymask = 0;
    const int nch = (a_total + 31) >> 5;
    for (int c = 0; c < nch; c += 2) {
      const int e0 = (c << 5) + lane, e1 = e0 + 32;
      const unsigned j0 = e0 < a_total ? lds32(col_a + 4u * (unsigned)e0) : (unsigned)zero_j;
      const unsigned j1 = e1 < a_total ? lds32(col_a + 4u * (unsigned)e1) : (unsigned)zero_j;
      const uint32_t w0 = lds32(xs_a + ((j0 >> 3) & ~3u));
      const uint32_t w1 = lds32(xs_a + ((j1 >> 3) & ~3u));
      const uint32_t m0 = __ballot_sync(FULL, __funnelshift_r(w0, w0, j0) & 1u);
      const uint32_t m1 = __ballot_sync(FULL, __funnelshift_r(w1, w1, j1) & 1u);
      mymask = lane == c ? m0 : mymask;
      mymask = lane == c + 1 ? m1 : mymask;
    }
    const uint32_t lo = __shfl_sync(FULL, mymask, (off >> 5) & 31);
    const uint32_t hi = __shfl_sync(FULL, mymask, ((off >> 5) + 1) & 31);
    val = rule && len > 0 && (__funnelshift_r(lo, hi, off) & want) == want;
  }
  if ((hflags & kHasOr) && kind == SK_OR) {
    const unsigned p = (unsigned)(or_base + off - or_shift);
    const uint32_t lo = lds32(or_a + ((p >> 3) & ~3u));
    const uint32_t hi = lds32(or_a + (((p + (unsigned)len - 1u) >> 3) & ~3u));
    val = (__funnelshift_r(lo, hi, p) & want) != 0u;
  }
  if ((hflags & kHasSelf) && kind == SK_SELF) val = (self_word >> lane) & 1u;
  return __ballot_sync(FULL, val);
}

// theta of the 32 rows of a long word (some row has more than 32 entries): offsets come from
// prefix sums of the row lengths. col points at the word's first rule entry.
__device__ __noinline__ uint32_t stream_word_long(int lane, uint32_t d, int or_base, const int32_t* col,
                                                  const XView& x, uint32_t self_word) {
  const uint32_t kind = d >> 30;
  const int len = (int)(d & 0x3fffffffu);
  const int and_len = kind == SK_RULE ? len : 0;
  const int or_len = kind == SK_OR ? len : 0;
  int a_inc = and_len, o_inc = or_len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y1 = __shfl_up_sync(FULL, a_inc, o);
    const int y2 = __shfl_up_sync(FULL, o_inc, o);
    if (lane >= o) {
      a_inc += y1;
      o_inc += y2;
    }
  }
  const int a_off = a_inc - and_len;
  const int o_off = o_inc - or_len;
  const int a_total = __shfl_sync(FULL, a_inc, 31);
  int cnt = 0;  // true entries of this lane's rule row
  for (int c = 0; c < a_total; c += 32) {
    const int e = c + lane;
    uint32_t bit = 0;
    if (e < a_total) {
      const int jj = col[e];
      bit = (x[jj >> 5] >> (jj & 31)) & 1u;
    }
    const uint32_t m = __ballot_sync(FULL, bit);
    const int lo = max(a_off - c, 0), hi = min(a_off + and_len - c, 32);
    if (hi > lo) cnt += __popc(m & ((hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo)));
  }
  bool val = kind == SK_RULE && len > 0 && cnt == len;
  if (kind == SK_OR) {  // one of the row's new atoms, a contiguous bit range (global reads)
    bool any = false;
    int p = or_base + o_off, rem = len;
    while (rem > 0 && !any) {
      const int bpos = p & 31;
      const int take = min(32 - bpos, rem);
      const uint32_t want = take == 32 ? FULL : ((1u << take) - 1u);
      any = ((x.src[p >> 5] >> bpos) & want) != 0u;
      p += take;
      rem -= take;
    }
    val = any;
  } else if (kind == SK_SELF) {
    val = (self_word >> lane) & 1u;
  }
  return __ballot_sync(FULL, val);
}

__global__ void __launch_bounds__(kStreamThreads, 1) fixpoint_stream_kernel(StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ int s_flag;
  __shared__ int s_fail;
  __shared__ unsigned long long s_count;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  const int gwarp = gtid >> 5;
  const int nwarps = nthreads >> 5;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;
  uint32_t* xs = reinterpret_cast<uint32_t*>(smem + kStageRegion);
  uint32_t* own = xs + a.xs_words;

  // this CTA's groups and the words they cover
  const int g_beg = (int)((long long)a.n_groups * blockIdx.x / gridDim.x);
  const int g_end = (int)((long long)a.n_groups * (blockIdx.x + 1) / gridDim.x);
  const int ng = g_end - g_beg;
  const int own0 = ng > 0 ? __ldg(a.groups + kGroupInts * g_beg) : 0;
  const int own1 = ng > 0 ? __ldg(a.groups + kGroupInts * (g_end - 1) + 1) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full_bar[s], 2);  // static part + vector slice
      mbar_init(&empty_bar[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    s_count = 0;
  }
  __syncthreads();

  // ---- initial vector (as in fixpoint.cu); in the default mode count its true rows
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
    unsigned long long mine = 0;
    for (int i = gtid; i < a.n_facts; i += nthreads) {
      const int own_atom = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own_atom >> 6] >> (own_atom & 63)) & 1ull) : true;
      if (sel) {
        const uint32_t bit = 1u << (a.fact_row[i] & 31);
        if (!(atomicOr(a.x0 + (a.fact_row[i] >> 5), bit) & bit)) mine++;
      }
    }
    if (mine) atomicAdd(&ctl->init_count, mine);
    if (a.init)
      for (int i = gtid; i < a.n_atom_words; i += nthreads)
        if (a.init[i] & ~a.fact_mask[i]) atomicCAS(&ctl->status, 0, LP_ERR_INVALID);
  }
  bool ok = grid_barrier(ctl, ++round, LP_ERR_TIMEOUT);
  if (threadIdx.x == 0) s_flag = (int)ld_volatile((const unsigned*)&ctl->status);
  __syncthreads();
  if (s_flag != 0) ok = false;  // bad initial vector: nothing to iterate
  unsigned long long prev_count = ld_volatile64(&ctl->init_count);
  for (int i = threadIdx.x; i < own1 - own0; i += blockDim.x) own[i] = __ldcg(a.x0 + own0 + i);

  // ---- producer (thread 0): static stage parts run ahead; vector slices follow the barrier
  long long q_static = 0, q_dyn = 0;
  auto group_of = [&](long long q) { return a.groups + kGroupInts * (g_beg + (int)(q % ng)); };
  auto issue_static = [&](long long q) -> bool {
    const int s = (int)(q % kStages);
    if (q >= kStages && !mbar_wait(&empty_bar[s], (unsigned)(((q / kStages) + 1) & 1), ctl)) return false;
    const int32_t* gr = group_of(q);
    const int w0 = __ldg(gr), w1 = __ldg(gr + 1), col0 = __ldg(gr + 2), ncol = __ldg(gr + 3);
    unsigned char* st = smem + (size_t)s * kStageBytes;
    const unsigned hb = 8u * (unsigned)(w1 - w0), db = 128u * (unsigned)(w1 - w0);
    const unsigned cb = ncol > 0 ? 4u * (unsigned)ncol : 0u;
    mbar_arrive_expect_tx(&full_bar[s], hb + db + cb);
    bulk_copy_g2s(st, a.word_hdr + 2 * w0, hb, &full_bar[s]);
    bulk_copy_g2s(st + kStageHdrBytes, a.desc + 32 * w0, db, &full_bar[s]);
    if (cb) bulk_copy_g2s(st + kStageColOff, a.and_col + col0, cb, &full_bar[s]);
    return true;
  };
  auto issue_dyn = [&](long long q, const uint32_t* src) {
    const int s = (int)(q % kStages);
    const int32_t* gr = group_of(q);
    const int xw0 = __ldg(gr + 4), nxw = __ldg(gr + 5);
    const unsigned xb = nxw > 0 ? 4u * (unsigned)nxw : 0u;
    mbar_arrive_expect_tx(&full_bar[s], xb);
    if (xb) bulk_copy_g2s(smem + (size_t)s * kStageBytes + kStageXOff, src + xw0, xb, &full_bar[s]);
  };

  const uint32_t* fin = a.x0;
  int it = 0;
  bool converged = false;
  for (; ok && it < a.max_iters; ++it) {
    const uint32_t* src = (it & 1) ? a.x1 : a.x0;
    uint32_t* dst = (it & 1) ? a.x0 : a.x1;
    // the vector slices of the stages prefetched during the last iteration can go now
    if (threadIdx.x == 0 && ng > 0) {
      // order the last iteration's writes (seen through the grid barrier) before the bulk
      // copies that read the vector
      asm volatile("fence.proxy.async;" ::: "memory");
      const long long hi = (long long)(it + 1) * ng;
      while (q_dyn < q_static && q_dyn < hi) issue_dyn(q_dyn++, src);
    }
    // stage the vector's prefix (the atoms rule rows refer to) in shared memory; the word after
    // it is kept at zero (the gather target of lanes without an entry). Four loads in flight
    // per thread.
    {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      uint4* d4 = reinterpret_cast<uint4*>(xs);
      const int n4 = a.xs_words >> 2;
      const int copy_words = min(a.sec_a_words, a.xs_words);
      for (int base = threadIdx.x; base < n4; base += 4 * (int)blockDim.x) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int i = base + u * (int)blockDim.x;
          if (i < n4) v[u] = __ldcg(s4 + i);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int i = base + u * (int)blockDim.x;
          if (i < n4) {
            const int w0 = 4 * i;
            if (w0 + 0 >= copy_words) v[u].x = 0u;
            if (w0 + 1 >= copy_words) v[u].y = 0u;
            if (w0 + 2 >= copy_words) v[u].z = 0u;
            if (w0 + 3 >= copy_words) v[u].w = 0u;
            d4[i] = v[u];
          }
        }
      }
    }
    __syncthreads();
    // only the copied words are the vector's; the staged words after them read as zero
    const XView x{xs, src, min(a.sec_a_words, a.xs_words)};
    const bool all_smem = a.xs_words > a.sec_a_words;
    bool changed = false;
    unsigned long long ones = 0;
    if (ng > 0) {
      if (warp == 0) {
        if (lane == 0) {
          const long long hi = (long long)(it + 1) * ng;
          bool good = true;
          while (good && q_static < hi) {
            good = issue_static(q_static);
            if (!good) break;
            issue_dyn(q_static, src);
            q_dyn = ++q_static;
          }
          // the next iteration's first stages (static part only)
          const long long target = (it + 1 < a.max_iters) ? hi + min(ng, kStages) : hi;
          while (good && q_static < target) {
            good = issue_static(q_static);
            if (good) ++q_static;
          }
          if (!good) s_fail = 1;
        }
      } else {
        const int cw = warp - 1;
        for (int k = 0; k < ng; k++) {
          const long long q = (long long)it * ng + k;
          const int s = (int)(q % kStages);
          if (!mbar_wait(&full_bar[s], (unsigned)((q / kStages) & 1), ctl)) {
            if (lane == 0) s_fail = 1;
            break;
          }
          const int32_t* gr = a.groups + kGroupInts * (g_beg + k);
          const int w0 = __ldg(gr), w1 = __ldg(gr + 1), col0 = __ldg(gr + 2), ncol = __ldg(gr + 3);
          const int xw0 = __ldg(gr + 4), nxw = __ldg(gr + 5);
          const unsigned char* st = smem + (size_t)s * kStageBytes;
          const int2* hdr = reinterpret_cast<const int2*>(st);
          const uint32_t* dsc = reinterpret_cast<const uint32_t*>(st + kStageHdrBytes);
          const uint32_t* sx = reinterpret_cast<const uint32_t*>(st + kStageXOff);
          const int32_t* scol = reinterpret_cast<const int32_t*>(st + kStageColOff);
          WordCtx ctx;
          ctx.or_src = nxw >= 0 ? sx : src;
          ctx.or_shift = nxw >= 0 ? xw0 * 32 : 0;
          ctx.zero_j = a.sec_a_words * 32;
          const bool smem_path = all_smem && ncol >= 0 && nxw >= 0;
          const unsigned st_a = smem_u32(st), xs_a = smem_u32(xs);
          for (int w = w0 + cw; w < w1; w += kConsumerWarps) {
            const int2 h = hdr[w - w0];
            const uint32_t d = dsc[(w - w0) * 32 + lane];
            const uint32_t hflags = (uint32_t)h.x & (kHasOr | kHasSelf);
            const int hcol = (int)((uint32_t)h.x & ~(kHasOr | kHasSelf));
            const int32_t* colp = ncol >= 0 ? scol + (hcol - col0) : a.and_col + hcol;
            ctx.self_word = own[w - own0];
            uint32_t u;
            if (smem_path && !((uint32_t)h.y & kLongWord))
              u = stream_word_smem(lane, d, hflags, h.y, st_a + kStageColOff + 4u * (unsigned)(hcol - col0), xs_a,
                                   st_a + kStageXOff, xw0 * 32, ctx.self_word, ctx.zero_j);
            else if ((uint32_t)h.y & kLongWord)
              u = stream_word_long(lane, d, (int)((uint32_t)h.y & ~kLongWord), colp, x, ctx.self_word);
            else if (all_smem)
              u = stream_word_fast<true>(lane, d, hflags, h.y, colp, x, ctx);
            else
              u = stream_word_fast<false>(lane, d, hflags, h.y, colp, x, ctx);
            if (lane == 0) {
              dst[w] = u;
              if (a.monotone) ones += __popc(u);
              else changed |= (u != ctx.self_word);
              own[w - own0] = u;
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty_bar[s]);
        }
      }
    }
    if (a.monotone && ones) atomicAdd(&s_count, ones);
    const int any_changed = __syncthreads_or(changed);
    if (threadIdx.x == 0) {
      if (s_fail) {
        atomicExch(&ctl->abort, 1u);
        atomicCAS(&ctl->status, 0, LP_ERR_TIMEOUT);
      }
      if (a.monotone) {
        if (s_count) atomicAdd(&ctl->count[it % 3], s_count);
        s_count = 0;
        if (blockIdx.x == 0) ctl->count[(it + 1) % 3] = 0ull;  // nobody reads or writes it now
      } else {
        if (any_changed) atomicOr(&ctl->flag[it % 3], 1u);
        if (blockIdx.x == 0) ctl->flag[(it + 1) % 3] = 0u;
      }
    }
    if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) {
      ok = false;
      break;
    }
    bool again;
    if (a.monotone) {
      const unsigned long long now = ld_volatile64(&ctl->count[it % 3]);
      again = now != prev_count;  // the iterates only grow: same count, same vector
      prev_count = now;
    } else {
      if (threadIdx.x == 0) s_flag = (int)ld_volatile(&ctl->flag[it % 3]);
      __syncthreads();
      again = s_flag != 0;
    }
    fin = dst;
    if (!again) {
      converged = true;
      ++it;
      break;
    }
  }
  // Stages prefetched for an iteration that did not run still have bulk copies in flight.
  // Give them their missing vector-slice arrival (zero bytes) so their phase can complete,
  // then wait (bounded) until every copy this CTA issued has landed.
  if (threadIdx.x == 0 && ng > 0) {
    for (long long q = q_dyn; q < q_static; ++q) mbar_arrive_expect_tx(&full_bar[(int)(q % kStages)], 0u);
    const long long consumed = (long long)it * ng;  // groups of iterations 0 .. it-1
    for (long long q = consumed; q < q_static; ++q)
      if (!mbar_wait(&full_bar[(int)(q % kStages)], (unsigned)((q / kStages) & 1), ctl)) break;
  }
  __syncthreads();
  if (!ok) return;
  if (gtid == 0) {
    ctl->iters = it;
    if (!converged) atomicCAS(&ctl->status, 0, LP_ERR_NO_FIXPOINT);
  }
  if (a.out) {
    uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
    const int n32 = 2 * ((a.n_out + 63) >> 6);
    for (int u = gwarp; u < n32; u += nwarps) {
      const int i = (u << 5) + lane;
      const uint32_t bit = i < a.n_out ? (fin[a.perm[i] >> 5] >> (a.perm[i] & 31)) & 1u : 0u;
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) out32[u] = word;
    }
  }
}

static int g_max_dyn_smem = -1;

static int max_dyn_smem() {
  if (g_max_dyn_smem < 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      v = 0;
    g_max_dyn_smem = v;
  }
  return g_max_dyn_smem;
}

// Shared-memory words for the CTA's own output words: the most words a CTA's groups cover.
static int own_words_for(const StreamLayout& L, int grid) {
  int most = 0;
  for (int c = 0; c < grid; c++) {
    const int gb = (int)((long long)L.n_groups * c / grid), ge = (int)((long long)L.n_groups * (c + 1) / grid);
    if (ge > gb) most = std::max(most, L.host_groups[kGroupInts * (ge - 1) + 1] - L.host_groups[kGroupInts * gb]);
  }
  return (most + 3) & ~3;
}

cudaError_t launch_fixpoint_stream(const FixArgs& f, const StreamLayout& L, int grid, cudaStream_t s) {
  const int own_words = own_words_for(L, grid);
  const int budget = max_dyn_smem() - kStageRegion - 1024 - 4 * own_words;  // 1 KiB for static shared data
  if (budget < 16) return cudaErrorInvalidConfiguration;
  const int want = ((L.n_sec_a + 31) / 32 + 1 + 3) & ~3;  // the referenced words and a zero word
  const int xs_words = std::min(want, (budget / 16) * 4);
  const size_t dyn = (size_t)kStageRegion + 4 * (size_t)(xs_words + own_words);
  cudaError_t e = set_kernel_smem((const void*)fixpoint_stream_kernel, (int)dyn, -1);
  if (e != cudaSuccess) return e;
  StreamArgs a{};
  a.desc = L.desc;
  a.word_hdr = L.word_hdr;
  a.and_col = L.and_col;
  a.groups = L.groups;
  a.n_groups = L.n_groups;
  a.xs_words = xs_words;
  a.sec_a_words = (L.n_sec_a + 31) / 32;
  a.own_words = own_words;
  a.monotone = f.rows_init ? 0 : 1;
  a.x0 = f.x0;
  a.x1 = f.x1;
  a.n_words = f.n_words;
  a.max_iters = f.max_iters;
  a.ctl = f.ctl;
  a.init = f.init;
  a.fact_row = f.fact_row;
  a.fact_owner = f.fact_owner;
  a.n_facts = f.n_facts;
  a.fact_mask = f.fact_mask;
  a.n_atom_words = f.n_atom_words;
  a.rows_init = f.rows_init;
  a.inv = f.inv;
  a.n_prime = f.n_prime;
  a.out = f.out;
  a.perm = f.perm;
  a.n_out = f.n_out;
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)fixpoint_stream_kernel, dim3(grid), dim3(kStreamThreads), params,
                                     dyn, s);
}

int fixpoint_stream_blocks_per_sm() {
  const int dyn = max_dyn_smem() - 1024;
  if (dyn <= kStageRegion) return 0;
  if (set_kernel_smem((const void*)fixpoint_stream_kernel, dyn, -1) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fixpoint_stream_kernel, kStreamThreads, (size_t)dyn) !=
      cudaSuccess)
    return 0;
  return nb;
}

}  // namespace lp

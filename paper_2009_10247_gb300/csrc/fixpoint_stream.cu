// fixpoint_stream.cu -- Algorithm 1 as a persistent kernel fed by bulk asynchronous copies.
//
// Same loop as fixpoint.cu (v0 of Def. 4, u = theta(M_P v) until u = v, projection), laid out
// for GB300:
//  * one 1024-thread CTA per SM owns a contiguous range of "groups" (<= 64 words of 32 rows
//    whose headers, row descriptors and rule entries fit a 32 KiB stage); a producer thread
//    copies them with cp.async.bulk into a ring of stages guarded by mbarriers and 31 consumer
//    warps evaluate the words. The matrix never changes, so the producer prefetches the next
//    iteration's first groups while the grid meets at its barrier.
//  * every rule-row entry is an original or barred atom, and those atoms form the first rows
//    of the internal order, most referenced first. After each grid barrier every CTA copies
//    that prefix of the current vector into shared memory (as much as fits), so the random
//    bit gathers of rule rows are shared-memory reads.
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

#include "device.cuh"
#include "internal.h"
#include "kernels.h"

namespace lp {

constexpr int kStreamThreads = 1024;
constexpr int kConsumerWarps = kStreamThreads / 32 - 1;
constexpr int kStages = 3;
constexpr int kStageRegion = kStages * kStageBytes;

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

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false when the grid is aborting or the wait timed out
// (then the abort flag and LP_ERR_TIMEOUT are recorded).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, DeviceCtl* ctl) {
  unsigned polls = 0;
  unsigned long long t0 = 0;
  while (!mbar_try_wait(bar, parity)) {
    ++polls;
    if (polls == 16) t0 = global_ns();
    if (polls > 16 && (polls & 31) == 0) {
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
  const int32_t* groups;    // 4 per group
  int32_t n_groups;
  int32_t xs_words;         // words of the vector staged in shared memory (multiple of 4)
  int32_t sec_a_words;      // words holding the rows rule rows refer to: ceil(n_sec_a / 32)
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

// theta of the 32 rows of a word whose rows all have <= 32 entries; each descriptor carries
// its row's offset. col points at the word's first rule entry, or_base is the word's first
// new atom. Rule entries are gathered 32 per ballot (lanes past the word's last entry read a
// bit that is always 0) and chunk c's ballot is kept in lane c; a rule row then reads its
// (at most 32) bits from two ballots with one funnel shift, an OR row tests its contiguous
// range of new atoms with one funnel shift, a self-loop reads its own bit.
// kAllSmem: every gathered atom lies in the shared-memory copy of the vector.
template <bool kAllSmem>
__device__ __forceinline__ uint32_t stream_word_fast(int w, int lane, uint32_t d, int or_base, const int32_t* col,
                                                     const XView& x, int zero_j) {
  const uint32_t kind = d >> 30;
  const int off = (int)((d >> 6) & 0xffffffu);
  const int len = (int)(d & 63u);
  const bool rule = kind == SK_RULE;
  const int a_total = (int)__reduce_max_sync(FULL, rule ? (unsigned)(off + len) : 0u);
  const uint32_t want = __funnelshift_rc(FULL, 0u, 32 - len);  // len low bits set (len <= 32)
  uint32_t mymask = 0;
  const int nch = (a_total + 31) >> 5;
  for (int c = 0; c < nch; c++) {
    const int e = (c << 5) + lane;
    uint32_t bit;
    if (kAllSmem) {
      const int j = e < a_total ? col[e] : zero_j;
      const uint32_t wd = x.xs[j >> 5];
      bit = __funnelshift_r(wd, wd, j) & 1u;
    } else {
      bit = 0u;
      if (e < a_total) {
        const int j = col[e];
        const uint32_t wd = x[j >> 5];
        bit = __funnelshift_r(wd, wd, j) & 1u;
      }
    }
    const uint32_t m = __ballot_sync(FULL, bit);
    if (lane == c) mymask = m;
  }
  bool val = false;
  if (a_total > 0) {  // warp-uniform: the shuffles need every lane
    const uint32_t m0 = __shfl_sync(FULL, mymask, (off >> 5) & 31);
    const uint32_t m1 = __shfl_sync(FULL, mymask, ((off >> 5) + 1) & 31);
    val = rule && len > 0 && (__funnelshift_r(m0, m1, off) & want) == want;
  }
  if (kind == SK_OR) {  // new atoms lie past the shared copy: global reads
    const int p = or_base + off;
    const uint32_t lo = x.src[p >> 5], hi = x.src[(p + len - 1) >> 5];
    val = (__funnelshift_r(lo, hi, p) & want) != 0u;
  } else if (kind == SK_SELF) {
    val = (x[w] >> lane) & 1u;
  }
  return __ballot_sync(FULL, val);
}

// theta of the 32 rows of a long word (some row has more than 32 entries): offsets come from
// prefix sums of the row lengths. col points at the word's first rule entry.
__device__ __noinline__ uint32_t stream_word_long(int w, int lane, uint32_t d, int or_base, const int32_t* col,
                                                  const XView& x) {
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
  if (kind == SK_OR) {  // one of the row's new atoms, a contiguous bit range
    bool any = false;
    int p = or_base + o_off, rem = len;
    while (rem > 0 && !any) {
      const int bpos = p & 31;
      const int take = min(32 - bpos, rem);
      const uint32_t want = take == 32 ? FULL : ((1u << take) - 1u);
      any = ((x[p >> 5] >> bpos) & want) != 0u;
      p += take;
      rem -= take;
    }
    val = any;
  } else if (kind == SK_SELF) {
    val = (x[w] >> lane) & 1u;
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

  // this CTA's groups
  const int g_beg = (int)((long long)a.n_groups * blockIdx.x / gridDim.x);
  const int g_end = (int)((long long)a.n_groups * (blockIdx.x + 1) / gridDim.x);
  const int ng = g_end - g_beg;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(&full_bar[s], 1);
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
      const int own = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own >> 6] >> (own & 63)) & 1ull) : true;
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

  // producer state (thread 0 only): next sequence number to issue
  long long q_issue = 0;
  auto issue_upto = [&](long long q_target) -> bool {
    for (; q_issue < q_target; ++q_issue) {
      const int s = (int)(q_issue % kStages);
      if (q_issue >= kStages && !mbar_wait(&empty_bar[s], (unsigned)(((q_issue / kStages) + 1) & 1), ctl))
        return false;
      const int g = g_beg + (int)(q_issue % ng);
      const int w0 = __ldg(a.groups + 4 * g), w1 = __ldg(a.groups + 4 * g + 1);
      const int col0 = __ldg(a.groups + 4 * g + 2), ncol = __ldg(a.groups + 4 * g + 3);
      unsigned char* st = smem + (size_t)s * kStageBytes;
      const unsigned hb = 8u * (unsigned)(w1 - w0), db = 128u * (unsigned)(w1 - w0);
      const unsigned cb = ncol > 0 ? 4u * (unsigned)ncol : 0u;
      mbar_arrive_expect_tx(&full_bar[s], hb + db + cb);
      bulk_copy_g2s(st, a.word_hdr + 2 * w0, hb, &full_bar[s]);
      bulk_copy_g2s(st + kStageHdrBytes, a.desc + 32 * w0, db, &full_bar[s]);
      if (cb) bulk_copy_g2s(st + kStageHdrBytes + kStageDescBytes, a.and_col + col0, cb, &full_bar[s]);
    }
    return true;
  };

  const uint32_t* fin = a.x0;
  int it = 0;
  bool converged = false;
  for (; ok && it < a.max_iters; ++it) {
    const uint32_t* src = (it & 1) ? a.x1 : a.x0;
    uint32_t* dst = (it & 1) ? a.x0 : a.x1;
    // stage the vector's prefix (the atoms rule rows refer to) in shared memory
    {
      // words [0, sec_a_words) from the vector; the word after them is kept at zero (the
      // gather target of lanes without an entry)
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      uint4* d4 = reinterpret_cast<uint4*>(xs);
      const int n4 = a.xs_words >> 2;
      const int copy_words = min(a.sec_a_words, a.xs_words);
      for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        uint4 v = __ldcg(s4 + i);
        const int w0 = 4 * i;
        if (w0 + 0 >= copy_words) v.x = 0u;
        if (w0 + 1 >= copy_words) v.y = 0u;
        if (w0 + 2 >= copy_words) v.z = 0u;
        if (w0 + 3 >= copy_words) v.w = 0u;
        d4[i] = v;
      }
    }
    __syncthreads();
    // only the copied words are the vector's; the staged words after them read as zero
    const XView x{xs, src, min(a.sec_a_words, a.xs_words)};
    const bool all_smem = a.xs_words > a.sec_a_words;  // the gathered atoms and a zero word
    const int zero_j = a.sec_a_words * 32;              // a bit of that always-zero word
    bool changed = false;
    unsigned long long ones = 0;
    if (ng > 0) {
      if (warp == 0) {
        if (lane == 0) {
          // this iteration's groups, then the next iteration's first stages
          const long long next = (long long)(it + 1) * ng;
          const long long target = (it + 1 < a.max_iters) ? next + min(ng, kStages) : next;
          if (!issue_upto(target)) s_fail = 1;
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
          const int g = g_beg + k;
          const int w0 = __ldg(a.groups + 4 * g), w1 = __ldg(a.groups + 4 * g + 1);
          const int col0 = __ldg(a.groups + 4 * g + 2), ncol = __ldg(a.groups + 4 * g + 3);
          const unsigned char* st = smem + (size_t)s * kStageBytes;
          const int2* hdr = reinterpret_cast<const int2*>(st);
          const uint32_t* dsc = reinterpret_cast<const uint32_t*>(st + kStageHdrBytes);
          const int32_t* scol = reinterpret_cast<const int32_t*>(st + kStageHdrBytes + kStageDescBytes);
          for (int w = w0 + cw; w < w1; w += kConsumerWarps) {
            const int2 h = hdr[w - w0];
            const uint32_t d = dsc[(w - w0) * 32 + lane];
            const int32_t* colp = ncol >= 0 ? scol + (h.x - col0) : a.and_col + h.x;
            uint32_t u;
            if ((uint32_t)h.y & kLongWord)
              u = stream_word_long(w, lane, d, (int)((uint32_t)h.y & ~kLongWord), colp, x);
            else if (all_smem)
              u = stream_word_fast<true>(w, lane, d, h.y, colp, x, zero_j);
            else
              u = stream_word_fast<false>(w, lane, d, h.y, colp, x, zero_j);
            if (lane == 0) {
              dst[w] = u;
              if (a.monotone) ones += __popc(u);
              else changed |= (u != x[w]);
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
  // copies still in flight (prefetched stages nobody will consume) must land before exit
  if (threadIdx.x == 0 && ng > 0) {
    const long long consumed = (long long)it * ng;  // groups of iterations 0 .. it-1
    for (long long q = consumed; q < q_issue; ++q)
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

// Words of the vector staged in shared memory (a multiple of 4) for a program whose first
// n_sec_a rows are the atoms rule rows gather: those words and one word kept at zero.
static int stream_xs_words(int n_sec_a) {
  const int budget_bytes = max_dyn_smem() - kStageRegion - 1024;  // room for static shared data
  const int want = ((n_sec_a + 31) / 32 + 1 + 3) & ~3;
  const int fit = budget_bytes > 0 ? (budget_bytes / 16) * 4 : 0;
  return want < fit ? want : fit;
}

int fixpoint_stream_xs_words(int n_sec_a) { return stream_xs_words(n_sec_a); }

cudaError_t launch_fixpoint_stream(const FixArgs& f, const StreamLayout& L, int grid, cudaStream_t s) {
  const int xs_words = stream_xs_words(L.n_sec_a);
  const size_t dyn = (size_t)kStageRegion + 4 * (size_t)xs_words;
  cudaError_t e = cudaFuncSetAttribute(fixpoint_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  StreamArgs a{};
  a.desc = L.desc;
  a.word_hdr = L.word_hdr;
  a.and_col = L.and_col;
  a.groups = L.groups;
  a.n_groups = L.n_groups;
  a.xs_words = xs_words;
  a.sec_a_words = (L.n_sec_a + 31) / 32;
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
  if (cudaFuncSetAttribute(fixpoint_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fixpoint_stream_kernel, kStreamThreads, (size_t)dyn) !=
      cudaSuccess)
    return 0;
  return nb;
}

}  // namespace lp

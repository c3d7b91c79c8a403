// fixpoint_stream.cu -- Algorithm 1 as a persistent kernel fed by bulk asynchronous copies.
//
// Same loop as fixpoint.cu (v0 of Def. 4, u = theta(M_P v) until u = v, projection), with the
// matrix streamed through shared memory: one CTA per SM owns a contiguous range of "groups"
// (<= 64 words of 32 rows whose data fit a 32 KiB stage). A producer thread copies each
// group's word headers, row descriptors and rule-row entries with cp.async.bulk into a ring
// of stages guarded by mbarriers; 15 consumer warps evaluate the words. The matrix never
// changes, so the producer keeps prefetching the next iteration's first groups while the
// consumers finish the current one and the grid meets at its barrier.
//
// Rows (compile.cpp builds the layout):
//   rule row  (entries 1/m): true iff all m listed body atoms are true;
//   OR-rule row (entries 1): true iff one of its new atoms is true; those atoms are a
//             contiguous bit range (the OR rows' new atoms are laid out in OR-row order), so
//             the row stores only its length;
//   self-loop (a_ii = 1, facts and barred atoms): its own bit.
// That is theta(M_P v) of Def. 5 row by row, exactly.
//
// Per word a warp walks the word's rule entries 32 at a time (coalesced shared-memory reads),
// gathers the 32 bits and keeps each chunk's ballot in one lane; every lane then tests its
// own row's bit range with two shuffles.
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"
#include "kernels.h"

namespace lp {

constexpr int kStreamThreads = 512;
constexpr int kConsumerWarps = kStreamThreads / 32 - 1;
constexpr int kStages = 4;

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

// theta of the 32 rows of word w. col points at the word's first rule entry.
__device__ __forceinline__ uint32_t stream_word(int w, int lane, uint32_t d, int col_base_rel, int or_base,
                                                const int32_t* col, const uint32_t* src) {
  const uint32_t kind = d >> 30;
  const int len = (int)(d & 0x3fffffffu);
  const int and_len = kind == SK_RULE ? len : 0;
  const int or_len = kind == SK_OR ? len : 0;
  int a_inc = and_len, o_inc = or_len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int x = __shfl_up_sync(FULL, a_inc, o);
    const int y = __shfl_up_sync(FULL, o_inc, o);
    if (lane >= o) {
      a_inc += x;
      o_inc += y;
    }
  }
  const int a_off = a_inc - and_len;
  const int o_off = o_inc - or_len;
  const int a_total = __shfl_sync(FULL, a_inc, 31);
  const int32_t* wc = col + col_base_rel;
  bool val;
  if (a_total <= 1024) {
    // chunk c's ballot lives in lane c
    uint32_t mymask = 0;
    for (int c0 = 0; c0 < a_total; c0 += 128) {
      int j[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int e = c0 + 32 * u + lane;
        j[u] = e < a_total ? wc[e] : -1;
      }
      uint32_t b[4];
#pragma unroll
      for (int u = 0; u < 4; u++) b[u] = j[u] >= 0 ? (src[j[u] >> 5] >> (j[u] & 31)) & 1u : 0u;
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const uint32_t m = __ballot_sync(FULL, b[u]);
        if (lane == (c0 >> 5) + u) mymask = m;
      }
    }
    // rule rows: every bit of [a_off, a_off + len) set
    bool all = true;
    int pos = a_off, rem = and_len;
    while (__any_sync(FULL, rem > 0)) {
      const int bpos = pos & 31;
      const uint32_t m = __shfl_sync(FULL, mymask, (pos >> 5) & 31);
      if (rem > 0) {
        const int take = min(32 - bpos, rem);
        const uint32_t want = take == 32 ? FULL : ((1u << take) - 1u);
        all &= ((m >> bpos) & want) == want;
        pos += take;
        rem -= take;
      }
    }
    val = kind == SK_RULE && len > 0 && all;
  } else {
    // long word: count each row's true entries chunk by chunk
    int cnt = 0;
    for (int c = 0; c < a_total; c += 32) {
      const int e = c + lane;
      uint32_t bit = 0;
      if (e < a_total) {
        const int jj = wc[e];
        bit = (src[jj >> 5] >> (jj & 31)) & 1u;
      }
      const uint32_t m = __ballot_sync(FULL, bit);
      const int lo = max(a_off - c, 0), hi = min(a_off + and_len - c, 32);
      if (hi > lo) cnt += __popc(m & ((hi - lo == 32) ? FULL : (((1u << (hi - lo)) - 1u) << lo)));
    }
    val = kind == SK_RULE && len > 0 && cnt == len;
  }
  if (kind == SK_OR) {  // one of the row's new atoms, a contiguous bit range
    bool any = false;
    int p = or_base + o_off, rem = len;
    while (rem > 0 && !any) {
      const int bpos = p & 31;
      const int take = min(32 - bpos, rem);
      const uint32_t want = take == 32 ? FULL : ((1u << take) - 1u);
      any = ((src[p >> 5] >> bpos) & want) != 0u;
      p += take;
      rem -= take;
    }
    val = any;
  } else if (kind == SK_SELF) {
    val = (src[w] >> lane) & 1u;
  }
  return __ballot_sync(FULL, val);
}

__global__ void __launch_bounds__(kStreamThreads, 1) fixpoint_stream_kernel(StreamArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ int s_flag;
  __shared__ int s_fail;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  const int gwarp = gtid >> 5;
  const int nwarps = nthreads >> 5;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;

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
  }
  __syncthreads();

  // ---- initial vector (as in fixpoint.cu)
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
        if (a.init[i] & ~a.fact_mask[i]) atomicCAS(&ctl->status, 0, LP_ERR_INVALID);
  }
  bool ok = grid_barrier(ctl, ++round, LP_ERR_TIMEOUT);
  if (threadIdx.x == 0) s_flag = (int)ld_volatile((const unsigned*)&ctl->status);
  __syncthreads();
  if (s_flag != 0) ok = false;  // bad initial vector: nothing to iterate

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
    bool changed = false;
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
            const int32_t* colp = ncol >= 0 ? scol : a.and_col;
            const int rel = ncol >= 0 ? h.x - col0 : h.x;
            const uint32_t u = stream_word(w, lane, d, rel, h.y, colp, src);
            if (lane == 0) {
              dst[w] = u;
              changed |= (u != src[w]);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty_bar[s]);
        }
      }
    }
    const int any_changed = __syncthreads_or(changed);
    if (threadIdx.x == 0) {
      if (s_fail) {
        atomicExch(&ctl->abort, 1u);
        atomicCAS(&ctl->status, 0, LP_ERR_TIMEOUT);
      }
      if (any_changed) atomicOr(&ctl->flag[it % 3], 1u);
      if (blockIdx.x == 0) ctl->flag[(it + 1) % 3] = 0u;
    }
    if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) s_flag = (int)ld_volatile(&ctl->flag[it % 3]);
    __syncthreads();
    fin = dst;
    if (!s_flag) {
      converged = true;
      ++it;
      break;
    }
  }
  // copies still in flight (prefetched stages nobody will consume) must land before exit
  if (threadIdx.x == 0 && ng > 0) {
    const long long consumed = (long long)it * ng;  // groups of iterations 0 .. it-1
    for (long long q = consumed; q < q_issue; ++q)
      if (q >= 0 && !mbar_wait(&full_bar[(int)(q % kStages)], (unsigned)((q / kStages) & 1), ctl)) break;
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

}  // namespace lp

namespace lp {

cudaError_t launch_fixpoint_stream(const FixArgs& f, const StreamLayout& L, int grid, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(fixpoint_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kStages * kStageBytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  StreamArgs a{};
  a.desc = L.desc;
  a.word_hdr = L.word_hdr;
  a.and_col = L.and_col;
  a.groups = L.groups;
  a.n_groups = L.n_groups;
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
                                     (size_t)kStages * kStageBytes, s);
}

int fixpoint_stream_blocks_per_sm() {
  if (cudaFuncSetAttribute(fixpoint_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kStages * kStageBytes) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fixpoint_stream_kernel, kStreamThreads,
                                                    (size_t)kStages * kStageBytes) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace lp

// fixpoint_sliced.cu -- Algorithm 1 on a sliced layout of M_P (kernel 2 of the least-model
// schedule), and the device-side build of that layout from the CSR.
//
// theta(M_P v) for a row needs only a logical reduction of the vector bits its entries select
// (Def. 2 and Def. 5 with the values 1/m implicit): a rule row of m body atoms fires iff all m
// bits are 1 (AND), an OR-rule row or a self-loop iff one is (OR), an empty row never. With
// inv = all ones on OR rows and 0 elsewhere, both are one AND: a row fires iff
// AND_e (x_e XOR inv) XOR inv = 1, and repeating one of a row's entries changes neither
// reduction. That gives a padded, column-major layout ("sliced ELL") in which one lane owns a
// row and reads its k-th entry with a coalesced load:
//   - rows are renumbered: within windows of 1024 consecutive rows they are sorted by (gather
//     class, length), so neighbouring rows have similar lengths; the renumbering keeps the
//     leading n_sec_a rows (every row a rule row refers to) in front;
//   - a group is 128 consecutive rows (four 32-row output words) padded to one width K, its
//     longest row; lane l holds rows l, 32 + l, 64 + l, 96 + l, and slot k of the group is 128
//     entries stored so that lane l reads its four rows' k-th entries as one 16-byte load. A
//     shorter row repeats its first entry, an empty row is masked;
//   - a group header (48 bytes): {first entry, K | gather flag}, the four words' OR-row masks,
//     their empty-row masks.
// Column ids, the iterate vectors and the fact rows are all in the new numbering; the output
// projection goes through perm composed with it. The fixpoint and the iteration count are those
// of Algorithm 1 on M_P: renumbering rows and columns together does not change the iteration.
//
// Per iteration every block copies the leading n_sec_a bits of the vector into shared memory;
// groups whose entries all lie there (gather flag) read shared memory, the others (OR rows over
// new atoms) global memory. Each block owns a contiguous range of groups with an equal share of
// the work (stored slots plus a per-group cost), and its warps take the range's groups one at a
// time from a shared counter; the next group's header loads while the current one is evaluated.
#include <cuda_runtime.h>

#include <climits>

#include "device.cuh"
#include "kernels.h"

namespace lp {

namespace {

constexpr int kWindow = 1024;                // rows sorted together
constexpr int kGroupRows = 128;              // rows of a group: four 32-row output words
constexpr uint32_t kStagedFlag = 0x80000000u;  // header .y: every entry of the group is staged
constexpr int kGroupCost = 2;                // per-group cost, in slots, of the block partition

// The layout is read many times per solve and stays in L2: read-only loads with an evict-last
// L2 policy (so that other data, such as dirty lines another kernel left behind, is evicted
// first) that do not allocate in L1, which holds the gathered vector words.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int4 ld_stream4(const int4* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}

// Window i of the renumbering: [lo, hi), windows never straddle n_sec_a.
__device__ __forceinline__ void window_range(int i, int n_sec_a, int n_pad, int* lo, int* hi) {
  const int wa = (n_sec_a + kWindow - 1) / kWindow;
  if (i < wa) {
    *lo = i * kWindow;
    *hi = min(n_sec_a, *lo + kWindow);
  } else {
    *lo = n_sec_a + (i - wa) * kWindow;
    *hi = min(n_pad, *lo + kWindow);
  }
}

// Pass 1: the renumbering. One block per window: sort key = class << 20 | min(length, 2^20 - 1),
// class 1 if some entry lies outside the leading n_sec_a rows; a row's rank is its place in the
// window sorted by (key, row id), a stable sort: a bitonic sort of key << 10 | i (unique) in
// shared memory, padded with all-ones keys to the window size.
static_assert(kWindow == 1024, "the composite key keeps 10 bits of row id");
__global__ void __launch_bounds__(256) sliced_order_kernel(const int32_t* __restrict__ row_ptr,
                                                           const int32_t* __restrict__ col, int n_sec_a, int n_pad,
                                                           int32_t* __restrict__ q, int32_t* __restrict__ qinv) {
  __shared__ uint32_t s_key[kWindow];
  int lo, hi;
  window_range(blockIdx.x, n_sec_a, n_pad, &lo, &hi);
  const int n = hi - lo;
  for (int i = threadIdx.x; i < kWindow; i += blockDim.x) {
    uint32_t key = 0xFFFFFFFFu;
    if (i < n) {
      const int r = lo + i;
      const int b = row_ptr[r], e = row_ptr[r + 1];
      int cls = n_sec_a > 0 ? 0 : 1;
      for (int t = b; t < e && cls == 0; t++) cls = (unsigned)col[t] >= (unsigned)n_sec_a;
      key = ((uint32_t)((cls << 20) | min(e - b, (1 << 20) - 1)) << 10) | (uint32_t)i;
    }
    s_key[i] = key;
  }
  __syncthreads();
  for (int k = 2; k <= kWindow; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kWindow; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const uint32_t x = s_key[i], y = s_key[ixj];
          if ((x > y) == ((i & k) == 0)) {
            s_key[i] = y;
            s_key[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int i = (int)(s_key[p] & (kWindow - 1));
    q[lo + i] = lo + p;
    qinv[lo + p] = lo + i;
  }
}

// Pass 2: group headers (one warp per group): width K = longest row, gather flag, the four words'
// OR-row and empty-row masks; cnt[g] = 128 K (entries to store). Rows past n_pad are empty.
__global__ void sliced_header_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     const uint32_t* __restrict__ any_mask, const int32_t* __restrict__ qinv,
                                     int n_sec_a, int n_pad, int n_groups, int4* __restrict__ hdr,
                                     int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int g = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (g >= n_groups) return;
  int K = 0;
  bool staged = n_sec_a > 0;
  uint32_t orm[4], emm[4];
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int t = g * kGroupRows + 32 * u + lane;
    int len = 0;
    bool anyb = false;
    if (t < n_pad) {
      const int r = qinv[t];
      const int b = row_ptr[r], e = row_ptr[r + 1];
      len = e - b;
      for (int i = b; i < e && staged; i++) staged = (unsigned)col[i] < (unsigned)n_sec_a;
      anyb = (any_mask[r >> 5] >> (r & 31)) & 1u;
    }
    K = max(K, len);
    orm[u] = __ballot_sync(FULL, anyb);
    emm[u] = __ballot_sync(FULL, len == 0);
  }
  K = __reduce_max_sync(FULL, K);
  const bool all_staged = __all_sync(FULL, staged);
  if (lane == 0) {
    hdr[3 * g] = make_int4(0, K | (all_staged ? (int)kStagedFlag : 0), 0, 0);
    hdr[3 * g + 1] = make_int4((int)orm[0], (int)orm[1], (int)orm[2], (int)orm[3]);
    hdr[3 * g + 2] = make_int4((int)emm[0], (int)emm[1], (int)emm[2], (int)emm[3]);
    cnt[g] = kGroupRows * K;
  }
}

// Pass 3: exclusive prefix sum of the groups' entry counts (one block) into hdr[3 g].x; the
// total into *total_out.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) sliced_scan_kernel(const int32_t* __restrict__ cnt, int n_groups,
                                                                  int4* __restrict__ hdr,
                                                                  long long* __restrict__ total_out) {
  __shared__ long long s_sum[kScanThreads];
  const int t = threadIdx.x;
  const int per = (n_groups + kScanThreads - 1) / kScanThreads;
  const int lo = min(n_groups, t * per), hi = min(n_groups, lo + per);
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
    hdr[3 * i].x = (int)min(run, (long long)INT_MAX);
    run += cnt[i];
  }
  if (t == kScanThreads - 1) *total_out = s_sum[t];
}

// Pass 4: the entries, renumbered. Entry k of row 32 u + l of group g sits at
// off_g + 4 (32 k + l) + u; a row repeats its first entry past its length (0 if empty).
__global__ void sliced_fill_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const int32_t* __restrict__ q, const int32_t* __restrict__ qinv,
                                   const int4* __restrict__ hdr, int n_pad, int n_groups,
                                   int32_t* __restrict__ scol) {
  const int lane = threadIdx.x & 31;
  const int g = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (g >= n_groups) return;
  const int4 h = hdr[3 * g];
  const int K = h.y & ~(int)kStagedFlag;
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const int t = g * kGroupRows + 32 * u + lane;
    int b = 0, len = 0;
    if (t < n_pad) {
      const int r = qinv[t];
      b = row_ptr[r];
      len = row_ptr[r + 1] - b;
    }
    const int first = len > 0 ? q[col[b]] : 0;
    for (int k = 0; k < K; k++) scol[(long long)h.x + 4ll * (32 * k + lane) + u] = k < len ? q[col[b + k]] : first;
  }
}

// Pass 5: a[i] = q[src[i]] (fact rows and the output permutation in the new numbering).
__global__ void sliced_map_kernel(const int32_t* __restrict__ src, int n, const int32_t* __restrict__ q,
                                  int32_t* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = q[src[i]];
}

// ---------------------------------------------------------------------------------------
// The least-model loop.

// Bit 0 = bit j of the vector word x (a rotate by j mod 32).
__device__ __forceinline__ uint32_t rot(uint32_t x, int j) { return __funnelshift_r(x, x, (uint32_t)j); }

// The four output words of group g: acc[u] = AND over the slots of (bit XOR inv[u]).
template <bool SMEM>
__device__ __forceinline__ void group_acc(const int4* __restrict__ e, int K, const uint32_t* x, const uint32_t inv[4],
                                          uint32_t acc[4], uint64_t pol) {
  int k = 0;
  for (; k + 2 <= K; k += 2) {  // two slots per step: two 16-byte loads in flight, then 8 gathers
    const int4 a = ld_stream4(e + 32 * k, pol), b = ld_stream4(e + 32 * (k + 1), pol);
    acc[0] &= (rot(x[a.x >> 5], a.x) ^ inv[0]) & (rot(x[b.x >> 5], b.x) ^ inv[0]);
    acc[1] &= (rot(x[a.y >> 5], a.y) ^ inv[1]) & (rot(x[b.y >> 5], b.y) ^ inv[1]);
    acc[2] &= (rot(x[a.z >> 5], a.z) ^ inv[2]) & (rot(x[b.z >> 5], b.z) ^ inv[2]);
    acc[3] &= (rot(x[a.w >> 5], a.w) ^ inv[3]) & (rot(x[b.w >> 5], b.w) ^ inv[3]);
  }
  if (k < K) {
    const int4 a = ld_stream4(e + 32 * k, pol);
    acc[0] &= rot(x[a.x >> 5], a.x) ^ inv[0];
    acc[1] &= rot(x[a.y >> 5], a.y) ^ inv[1];
    acc[2] &= rot(x[a.z >> 5], a.z) ^ inv[2];
    acc[3] &= rot(x[a.w >> 5], a.w) ^ inv[3];
  }
}

template <bool STAGE>
__global__ void __launch_bounds__(kSlicedBlock, 1) fixpoint_sliced_kernel(FixArgs a, SlicedLayout L) {
  extern __shared__ uint4 s_stage[];
  __shared__ int s_next, s_g0, s_g1;
  const uint32_t* s_x = reinterpret_cast<const uint32_t*>(s_stage);
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = gridDim.x * blockDim.x;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;
  const int n_stage4 = STAGE ? L.n_stage_words >> 2 : 0;
  const int n_groups = L.n_groups;
  const uint64_t pol = l2_evict_last_policy();

  // ---- this block's groups: an equal share of the cost (slots + kGroupCost per group); the
  // cost before group g is off_g / 128 + kGroupCost g (the offsets are a prefix sum)
  if (threadIdx.x == 0) {
    const long long total = L.total_entries / kGroupRows + (long long)kGroupCost * n_groups;
    int bounds[2];
    for (int side = 0; side < 2; side++) {
      const long long target = total * (blockIdx.x + side) / gridDim.x;
      int lo = 0, hi = n_groups;  // first g with cost_before(g) >= target
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const long long c = (long long)L.hdr[3 * mid].x / kGroupRows + (long long)kGroupCost * mid;
        if (c >= target) hi = mid; else lo = mid + 1;
      }
      bounds[side] = lo;
    }
    s_g0 = bounds[0];
    s_g1 = blockIdx.x + 1 == gridDim.x ? n_groups : bounds[1];
  }

  // ---- initial vector v0 in the new numbering (x0 was zeroed by the caller)
  if (a.rows_init) {
    // LP_ROWS: internal row r takes bit inv[r] of the caller's canonical vector
    for (int r = gtid; r < a.n_prime; r += nthreads) {
      const int c = a.inv[r];
      if ((a.rows_init[c >> 6] >> (c & 63)) & 1ull) {
        const int t = L.q[r];
        atomicOr(a.x0 + (t >> 5), 1u << (t & 31));
      }
    }
  } else {
    // Def. 4: a fact row is 1 when its atom is selected
    for (int i = gtid; i < a.n_facts; i += nthreads) {
      const int own = a.fact_owner[i];
      const bool sel = a.init ? ((a.init[own >> 6] >> (own & 63)) & 1ull) : true;
      if (sel) atomicOr(a.x0 + (L.fact_row[i] >> 5), 1u << (L.fact_row[i] & 31));
    }
    if (a.init)
      for (int i = gtid; i < a.n_atom_words; i += nthreads)
        if (a.init[i] & ~a.fact_mask[i]) atomicCAS(&ctl->status, 0, 1 /* LP_ERR_INVALID */);
  }
  bool dummy;
  if (!grid_barrier_or(ctl, ++round, false, &dummy, 6)) return;
  if (ld_volatile((const unsigned*)&ctl->status) != 0) return;
  const int g0 = s_g0, g1 = s_g1;

  const uint32_t* fin = a.x0;
  int it = 0;
  bool converged = false;
  for (; it < a.max_iters; ++it) {
    const uint32_t* src = (it & 1) ? a.x1 : a.x0;
    uint32_t* dst = (it & 1) ? a.x0 : a.x1;
    if (STAGE) {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      for (int i = threadIdx.x; i < n_stage4; i += blockDim.x) s_stage[i] = __ldcg(s4 + i);
    }
    if (threadIdx.x == 0) s_next = g0;
    __syncthreads();
    bool changed = false;
    // groups are taken one at a time from the block's counter; the next one is taken (and its
    // header loaded) before the current one is evaluated
    int g = 0;
    if (lane == 0) g = atomicAdd(&s_next, 1);
    g = __shfl_sync(FULL, g, 0);
    int4 h0, h1, h2;
    if (g < g1) {
      h0 = ld_stream4(L.hdr + 3 * g, pol);
      h1 = ld_stream4(L.hdr + 3 * g + 1, pol);
      h2 = ld_stream4(L.hdr + 3 * g + 2, pol);
    }
    while (g < g1) {  // uniform in the warp
      int gn = 0;
      if (lane == 0) gn = atomicAdd(&s_next, 1);
      gn = __shfl_sync(FULL, gn, 0);
      int4 n0, n1, n2;
      if (gn < g1) {
        n0 = ld_stream4(L.hdr + 3 * gn, pol);
        n1 = ld_stream4(L.hdr + 3 * gn + 1, pol);
        n2 = ld_stream4(L.hdr + 3 * gn + 2, pol);
      }
      const int w0 = g * (kGroupRows / 32);
      const uint32_t old = lane < 4 && w0 + lane < a.n_words ? src[w0 + lane] : 0u;
      const int K = h0.y & ~(int)kStagedFlag;
      const uint32_t inv[4] = {((uint32_t)h1.x >> lane) & 1u ? FULL : 0u, ((uint32_t)h1.y >> lane) & 1u ? FULL : 0u,
                               ((uint32_t)h1.z >> lane) & 1u ? FULL : 0u, ((uint32_t)h1.w >> lane) & 1u ? FULL : 0u};
      uint32_t acc[4] = {FULL, FULL, FULL, FULL};
      const int4* e = reinterpret_cast<const int4*>(L.col + h0.x) + lane;
      if (STAGE && ((uint32_t)h0.y & kStagedFlag)) group_acc<true>(e, K, s_x, inv, acc, pol);
      else group_acc<false>(e, K, src, inv, acc, pol);
      const uint32_t u0 = __ballot_sync(FULL, ((acc[0] ^ inv[0]) & ~((uint32_t)h2.x >> lane)) & 1u);
      const uint32_t u1 = __ballot_sync(FULL, ((acc[1] ^ inv[1]) & ~((uint32_t)h2.y >> lane)) & 1u);
      const uint32_t u2 = __ballot_sync(FULL, ((acc[2] ^ inv[2]) & ~((uint32_t)h2.z >> lane)) & 1u);
      const uint32_t u3 = __ballot_sync(FULL, ((acc[3] ^ inv[3]) & ~((uint32_t)h2.w >> lane)) & 1u);
      if (lane < 4 && w0 + lane < a.n_words) {
        const uint32_t word = lane == 0 ? u0 : lane == 1 ? u1 : lane == 2 ? u2 : u3;
        dst[w0 + lane] = word;
        changed |= word != old;
      }
      g = gn;
      h0 = n0;
      h1 = n1;
      h2 = n2;
    }
    bool any_changed;
    if (!grid_barrier_or(ctl, ++round, changed, &any_changed, 6)) return;
    fin = dst;
    if (!any_changed) {
      converged = true;
      ++it;
      break;
    }
  }
  if (gtid == 0) {
    ctl->iters = it;
    if (!converged) atomicCAS(&ctl->status, 0, 4 /* LP_ERR_NO_FIXPOINT */);
  }

  // ---- output: bit a of out = fixpoint bit of row q[perm[a]]
  if (a.out) {
    uint32_t* out32 = reinterpret_cast<uint32_t*>(a.out);
    const int n32 = 2 * ((a.n_out + 63) >> 6);
    for (int u = gwarp; u < n32; u += nwarps) {
      const int i = (u << 5) + lane;
      uint32_t bit = 0u;
      if (i < a.n_out) {
        const int r = L.perm[i];
        bit = (fin[r >> 5] >> (r & 31)) & 1u;
      }
      const uint32_t word = __ballot_sync(FULL, bit);
      if (lane == 0) out32[u] = word;
    }
  }
}

const void* sliced_entry(bool stage) {
  return stage ? (const void*)fixpoint_sliced_kernel<true> : (const void*)fixpoint_sliced_kernel<false>;
}

}  // namespace

int sliced_windows(int32_t n_sec_a, int32_t n_pad) {
  return (n_sec_a + kWindow - 1) / kWindow + (n_pad - n_sec_a + kWindow - 1) / kWindow;
}

int sliced_groups(int32_t n_pad) { return (n_pad + kGroupRows - 1) / kGroupRows; }

cudaError_t build_sliced_pass1(const int32_t* row_ptr, const int32_t* col, const uint32_t* any_mask, int32_t n_sec_a,
                               int32_t n_pad, int32_t* q, int32_t* qinv, int4* hdr, int32_t* cnt, long long* total_dev,
                               cudaStream_t s) {
  const int n_groups = sliced_groups(n_pad);
  if (n_groups <= 0) return cudaSuccess;
  sliced_order_kernel<<<sliced_windows(n_sec_a, n_pad), 256, 0, s>>>(row_ptr, col, n_sec_a, n_pad, q, qinv);
  const int threads = 256, blocks = (int)(((long long)n_groups * 32 + threads - 1) / threads);
  sliced_header_kernel<<<blocks, threads, 0, s>>>(row_ptr, col, any_mask, qinv, n_sec_a, n_pad, n_groups, hdr, cnt);
  sliced_scan_kernel<<<1, kScanThreads, 0, s>>>(cnt, n_groups, hdr, total_dev);
  return cudaGetLastError();
}

cudaError_t build_sliced_pass2(const int32_t* row_ptr, const int32_t* col, const int32_t* q, const int32_t* qinv,
                               const int4* hdr, int32_t n_pad, int32_t* scol, const int32_t* fact_row, int32_t n_facts,
                               int32_t* fact_row_out, const int32_t* perm, int32_t n_perm, int32_t* perm_out,
                               cudaStream_t s) {
  const int n_groups = sliced_groups(n_pad);
  if (n_groups <= 0) return cudaSuccess;
  const int threads = 256, blocks = (int)(((long long)n_groups * 32 + threads - 1) / threads);
  sliced_fill_kernel<<<blocks, threads, 0, s>>>(row_ptr, col, q, qinv, hdr, n_pad, n_groups, scol);
  if (n_facts > 0) sliced_map_kernel<<<(n_facts + 255) / 256, 256, 0, s>>>(fact_row, n_facts, q, fact_row_out);
  if (n_perm > 0) sliced_map_kernel<<<(n_perm + 255) / 256, 256, 0, s>>>(perm, n_perm, q, perm_out);
  return cudaGetLastError();
}

cudaError_t launch_fixpoint_sliced(const FixArgs& a, const SlicedLayout& L, bool stage, int grid, cudaStream_t s) {
  FixArgs ca = a;
  SlicedLayout cl = L;
  void* params[] = {&ca, &cl};
  const size_t smem = stage ? (size_t)L.n_stage_words * 4 : 0;
  const void* k = sliced_entry(stage);
  // the unified L1 / shared array: as much L1 as the staged prefix leaves (the gathers of the
  // unstaged groups and of the OR rows go through L1)
  cudaError_t e = set_kernel_smem(k, (int)smem, stage ? -1 : 0);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kSlicedBlock), params, smem, s);
}

int fixpoint_sliced_blocks_per_sm(bool stage, int stage_words) {
  const void* k = sliced_entry(stage);
  const size_t smem = stage ? (size_t)stage_words * 4 : 0;
  if (set_kernel_smem(k, (int)smem, stage ? -1 : 0) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kSlicedBlock, smem) != cudaSuccess) return 0;
  return nb;
}

}  // namespace lp

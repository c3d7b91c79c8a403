// compile_device.cu -- the standardization of lp_compile on the GPU: rules -> the program matrix
// M_P in the internal layout, array for array what the host compiler (compile.cpp) builds.
//
// Sec. 2.1 / 2.2 of the paper: a negated literal "not q" becomes the new atom q-bar (Eq. 4), a body
// is a set (footnote of Eq. 2), a head with several rules becomes an OR-rule over one new atom per
// rule, and M_P follows Def. 2 and Def. 7. The internal order is the host compiler's: section A
// (original and barred atoms) by descending number of rule-row references, ties by canonical id;
// section B (the new atoms) grouped by their OR row in section-A order, rule order within a row;
// padding rows up to a multiple of 64.
//
// The rules are uploaded as given (head, body offsets, body atoms, negation flags: about as many
// bytes as the compiled matrix) and every step runs as kernels on the call's stream: counts by
// atomics, ranks by exclusive scans, the groupings and the internal order by a stable LSD radix
// sort, bodies and rows sorted per rule (in a thread when short, by two stable sorts of their
// entries otherwise). The host reads a few scalars between steps (sizes it allocates by).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "program.h"

namespace lp {

namespace {

// ------------------------------------------------------------------------------------------
// Exclusive scan of f(0 .. n) into out[0 .. n) (int64), the total into *total: block sums, one
// block scanning them, then each block's items from its offset.
constexpr int kScanThreads = 512;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

// Exclusive prefix of v over the block; the block's sum into *sum. All threads call it.
__device__ __forceinline__ int64_t block_exclusive(int64_t v, int64_t* sum) {
  __shared__ int64_t s_warp[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t u = __shfl_up_sync(FULL, incl, d);
    if (lane >= d) incl += u;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
    int64_t wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t u = __shfl_up_sync(FULL, wi, d);
      if (lane >= d) wi += u;
    }
    if (lane < kScanThreads / 32) s_warp[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *sum = wi;
  }
  __syncthreads();
  const int64_t r = s_warp[warp] + incl - v;
  __syncthreads();
  return r;
}

template <class F>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(F f, int64_t n, int64_t* block_sums) {
  __shared__ int64_t s_sum;
  const int64_t i0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int64_t v = 0;
  for (int j = 0; j < kScanPer; j++)
    if (i0 + j < n) v += f(i0 + j);
  block_exclusive(v, &s_sum);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = s_sum;
}

// In place over sums[0 .. m): exclusive prefix; the total into *total (one block).
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int64_t* sums, int64_t m, int64_t* total) {
  __shared__ int64_t s_sum;
  int64_t run = 0;
  for (int64_t base = 0; base < m; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < m ? sums[i] : 0;
    const int64_t e = block_exclusive(v, &s_sum);
    if (i < m) sums[i] = run + e;
    run += s_sum;
  }
  if (threadIdx.x == 0) *total = run;
}

template <class F>
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(F f, int64_t n, const int64_t* block_off,
                                                                  int64_t* out) {
  __shared__ int64_t s_sum;
  const int64_t i0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int64_t vals[kScanPer];
  int64_t v = 0;
  for (int j = 0; j < kScanPer; j++) {
    vals[j] = i0 + j < n ? f(i0 + j) : 0;
    v += vals[j];
  }
  int64_t run = block_off[blockIdx.x] + block_exclusive(v, &s_sum);
  for (int j = 0; j < kScanPer; j++)
    if (i0 + j < n) {
      out[i0 + j] = run;
      run += vals[j];
    }
}

// Temporaries of one compile, stream-ordered on its stream and freed in stream order with it.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> bufs;
  cudaError_t err = cudaSuccess;
  int64_t* sums = nullptr;  // block sums of the scans, grown as needed
  int64_t sums_n = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    const cudaError_t e = device_malloc_async(&p, std::max<size_t>(count * sizeof(T), 16), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (err == cudaSuccess) err = e;
      return nullptr;
    }
    bufs.push_back(p);
    return (T*)p;
  }
  ~Scratch() {
    for (void* p : bufs) cudaFreeAsync(p, s);
  }
};

template <class F>
cudaError_t scan(F f, int64_t n, int64_t* out, int64_t* total, Scratch& sc) {
  const int64_t blocks = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
  if (blocks > sc.sums_n) {
    sc.sums = sc.get<int64_t>((size_t)std::max<int64_t>(blocks, 1024));
    if (!sc.sums) return sc.err;
    sc.sums_n = std::max<int64_t>(blocks, 1024);
  }
  cudaStream_t s = sc.s;
  if (n > 0) scan_reduce_kernel<<<(unsigned)blocks, kScanThreads, 0, s>>>(f, n, sc.sums);
  else cudaMemsetAsync(sc.sums, 0, 8, s);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sc.sums, blocks, total);
  if (n > 0) scan_apply_kernel<<<(unsigned)blocks, kScanThreads, 0, s>>>(f, n, sc.sums, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the keys, 8 bits per
// pass. A tile of 2048 pairs per block: per-tile digit counts, their exclusive scan in digit-major
// order (the tiles of digit 0, then of digit 1, ...), then each tile writes its pairs from its
// offsets, ranked within the tile in input order (warp by warp, lanes by match_any).
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsPer = 8;
constexpr int kRsTile = kRsThreads * kRsPer;
constexpr int kRsDigits = 256;

__global__ void __launch_bounds__(kRsThreads) rs_count_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                              int64_t n_tiles, int64_t* __restrict__ counts) {
  __shared__ int s_cnt[kRsDigits];
  for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads) s_cnt[d] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * (32 * kRsPer);
  for (int j = 0; j < kRsPer; j++) {
    const int64_t i = base + j * 32 + lane;
    if (i < n) atomicAdd(&s_cnt[(keys[i] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads) counts[(int64_t)d * n_tiles + blockIdx.x] = s_cnt[d];
}

__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(const uint32_t* __restrict__ keys,
                                                                const int32_t* __restrict__ vals, int64_t n, int shift,
                                                                int64_t n_tiles, const int64_t* __restrict__ offsets,
                                                                uint32_t* __restrict__ keys_out,
                                                                int32_t* __restrict__ vals_out) {
  __shared__ int s_cnt[kRsWarps][kRsDigits];
  for (int i = threadIdx.x; i < kRsWarps * kRsDigits; i += kRsThreads) (&s_cnt[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * kRsTile + warp * (32 * kRsPer);
  uint32_t k[kRsPer];
  int32_t v[kRsPer];
  int rank[kRsPer];
  for (int j = 0; j < kRsPer; j++) {
    const int64_t i = base + j * 32 + lane;
    const bool ok = i < n;
    k[j] = ok ? keys[i] : 0u;
    v[j] = ok ? vals[i] : 0;
    const int d = ok ? (int)((k[j] >> shift) & 0xFF) : kRsDigits;  // invalid pairs match only each other
    const unsigned peers = __match_any_sync(FULL, d);
    rank[j] = ok ? s_cnt[warp][d] + __popc(peers & lt) : 0;
    __syncwarp();
    if (ok && (peers & lt) == 0u) s_cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads) {  // warps in order within the tile
    int run = 0;
    for (int w = 0; w < kRsWarps; w++) {
      const int c = s_cnt[w][d];
      s_cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int j = 0; j < kRsPer; j++) {
    const int64_t i = base + j * 32 + lane;
    if (i < n) {
      const int d = (int)((k[j] >> shift) & 0xFF);
      const int64_t o = offsets[(int64_t)d * n_tiles + blockIdx.x] + s_cnt[warp][d] + rank[j];
      keys_out[o] = k[j];
      vals_out[o] = v[j];
    }
  }
}

struct CountAt {
  const int64_t* c;
  __device__ int64_t operator()(int64_t i) const { return c[i]; }
};

// Sorts (keys, vals)[0 .. n) by the low `bits` bits of the keys, stably. The result is in
// (keys, vals) again; (tk, tv) are buffers of n pairs.
cudaError_t radix_sort(uint32_t* keys, int32_t* vals, uint32_t* tk, int32_t* tv, int64_t n, int bits, Scratch& sc) {
  if (n <= 1 || bits <= 0) return cudaSuccess;
  cudaStream_t s = sc.s;
  const int64_t n_tiles = (n + kRsTile - 1) / kRsTile;
  int64_t* counts = sc.get<int64_t>((size_t)kRsDigits * n_tiles);
  int64_t* offs = sc.get<int64_t>((size_t)kRsDigits * n_tiles);
  int64_t* total = sc.get<int64_t>(1);
  if (!counts || !offs || !total) return sc.err;
  const int passes = (bits + 7) / 8;
  uint32_t *ka = keys, *kb = tk;
  int32_t *va = vals, *vb = tv;
  for (int p = 0; p < passes; p++) {
    rs_count_kernel<<<(unsigned)n_tiles, kRsThreads, 0, s>>>(ka, n, 8 * p, n_tiles, counts);
    cudaError_t e = scan(CountAt{counts}, kRsDigits * n_tiles, offs, total, sc);
    if (e != cudaSuccess) return e;
    rs_scatter_kernel<<<(unsigned)n_tiles, kRsThreads, 0, s>>>(ka, va, n, 8 * p, n_tiles, offs, kb, vb);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {  // an odd number of passes: the result is in the buffers
    cudaMemcpyAsync(keys, ka, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

int bit_width(uint64_t x) {
  int b = 0;
  while (x) {
    b++;
    x >>= 1;
  }
  return b;
}


// ------------------------------------------------------------------------------------------
// The standardization steps. Canonical ids: original atoms 0 .. n-1, barred atoms n .. n+nb-1 (in
// ascending order of their atom), new atoms n+nb .. n'-1 (one per rule of a multi-rule head, in
// rule order).
constexpr int kThreads = 256;
constexpr int kShortBody = 32;  // bodies and rows up to this length are sorted by one thread

inline unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// The first rule with a head out of range or a decreasing offset, the first literal with an atom
// out of range (atomicMin into err[0], err[1]).
__global__ void validate_kernel(const int32_t* head, const int64_t* off, int64_t n_rules, const int32_t* atom,
                                int64_t total, int32_t n, unsigned long long* err) {
  for (int64_t r = gtid(); r < n_rules; r += gstride())
    if (head[r] < 0 || head[r] >= n || off[r + 1] < off[r]) atomicMin(err, (unsigned long long)r);
  for (int64_t e = gtid(); e < total; e += gstride())
    if (atom[e] < 0 || atom[e] >= n) atomicMin(err + 1, (unsigned long long)e);
}

// Rules per head; atoms that occur negated.
__global__ void count_kernel(const int32_t* head, int64_t n_rules, const int32_t* atom, const uint8_t* neg,
                             int64_t total, int32_t* cnt, uint8_t* negated) {
  for (int64_t r = gtid(); r < n_rules; r += gstride()) atomicAdd(cnt + head[r], 1);
  if (neg)
    for (int64_t e = gtid(); e < total; e += gstride())
      if (neg[e]) negated[atom[e]] = 1;  // every writer stores the same value
}

struct FlagU8 {
  const uint8_t* f;
  __device__ int64_t operator()(int64_t i) const { return f[i] != 0; }
};
struct MultiRuleHead {
  const int32_t* head;
  const int32_t* cnt;
  __device__ int64_t operator()(int64_t r) const { return cnt[head[r]] >= 2; }
};
struct CountI32 {
  const int32_t* c;
  __device__ int64_t operator()(int64_t i) const { return c[i]; }
};

// bar_id[a] = n + rank of a among the negated atoms (-1 if a never occurs negated); bar_atom is
// the inverse.
__global__ void bar_kernel(const uint8_t* negated, const int64_t* rank, int32_t n, int32_t* bar_id,
                           int32_t* bar_atom) {
  for (int64_t a = gtid(); a < n; a += gstride()) {
    if (negated[a]) {
      bar_id[a] = (int32_t)(n + rank[a]);
      bar_atom[rank[a]] = (int32_t)a;
    } else {
      bar_id[a] = -1;
    }
  }
}

// aux[r] = n + nb + rank of r among the rules of multi-rule heads (-1 for a head's only rule);
// aux_rule is the inverse.
__global__ void aux_kernel(const int32_t* head, const int32_t* cnt, const int64_t* rank, int64_t n_rules,
                           int64_t first, int32_t* aux, int32_t* aux_rule) {
  for (int64_t r = gtid(); r < n_rules; r += gstride()) {
    if (cnt[head[r]] >= 2) {
      aux[r] = (int32_t)(first + rank[r]);
      aux_rule[rank[r]] = (int32_t)r;
    } else {
      aux[r] = -1;
    }
  }
}

// The body of rule r in canonical ids (a negated literal is its barred atom). Short bodies are
// sorted and deduplicated here (setlen = the set's size); a long one is only mapped and flagged.
__global__ void body_kernel(const int64_t* off, int64_t n_rules, const int32_t* atom, const uint8_t* neg,
                            const int32_t* bar_id, int32_t* rb, int32_t* setlen, uint8_t* is_long) {
  for (int64_t r = gtid(); r < n_rules; r += gstride()) {
    const int64_t b = off[r], m = off[r + 1] - b;
    int32_t* d = rb + b;
    for (int64_t i = 0; i < m; i++) {
      const int32_t a = atom[b + i];
      d[i] = (neg && neg[b + i]) ? bar_id[a] : a;
    }
    if (m > kShortBody) {
      is_long[r] = 1;
      continue;
    }
    is_long[r] = 0;
    for (int i = 1; i < (int)m; i++) {  // insertion sort
      const int32_t x = d[i];
      int j = i - 1;
      while (j >= 0 && d[j] > x) {
        d[j + 1] = d[j];
        j--;
      }
      d[j + 1] = x;
    }
    int u = 0;
    for (int i = 0; i < (int)m; i++)
      if (u == 0 || d[u - 1] != d[i]) d[u++] = d[i];
    setlen[r] = u;
  }
}

// Entries of the long segments (segment s = [seg_off[s], seg_off[s+1]) of `data` at data_off)
// as (key = value, val = segment) pairs, in segment order.
__global__ void long_gather_kernel(const int64_t* seg_first, const int32_t* seg_src, int64_t n_seg,
                                   const int64_t* src_off, const int32_t* seg_len, const int32_t* data,
                                   uint32_t* keys, int32_t* vals) {
  for (int64_t sgi = blockIdx.x; sgi < n_seg; sgi += gridDim.x) {
    const int32_t r = seg_src[sgi];
    const int64_t b = src_off[r], o = seg_first[sgi];
    for (int64_t i = threadIdx.x; i < seg_len[r]; i += blockDim.x) {
      keys[o + i] = (uint32_t)data[b + i];
      vals[o + i] = (int32_t)sgi;
    }
  }
}

// After the two sorts, each long segment's values are in ascending order at seg_first[s]: write
// them back, deduplicated when `dedup` (the set's size into setlen[r]).
__global__ void long_scatter_kernel(const int64_t* seg_first, const int32_t* seg_src, int64_t n_seg,
                                    const int64_t* dst_off, const int32_t* seg_len, const uint32_t* sorted,
                                    int32_t* data, int32_t* setlen, bool dedup) {
  for (int64_t sgi = gtid(); sgi < n_seg; sgi += gstride()) {
    const int32_t r = seg_src[sgi];
    const int64_t o = seg_first[sgi], m = seg_len[r];
    int32_t* d = data + dst_off[r];
    int64_t u = 0;
    for (int64_t i = 0; i < m; i++) {
      const int32_t x = (int32_t)sorted[o + i];
      if (!dedup || u == 0 || d[u - 1] != x) d[u++] = x;
    }
    if (dedup) setlen[r] = (int32_t)u;
  }
}

struct LongFlag {
  const uint8_t* f;
  __device__ int64_t operator()(int64_t i) const { return f[i]; }
};
struct LongLen {
  const uint8_t* f;
  const int32_t* len;
  __device__ int64_t operator()(int64_t r) const { return f[r] ? len[r] : 0; }
};

// seg_src[rank[r]] = r for the flagged rules; seg_len for the raw bodies (setlen = raw length
// until the sort deduplicates them).
__global__ void long_list_kernel(const uint8_t* flag, const int64_t* rank, const int64_t* len_scan, int64_t n_rules,
                                 int32_t* seg_src, int64_t* seg_first) {
  for (int64_t r = gtid(); r < n_rules; r += gstride())
    if (flag[r]) {
      seg_src[rank[r]] = (int32_t)r;
      seg_first[rank[r]] = len_scan[r];
    }
}
__global__ void raw_len_kernel(const uint8_t* flag, const int64_t* off, int64_t n_rules, int32_t* len) {
  for (int64_t r = gtid(); r < n_rules; r += gstride())
    if (flag[r]) len[r] = (int32_t)(off[r + 1] - off[r]);
}

// Keys and values of the grouping by head: (head[r], r).
__global__ void iota_keys_kernel(const int32_t* key_src, int64_t n, uint32_t* keys, int32_t* vals) {
  for (int64_t i = gtid(); i < n; i += gstride()) {
    keys[i] = (uint32_t)key_src[i];
    vals[i] = (int32_t)i;
  }
}

// Row kinds and defining rules in canonical order (Def. 2, Def. 7).
__global__ void kind_rules_kernel(const int32_t* aux, const int32_t* setlen, int64_t n_rules, int8_t* kind,
                                  int32_t* row_rule) {
  for (int64_t r = gtid(); r < n_rules; r += gstride())
    if (aux[r] >= 0) {  // a rule of a multi-rule head defines its new atom's row
      kind[aux[r]] = setlen[r] == 0 ? K_FACT : K_RULE;
      row_rule[aux[r]] = (int32_t)r;
    }
}
__global__ void kind_atoms_kernel(const int32_t* cnt, const int64_t* hr_off, const int32_t* by_head,
                                  const int32_t* setlen, const int32_t* bar_id, int32_t n, int8_t* kind,
                                  int32_t* row_rule) {
  for (int64_t a = gtid(); a < n; a += gstride()) {
    if (cnt[a] >= 2) {
      kind[a] = K_OR;
    } else if (cnt[a] == 1) {
      const int32_t r = by_head[hr_off[a]];
      kind[a] = setlen[r] == 0 ? K_FACT : K_RULE;
      row_rule[a] = r;
    }
    if (bar_id[a] >= 0) kind[bar_id[a]] = K_BARRED;
  }
}

struct RowLen {
  const int8_t* kind;
  const int32_t* row_rule;
  const int32_t* setlen;
  const int32_t* cnt;  // rules of each original atom (OR rows are original atoms)
  __device__ int64_t operator()(int64_t c) const {
    switch (kind[c]) {
      case K_RULE: return setlen[row_rule[c]];
      case K_OR: return cnt[c];
      case K_FACT:
      case K_BARRED: return 1;
      default: return 0;
    }
  }
};

// References of each section-A column by rule-row entries (facts define self-loops). A warp
// takes 32 rules and walks their entries in step; lanes holding the same column add once (the
// most referenced atoms of a skewed program would otherwise serialize on one counter).
__global__ void deg_kernel(const int64_t* off, const int32_t* setlen, int64_t n_rules, const int32_t* rb,
                           int32_t* deg) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = gtid() - lane; base < n_rules; base += gstride()) {  // uniform in the warp
    const int64_t r = base + lane;
    const int m = r < n_rules ? setlen[r] : 0;
    const int32_t* sb = rb + (r < n_rules ? off[r] : 0);
    const int steps = (int)__reduce_max_sync(FULL, (unsigned)m);
    for (int i = 0; i < steps; i++) {
      const int c = i < m ? sb[i] : -1;
      const unsigned peers = __match_any_sync(FULL, c);
      if (c >= 0 && (peers & lt) == 0u) atomicAdd(deg + c, __popc(peers));
    }
  }
}
__global__ void max_kernel(const int32_t* v, int64_t n, unsigned* out) {
  unsigned m = 0;
  for (int64_t i = gtid(); i < n; i += gstride()) m = max(m, (unsigned)v[i]);
  m = __reduce_max_sync(FULL, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
// key = maxdeg - deg (ascending = most referenced first), value = canonical id
__global__ void order_keys_kernel(const int32_t* deg, int64_t nA, const unsigned* maxdeg, uint32_t* keys,
                                  int32_t* vals) {
  const unsigned md = *maxdeg;
  for (int64_t c = gtid(); c < nA; c += gstride()) {
    keys[c] = md - (unsigned)deg[c];
    vals[c] = (int32_t)c;
  }
}

struct NewAtoms {
  const int32_t* inv;
  const int8_t* kind;
  const int32_t* cnt;
  __device__ int64_t operator()(int64_t i) const {
    const int32_t c = inv[i];
    return kind[c] == K_OR ? cnt[c] : 0;
  }
};

// Section B: each OR row's new atoms, in rule order, from its section-B position on.
__global__ void section_b_kernel(const int64_t* bpos, int64_t nA, const int8_t* kind, const int64_t* hr_off,
                                 const int32_t* by_head, const int32_t* aux, int32_t* inv) {
  for (int64_t i = gtid(); i < nA; i += gstride()) {
    const int32_t c = inv[i];
    if (kind[c] != K_OR) continue;
    int64_t pos = nA + bpos[i];
    for (int64_t t = hr_off[c]; t < hr_off[c + 1]; t++) inv[pos++] = aux[by_head[t]];
  }
}
__global__ void perm_kernel(const int32_t* inv, int64_t np, int32_t* perm) {
  for (int64_t i = gtid(); i < np; i += gstride()) perm[inv[i]] = (int32_t)i;
}

struct InternalLen {
  const int32_t* inv;
  RowLen len;
  int64_t np;
  __device__ int64_t operator()(int64_t i) const { return i < np ? len(inv[i]) : 0; }
};
__global__ void row_ptr_kernel(const int64_t* scan, int64_t npad, int64_t nnz, int32_t* row_ptr) {
  for (int64_t i = gtid(); i <= npad; i += gstride()) row_ptr[i] = (int32_t)(i < npad ? scan[i] : nnz);
}
__global__ void ikind_kernel(const int32_t* inv, const int8_t* kind, int64_t np, int64_t npad, int8_t* ikind) {
  for (int64_t i = gtid(); i < npad; i += gstride()) ikind[i] = i < np ? kind[inv[i]] : (int8_t)K_EMPTY;
}

// Rule rows: each body mapped to internal ids, sorted when short (long ones are sorted below).
__global__ void rule_rows_kernel(const int64_t* off, const int32_t* setlen, int64_t n_rules, const int32_t* rb,
                                 const int32_t* aux, const int32_t* head, const int32_t* perm, const int32_t* row_ptr,
                                 int32_t* col, uint8_t* is_long) {
  for (int64_t r = gtid(); r < n_rules; r += gstride()) {
    const int32_t m = setlen[r];
    is_long[r] = m > kShortBody;
    if (m == 0) continue;  // a fact: its row is a self-loop
    const int32_t i = perm[aux[r] >= 0 ? aux[r] : head[r]];
    int32_t* d = col + row_ptr[i];
    const int32_t* sb = rb + off[r];
    for (int32_t t = 0; t < m; t++) d[t] = perm[sb[t]];
    if (m > kShortBody) continue;
    for (int a = 1; a < m; a++) {
      const int32_t x = d[a];
      int j = a - 1;
      while (j >= 0 && d[j] > x) {
        d[j + 1] = d[j];
        j--;
      }
      d[j + 1] = x;
    }
  }
}
// Row start of each long rule row (for the long-segment passes).
__global__ void rule_row_start_kernel(const uint8_t* flag, const int32_t* aux, const int32_t* head,
                                      const int32_t* perm, const int32_t* row_ptr, int64_t n_rules,
                                      int64_t* start) {
  for (int64_t r = gtid(); r < n_rules; r += gstride())
    if (flag[r]) start[r] = row_ptr[perm[aux[r] >= 0 ? aux[r] : head[r]]];
}

// Self-loop rows hold their own column, OR rows their run of new atoms; the OR-row mask.
__global__ void loop_or_rows_kernel(const int8_t* ikind, const int64_t* bpos, int64_t np, int64_t nA,
                                    const int32_t* row_ptr, int32_t* col) {
  for (int64_t i = gtid(); i < np; i += gstride()) {
    int32_t* d = col + row_ptr[i];
    if (ikind[i] == K_FACT || ikind[i] == K_BARRED) {
      *d = (int32_t)i;
    } else if (ikind[i] == K_OR) {
      for (int64_t t = bpos[i]; t < bpos[i + 1]; t++) *d++ = (int32_t)(nA + t);
    }
  }
}
__global__ void any_mask_kernel(const int8_t* ikind, int64_t npad, uint32_t* any_mask) {
  for (int64_t w = gtid(); w < npad / 32; w += gstride()) {
    uint32_t bits = 0;
    for (int l = 0; l < 32; l++)
      if (ikind[32 * w + l] == K_OR) bits |= 1u << l;
    any_mask[w] = bits;
  }
}

struct IsFact {
  const int8_t* kind;
  __device__ int64_t operator()(int64_t c) const { return kind[c] == K_FACT; }
};
// The original atom a row belongs to: itself, the atom of a barred row, the head of a new atom.
__device__ __forceinline__ int32_t owner_of(int64_t c, int32_t n, int32_t nb, const int32_t* bar_atom,
                                            const int32_t* aux_rule, const int32_t* head) {
  if (c < n) return (int32_t)c;
  if (c < (int64_t)n + nb) return bar_atom[c - n];
  return head[aux_rule[c - n - nb]];
}
// Fact rows in canonical order (Def. 4) and the atoms with a fact.
__global__ void facts_kernel(const int8_t* kind, const int64_t* rank, int64_t np, int32_t n, int32_t nb,
                             const int32_t* bar_atom, const int32_t* aux_rule, const int32_t* head,
                             const int32_t* perm, int32_t* fact_row, int32_t* fact_owner,
                             unsigned long long* fact_mask, int32_t* row_tag) {
  for (int64_t c = gtid(); c < np; c += gstride())
    if (kind[c] == K_FACT) {
      const int32_t a = owner_of(c, n, nb, bar_atom, aux_rule, head);
      fact_row[rank[c]] = perm[c];
      fact_owner[rank[c]] = a;
      atomicOr(fact_mask + (a >> 6), 1ull << (a & 63));
      row_tag[perm[c]] = -2;
    }
}
struct NotFactNegated {
  const int32_t* bar_atom;
  const unsigned long long* fact_mask;
  __device__ int64_t operator()(int64_t j) const {
    const int32_t a = bar_atom[j];
    return ((fact_mask[a >> 6] >> (a & 63)) & 1ull) ? 0 : 1;
  }
};
// Negated atoms (ascending): their rows, and the initial column of Def. 8 on the barred rows.
__global__ void guess_kernel(const int32_t* bar_atom, int32_t nb, int32_t n, const unsigned long long* fact_mask,
                             const int64_t* grank, const int32_t* perm, int32_t* neg_row, int32_t* bar_row,
                             int32_t* guess_row, int32_t* row_tag) {
  for (int64_t j = gtid(); j < nb; j += gstride()) {
    const int32_t a = bar_atom[j];
    const int32_t q = perm[a], qb = perm[n + j];
    neg_row[j] = q;
    bar_row[j] = qb;
    if ((fact_mask[a >> 6] >> (a & 63)) & 1ull) {
      row_tag[qb] = -3;
    } else {
      row_tag[qb] = (int32_t)grank[j];
      guess_row[grank[j]] = qb;
    }
  }
}
// Row counts by kind; the leading referenced section-A rows (order is by descending references).
__global__ void stats_kernel(const int8_t* kind, int64_t np, const int32_t* deg, int64_t nA,
                             unsigned long long* out) {
  unsigned long long rule = 0, orr = 0, refd = 0;
  for (int64_t c = gtid(); c < np; c += gstride()) {
    rule += kind[c] == K_RULE;
    orr += kind[c] == K_OR;
  }
  for (int64_t c = gtid(); c < nA; c += gstride()) refd += deg[c] > 0;
  rule = __reduce_add_sync(FULL, (unsigned)rule);
  orr = __reduce_add_sync(FULL, (unsigned)orr);
  refd = __reduce_add_sync(FULL, (unsigned)refd);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, rule);
    atomicAdd(out + 1, orr);
    atomicAdd(out + 2, refd);
  }
}
__global__ void canon_rule_kernel(const int8_t* kind, const int32_t* row_rule, int64_t np, int32_t* canon_rule) {
  for (int64_t c = gtid(); c < np; c += gstride()) canon_rule[c] = kind[c] == K_RULE ? row_rule[c] : -1;
}


#define DC_TRY(expr)                                \
  do {                                              \
    const cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return cuda_status(e_);  \
  } while (0)

lp_status cuda_status(cudaError_t e) {
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
              std::string("device compile: ") + cudaGetErrorString(e));
}

// Sorts the segments of the flagged rules in place: rule r's segment is data[off[r] ..
// off[r] + len[r]). Its entries become (key = entry, val = segment) pairs, sorted by entry and then,
// stably, by segment, and go back ascending (deduplicated into len[r] when `dedup`).
lp_status sort_long_segments(const uint8_t* flag, int64_t n_rules, const int64_t* off, int32_t* len, int32_t* data,
                             int key_bits, bool dedup, int64_t* tot, Scratch& sc) {
  cudaStream_t s = sc.s;
  int64_t* rank = sc.get<int64_t>((size_t)n_rules);
  int64_t* len_scan = sc.get<int64_t>((size_t)n_rules);
  if (!rank || !len_scan) return cuda_status(sc.err);
  DC_TRY(scan(LongFlag{flag}, n_rules, rank, tot, sc));
  DC_TRY(scan(LongLen{flag, len}, n_rules, len_scan, tot + 1, sc));
  int64_t h[2];
  DC_TRY(cudaMemcpyAsync(h, tot, 16, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  const int64_t n_seg = h[0], L = h[1];
  if (n_seg == 0) return LP_OK;
  int32_t* seg_src = sc.get<int32_t>((size_t)n_seg);
  int64_t* seg_first = sc.get<int64_t>((size_t)n_seg);
  uint32_t* keys = sc.get<uint32_t>((size_t)L);
  int32_t* vals = sc.get<int32_t>((size_t)L);
  uint32_t* tk = sc.get<uint32_t>((size_t)L);
  int32_t* tv = sc.get<int32_t>((size_t)L);
  if (!seg_src || !seg_first || !keys || !vals || !tk || !tv) return cuda_status(sc.err);
  long_list_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(flag, rank, len_scan, n_rules, seg_src, seg_first);
  long_gather_kernel<<<(unsigned)std::min<int64_t>(n_seg, 65535), kThreads, 0, s>>>(seg_first, seg_src, n_seg, off,
                                                                                   len, data, keys, vals);
  DC_TRY(cudaGetLastError());
  DC_TRY(radix_sort(keys, vals, tk, tv, L, key_bits, sc));
  DC_TRY(radix_sort((uint32_t*)vals, (int32_t*)keys, (uint32_t*)tv, (int32_t*)tk, L, bit_width((uint64_t)n_seg - 1),
                    sc));
  long_scatter_kernel<<<blocks_for(n_seg), kThreads, 0, s>>>(seg_first, seg_src, n_seg, off, len, keys, data, len,
                                                             dedup);
  DC_TRY(cudaGetLastError());
  return LP_OK;
}

}  // namespace

lp_status compile_on_device(lp_program* p, int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                            const int32_t* body_atom, const uint8_t* body_neg, cudaStream_t s) {
  HostMatrix& hm = p->hm;
  // ---- the checks that need no pass over the rules (the host compiler's messages)
  if (n < 0 || n_rules < 0) return fail(LP_ERR_INVALID, "negative atom or rule count");
  if (n_rules > 0 && (!head || !body_off)) return fail(LP_ERR_INVALID, "head/body_off must not be NULL when n_rules > 0");
  if (n_rules > 0 && body_off[0] != 0) return fail(LP_ERR_INVALID, "body_off[0] must be 0");
  if (n_rules >= (int64_t(1) << 31) - 1) return fail(LP_ERR_INVALID, "too many rules (must be < 2^31 - 1)");
  const int64_t total = n_rules > 0 ? body_off[n_rules] : 0;
  if (total > 0 && !body_atom) return fail(LP_ERR_INVALID, "body_atom must not be NULL when there are body literals");
  if (total < 0 || total >= (int64_t(1) << 31)) return fail(LP_ERR_INVALID, "too many body literals (must be < 2^31)");

  Scratch sc(s);
  auto oom = [&]() { return cuda_status(sc.err == cudaSuccess ? cudaErrorMemoryAllocation : sc.err); };
  // ---- the rules, as given
  int32_t* d_head = sc.get<int32_t>((size_t)n_rules);
  int64_t* d_off = sc.get<int64_t>((size_t)n_rules + 1);
  int32_t* rb = sc.get<int32_t>((size_t)total);  // the literals, then the bodies in canonical ids
  uint8_t* d_neg = body_neg ? sc.get<uint8_t>((size_t)total) : nullptr;
  int64_t* tot = sc.get<int64_t>(16);  // scan totals and small results
  unsigned long long* err = sc.get<unsigned long long>(8);
  if (!d_head || !d_off || !rb || (body_neg && !d_neg) || !tot || !err) return oom();
  if (n_rules > 0) {
    DC_TRY(cudaMemcpyAsync(d_head, head, (size_t)n_rules * 4, cudaMemcpyHostToDevice, s));
    DC_TRY(cudaMemcpyAsync(d_off, body_off, ((size_t)n_rules + 1) * 8, cudaMemcpyHostToDevice, s));
  }
  if (total > 0) {
    DC_TRY(cudaMemcpyAsync(rb, body_atom, (size_t)total * 4, cudaMemcpyHostToDevice, s));
    if (d_neg) DC_TRY(cudaMemcpyAsync(d_neg, body_neg, (size_t)total, cudaMemcpyHostToDevice, s));
  }
  p->upload_bytes += n_rules * 12 + 8 + total * (d_neg ? 5 : 4);
  DC_TRY(cudaMemsetAsync(err, 0xFF, 8 * 8, s));
  DC_TRY(cudaMemsetAsync(tot, 0, 16 * 8, s));
  const unsigned vblocks = blocks_for(std::max<int64_t>(n_rules, total));
  validate_kernel<<<std::min(vblocks, 4096u), kThreads, 0, s>>>(d_head, d_off, n_rules, rb, total, n, err);
  DC_TRY(cudaGetLastError());
  unsigned long long herr[2];
  DC_TRY(cudaMemcpyAsync(herr, err, 16, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  if (herr[0] != ~0ull) {
    const int64_t r = (int64_t)herr[0];
    return fail(LP_ERR_INVALID, (head[r] < 0 || head[r] >= n) ? "head atom out of range at rule " + std::to_string(r)
                                                              : "body_off decreases at rule " + std::to_string(r));
  }
  if (herr[1] != ~0ull) return fail(LP_ERR_INVALID, "body atom out of range");

  // ---- rules per head, negated atoms, barred ids, new atoms of multi-rule heads
  int32_t* cnt = sc.get<int32_t>((size_t)n);
  uint8_t* negated = sc.get<uint8_t>((size_t)n);
  int64_t* rank_n = sc.get<int64_t>((size_t)n);
  int32_t* bar_id = sc.get<int32_t>((size_t)n);
  int32_t* bar_atom = sc.get<int32_t>((size_t)n);
  int64_t* rank_r = sc.get<int64_t>((size_t)n_rules);
  int32_t* aux = sc.get<int32_t>((size_t)n_rules);
  int32_t* aux_rule = sc.get<int32_t>((size_t)n_rules);
  int32_t* setlen = sc.get<int32_t>((size_t)n_rules);
  uint8_t* is_long = sc.get<uint8_t>((size_t)n_rules);
  if (!cnt || !negated || !rank_n || !bar_id || !bar_atom || !rank_r || !aux || !aux_rule || !setlen || !is_long)
    return oom();
  DC_TRY(cudaMemsetAsync(cnt, 0, (size_t)std::max(n, 1) * 4, s));
  DC_TRY(cudaMemsetAsync(negated, 0, (size_t)std::max(n, 1), s));
  count_kernel<<<std::min(vblocks, 4096u), kThreads, 0, s>>>(d_head, n_rules, rb, d_neg, total, cnt, negated);
  DC_TRY(scan(FlagU8{negated}, n, rank_n, tot + 0, sc));
  bar_kernel<<<blocks_for(n), kThreads, 0, s>>>(negated, rank_n, n, bar_id, bar_atom);
  DC_TRY(scan(MultiRuleHead{d_head, cnt}, n_rules, rank_r, tot + 1, sc));
  int64_t h2[2];
  DC_TRY(cudaMemcpyAsync(h2, tot, 16, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  const int64_t nb64 = h2[0], naux = h2[1];
  const int64_t np64 = (int64_t)n + nb64 + naux;
  if (np64 >= (int64_t(1) << 31) - 128) return fail(LP_ERR_INVALID, "standardized program too large (n' must be < 2^31 - 128)");
  const int32_t nb = (int32_t)nb64, np = (int32_t)np64, nA = n + nb;
  const int32_t npad = (int32_t)(((int64_t)np + 63) / 64 * 64);
  aux_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(d_head, cnt, rank_r, n_rules, (int64_t)n + nb, aux, aux_rule);

  // ---- body sets in canonical columns (sorted, duplicates removed), in place per rule
  body_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(d_off, n_rules, rb, d_neg, bar_id, rb, setlen, is_long);
  raw_len_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(is_long, d_off, n_rules, setlen);
  DC_TRY(cudaGetLastError());
  lp_status st = sort_long_segments(is_long, n_rules, d_off, setlen, rb, bit_width((uint64_t)std::max(nA, 1) - 1), true,
                                    tot + 2, sc);
  if (st != LP_OK) return st;

  // ---- rules grouped by head, in rule order within a head (stable sort by head)
  int64_t* hr_off = sc.get<int64_t>((size_t)n + 1);
  uint32_t* keys = sc.get<uint32_t>((size_t)std::max<int64_t>(n_rules, nA));
  int32_t* by_head = sc.get<int32_t>((size_t)std::max<int64_t>(n_rules, nA));
  uint32_t* tk = sc.get<uint32_t>((size_t)std::max<int64_t>(n_rules, nA));
  int32_t* tv = sc.get<int32_t>((size_t)std::max<int64_t>(n_rules, nA));
  if (!hr_off || !keys || !by_head || !tk || !tv) return oom();
  DC_TRY(scan(CountI32{cnt}, n, hr_off, tot + 4, sc));
  DC_TRY(cudaMemcpyAsync(hr_off + n, tot + 4, 8, cudaMemcpyDeviceToDevice, s));
  iota_keys_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(d_head, n_rules, keys, by_head);
  DC_TRY(radix_sort(keys, by_head, tk, tv, n_rules, bit_width((uint64_t)std::max(n, 1) - 1), sc));

  // ---- row kinds and defining rules (canonical order)
  int8_t* kind = sc.get<int8_t>((size_t)np);
  int32_t* row_rule = sc.get<int32_t>((size_t)np);
  if (!kind || !row_rule) return oom();
  DC_TRY(cudaMemsetAsync(kind, K_EMPTY, (size_t)std::max(np, 1), s));
  DC_TRY(cudaMemsetAsync(row_rule, 0xFF, (size_t)std::max(np, 1) * 4, s));
  kind_rules_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(aux, setlen, n_rules, kind, row_rule);
  kind_atoms_kernel<<<blocks_for(n), kThreads, 0, s>>>(cnt, hr_off, by_head, setlen, bar_id, n, kind, row_rule);

  // ---- references per section-A column, and the internal order
  int32_t* deg = sc.get<int32_t>((size_t)nA);
  int32_t* inv = sc.get<int32_t>((size_t)np);
  int64_t* bpos = sc.get<int64_t>((size_t)nA + 1);
  if (!deg || !inv || !bpos) return oom();
  DC_TRY(cudaMemsetAsync(deg, 0, (size_t)std::max(nA, 1) * 4, s));
  deg_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(d_off, setlen, n_rules, rb, deg);
  unsigned* maxdeg = (unsigned*)(tot + 6);
  max_kernel<<<std::min(blocks_for(nA), 1024u), kThreads, 0, s>>>(deg, nA, maxdeg);
  unsigned hmax = 0;
  DC_TRY(cudaMemcpyAsync(&hmax, maxdeg, 4, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  order_keys_kernel<<<blocks_for(nA), kThreads, 0, s>>>(deg, nA, maxdeg, keys, inv);
  DC_TRY(radix_sort(keys, inv, tk, tv, nA, bit_width(hmax), sc));
  // section B: each OR row's new atoms, OR rows in section-A order
  DC_TRY(scan(NewAtoms{inv, kind, cnt}, nA, bpos, tot + 7, sc));
  DC_TRY(cudaMemcpyAsync(bpos + nA, tot + 7, 8, cudaMemcpyDeviceToDevice, s));
  section_b_kernel<<<blocks_for(nA), kThreads, 0, s>>>(bpos, nA, kind, hr_off, by_head, aux, inv);
  // the permutation and the internal CSR's row pointers
  lp_status st2;
  if ((st2 = dalloc(p, &p->perm, (size_t)np)) != LP_OK) return st2;
  perm_kernel<<<blocks_for(np), kThreads, 0, s>>>(inv, np, p->perm);
  int64_t* row_scan = sc.get<int64_t>((size_t)npad + 1);
  int8_t* ikind = sc.get<int8_t>((size_t)npad + 1);
  if (!row_scan || !ikind) return oom();
  const RowLen rl{kind, row_rule, setlen, cnt};
  DC_TRY(scan(InternalLen{inv, rl, np}, npad, row_scan, tot + 8, sc));
  int64_t h3[2];
  DC_TRY(cudaMemcpyAsync(&h3[0], tot + 7, 8, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaMemcpyAsync(&h3[1], tot + 8, 8, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  if (nA + h3[0] != np) return fail(LP_ERR_INVALID, "internal error: new atoms not covered by OR rows");
  const int64_t nnz = h3[1];
  if (nnz >= (int64_t(1) << 31)) return fail(LP_ERR_INVALID, "too many matrix entries (nnz must be < 2^31)");
  if ((st2 = dalloc(p, &p->row_ptr, (size_t)npad + 1)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->col, (size_t)std::max<int64_t>(nnz, 1))) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->any_mask, (size_t)npad / 32)) != LP_OK) return st2;
  row_ptr_kernel<<<blocks_for(npad + 1), kThreads, 0, s>>>(row_scan, npad, nnz, p->row_ptr);
  ikind_kernel<<<blocks_for(npad), kThreads, 0, s>>>(inv, kind, np, npad, ikind);

  // ---- the entries: rule rows (bodies mapped to internal ids and sorted), self-loops, OR rows
  rule_rows_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(d_off, setlen, n_rules, rb, aux, d_head, p->perm,
                                                            p->row_ptr, p->col, is_long);
  int64_t* start = sc.get<int64_t>((size_t)n_rules);
  if (!start) return oom();
  rule_row_start_kernel<<<blocks_for(n_rules), kThreads, 0, s>>>(is_long, aux, d_head, p->perm, p->row_ptr, n_rules,
                                                                 start);
  DC_TRY(cudaGetLastError());
  if ((st = sort_long_segments(is_long, n_rules, start, setlen, p->col, bit_width((uint64_t)std::max(np, 1) - 1), false,
                               tot + 10, sc)) != LP_OK)
    return st;
  loop_or_rows_kernel<<<blocks_for(np), kThreads, 0, s>>>(ikind, bpos, np, nA, p->row_ptr, p->col);
  if (npad > 0) any_mask_kernel<<<blocks_for(npad / 32), kThreads, 0, s>>>(ikind, npad, p->any_mask);

  // ---- facts (Def. 4), negated atoms and guesses (Def. 8), row tags
  int64_t* frank = sc.get<int64_t>((size_t)np);
  int64_t* grank = sc.get<int64_t>((size_t)nb);
  if (!frank || !grank) return oom();
  DC_TRY(scan(IsFact{kind}, np, frank, tot + 12, sc));
  int64_t n_fact = 0;
  DC_TRY(cudaMemcpyAsync(&n_fact, tot + 12, 8, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  const size_t mask_words = ((size_t)n + 63) / 64;
  if ((st2 = dalloc(p, &p->fact_row, (size_t)n_fact)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->fact_owner, (size_t)n_fact)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->fact_mask, mask_words)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->row_tag, (size_t)npad)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->neg_row, (size_t)nb)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->bar_row, (size_t)nb)) != LP_OK) return st2;
  int32_t* guess_row = sc.get<int32_t>((size_t)nb);
  unsigned long long* stats = (unsigned long long*)(tot + 13);  // three counters
  if (!guess_row) return oom();
  DC_TRY(cudaMemsetAsync(p->fact_mask, 0, std::max<size_t>(mask_words, 1) * 8, s));
  DC_TRY(cudaMemsetAsync(p->row_tag, 0xFF, (size_t)std::max(npad, 1) * 4, s));
  facts_kernel<<<blocks_for(np), kThreads, 0, s>>>(kind, frank, np, n, nb, bar_atom, aux_rule, d_head, p->perm,
                                                   p->fact_row, p->fact_owner, (unsigned long long*)p->fact_mask,
                                                   p->row_tag);
  DC_TRY(scan(NotFactNegated{bar_atom, (const unsigned long long*)p->fact_mask}, nb, grank, tot + 5, sc));
  guess_kernel<<<blocks_for(nb), kThreads, 0, s>>>(bar_atom, nb, n, (const unsigned long long*)p->fact_mask, grank,
                                                   p->perm, p->neg_row, p->bar_row, guess_row, p->row_tag);
  stats_kernel<<<std::min(blocks_for(np), 1024u), kThreads, 0, s>>>(kind, np, deg, nA, stats);
  // canonical kinds and rules stay on the device until a host-side user asks for them
  if ((st2 = dalloc(p, &p->dc_kind, (size_t)np)) != LP_OK) return st2;
  if ((st2 = dalloc(p, &p->dc_rule, (size_t)np)) != LP_OK) return st2;
  DC_TRY(cudaMemcpyAsync(p->dc_kind, kind, (size_t)np, cudaMemcpyDeviceToDevice, s));
  canon_rule_kernel<<<blocks_for(np), kThreads, 0, s>>>(kind, row_rule, np, p->dc_rule);
  DC_TRY(cudaGetLastError());
  int64_t k = 0;
  unsigned long long hs[3] = {0, 0, 0};
  DC_TRY(cudaMemcpyAsync(&k, tot + 5, 8, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaMemcpyAsync(hs, stats, 24, cudaMemcpyDeviceToHost, s));
  hm.neg_row.resize((size_t)nb);
  hm.bar_row.resize((size_t)nb);
  if (nb > 0) {
    DC_TRY(cudaMemcpyAsync(hm.neg_row.data(), p->neg_row, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
    DC_TRY(cudaMemcpyAsync(hm.bar_row.data(), p->bar_row, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
  }
  std::vector<int32_t> gr((size_t)nb);
  if (nb > 0) DC_TRY(cudaMemcpyAsync(gr.data(), guess_row, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
  DC_TRY(cudaStreamSynchronize(s));
  hm.guess_row.assign(gr.begin(), gr.begin() + k);

  hm.n = n;
  hm.n_rules = n_rules;
  hm.n_prime = np;
  hm.n_pad = npad;
  hm.nnz = nnz;
  hm.n_barred = nb;
  hm.n_aux = (int32_t)naux;
  hm.k = (int32_t)k;
  hm.n_fact_rows = (int32_t)n_fact;
  hm.n_rule_rows = (int32_t)hs[0];
  hm.n_or_rows = (int32_t)hs[1];
  hm.n_sec_a = (int32_t)hs[2];
  p->host_tables = false;
  return LP_OK;
}

// perm, canonical kinds and rules on the host, for the host-side users of a device compile.
lp_status ensure_host_tables(lp_program* p, cudaStream_t s) {
  if (p->host_tables) return LP_OK;
  HostMatrix& hm = p->hm;
  try {
    hm.perm.resize((size_t)hm.n_prime);
    hm.canon_kind.resize((size_t)hm.n_prime);
    hm.canon_rule.resize((size_t)hm.n_prime);
  } catch (const std::bad_alloc&) {
    return fail(LP_ERR_OOM, "host allocation failed");
  }
  if (hm.n_prime > 0) {
    LP_CUDA(cudaMemcpyAsync(hm.perm.data(), p->perm, (size_t)hm.n_prime * 4, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaMemcpyAsync(hm.canon_kind.data(), p->dc_kind, (size_t)hm.n_prime, cudaMemcpyDeviceToHost, s));
    LP_CUDA(cudaMemcpyAsync(hm.canon_rule.data(), p->dc_rule, (size_t)hm.n_prime * 4, cudaMemcpyDeviceToHost, s));
  }
  LP_CUDA(cudaStreamSynchronize(s));
  p->host_tables = true;
  return LP_OK;
}

}  // namespace lp

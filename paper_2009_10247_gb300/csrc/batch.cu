// batch.cu -- Algorithms 2 and 3 for many independent normal programs in one launch
// (lp_compile_batch / lp_batch_stable_models in include/lp.h).
//
// Each program is compiled on the host exactly as lp_compile does (compile_host), and the
// programs are laid end to end: one block-diagonal CSR (every program's rows and columns
// shifted by its row offset, a multiple of 64), one row-tag array (Def. 8 initial column), the
// negated / barred row pairs of every program, and one iterate region per program of
// n_pad x W 64-bit words, W = ceil(2^k / 64) guess words (all 2^k guesses of the program).
//
// One cooperative persistent kernel runs all programs in lock step: iteration t applies
// M_{t+1} = theta(M_P M_t) (rule row: AND of the body words; OR row / self-loop: OR) to every
// program that changed in iteration t-1, and skips the others, whose iterates are final (both
// buffers hold the fixpoint). The work unit is a warp task of 32 consecutive 64-bit words of
// one program's iterate (row-major, W words per row); warps walk the tasks grid-stride, so a
// large program is spread over the whole GPU and small ones share it. A per-program change flag
// (four rotating slots) records which programs stay active; one grid barrier per iteration.
// After the last iteration Algorithm 3 runs on every program's W words: stable word = AND over
// its negated atoms q of word(q) XOR word(q-bar).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "program.h"

namespace lp {

struct BatchProgram {       // device table entry
  int64_t row0;             // first global row (multiple of 64)
  int64_t state0;           // first 64-bit word of the program's iterate region (per buffer)
  int64_t mask0;            // first 64-bit word of the program's stable mask
  int32_t n_pad;            // rows (multiple of 64)
  int32_t W;                // guess words per row (a power of two)
  int32_t log2W;
  int32_t k;                // guessed barred atoms
  int32_t n_neg;            // negated atoms (barred rows)
  int32_t pad_;
  int64_t neg0;             // first entry of the program's negated / barred row pairs
};

constexpr int kBatchBlock = 512;
constexpr int kSlots = 4;  // rotating change-flag slots per program

__device__ __forceinline__ uint64_t batch_m0(int tag, int w) {
  if (tag == -2) return ~0ull;  // fact row (Def. 8 item 2)
  if (tag < 0) return 0ull;     // other rows; barred atoms of facts (item 3)
  switch (tag) {                // guess g = 64 w + b carries bit tag of g
    case 0: return 0xAAAAAAAAAAAAAAAAull;
    case 1: return 0xCCCCCCCCCCCCCCCCull;
    case 2: return 0xF0F0F0F0F0F0F0F0ull;
    case 3: return 0xFF00FF00FF00FF00ull;
    case 4: return 0xFFFF0000FFFF0000ull;
    case 5: return 0xFFFFFFFF00000000ull;
    default: return ((w >> (tag - 6)) & 1) ? ~0ull : 0ull;
  }
}

constexpr int kBatchGroup = 4096;  // programs per launch (their task counts live in shared memory)
// Matrix + iterate bytes per launch. Unlimited by default: launches of L2-sized groups (so a
// group's data stays in L2 across its iterations) were measured slower on the 1000-program
// workload (6.3 ms at 64 MB, 10.8 ms at 16 MB, against 5.4 ms for one launch): the extra
// grid barriers cost more than the DRAM traffic they save. LP_BATCH_GROUP_BYTES overrides it.
constexpr int64_t kGroupBytes = int64_t(1) << 62;
constexpr int kPerThread = kBatchGroup / kBatchBlock;
static_assert(kBatchGroup % kBatchBlock == 0, "group must be a multiple of the block");

struct BatchArgs {
  const BatchProgram* progs;  // all programs of the batch
  const int64_t* cell_off;    // n_total + 1: first iterate word of each program (ascending)
  const int64_t* mask_off;    // n_total + 1: first stable-mask word of each program
  int p0, n;                  // this launch runs programs [p0, p0 + n), n <= kBatchGroup
  const int64_t* row_ptr;
  const int32_t* col;
  const uint32_t* any_mask;
  const int32_t* row_tag;
  const int32_t* neg_row;
  const int32_t* bar_row;
  uint64_t* X0;
  uint64_t* X1;
  uint64_t* stable_mask;
  long long* n_stable;        // zeroed before the launch
  int32_t* iters;             // zeroed before the launch; 0 = no fixpoint within max_iters
  unsigned* pflag;            // kSlots per program, zeroed before the launch
  unsigned* gflag;            // kSlots: some program of this launch changed, zeroed before the launch
  DeviceCtl* ctl;             // one per launch, zeroed before it
  int max_iters;
};

// largest p in [0, n) with off[p] <= x (off ascending, off[0] <= x)
template <typename T>
__device__ __forceinline__ int last_le(const T* off, int n, long long x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((long long)off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// s_pre[q] = number of tasks of the active programs before program q (q = 0..n); every block
// computes the same array. A program is active in iteration `it` if it == 0 or it changed in
// iteration it - 1 (flag slot `prev`).
__device__ __forceinline__ void active_prefix(const BatchArgs& a, int it, int prev, const int* s_cnt, int* s_pre,
                                              int* s_wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kBatchBlock / 32;
  const int q0 = threadIdx.x * kPerThread;
  int v[kPerThread];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < kPerThread; j++) {
    const int q = q0 + j;
    int cnt = 0;
    if (q < a.n && (it == 0 || ld_volatile(a.pflag + (long long)(a.p0 + q) * kSlots + prev) != 0u)) cnt = s_cnt[q];
    v[j] = sum;
    sum += cnt;
  }
  int incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int x = lane < nw ? s_wsum[lane] : 0;
    const int own = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane < nw) s_wsum[lane] = x - own;  // exclusive over warps
    if (lane == nw - 1) s_pre[a.n] = x;     // total
  }
  __syncthreads();
  const int off = s_wsum[warp] + incl - sum;
#pragma unroll
  for (int j = 0; j < kPerThread; j++)
    if (q0 + j < a.n) s_pre[q0 + j] = off + v[j];
  __syncthreads();
}

__global__ void __launch_bounds__(kBatchBlock, 2) batch_stable_kernel(BatchArgs a) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int s_cnt[kBatchGroup];      // tasks (32-word units) of each program
  __shared__ int s_pre[kBatchGroup + 1];  // prefix of active tasks, rebuilt every iteration
  __shared__ int s_wsum[kBatchBlock / 32];
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const int64_t* coff = a.cell_off + a.p0;
  const BatchProgram* progs = a.progs + a.p0;
  DeviceCtl* ctl = a.ctl;
  unsigned long long round = 0;
  for (int q = threadIdx.x; q < a.n; q += blockDim.x) s_cnt[q] = (int)((__ldg(coff + q + 1) - __ldg(coff + q)) >> 5);
  const long long cell_base = __ldg(coff);
  const long long n_tasks = (__ldg(coff + a.n) - cell_base) >> 5;

  // ---- 1. M_0 of every program (Def. 8): all 2^k guesses as columns; warp w takes the
  // contiguous task range [n_tasks w / nwarps, n_tasks (w + 1) / nwarps)
  {
    const long long i0 = n_tasks * gwarp / nwarps, i1 = n_tasks * (gwarp + 1) / nwarps;
    if (i0 < i1) {
      int p = last_le(coff, a.n, cell_base + i0 * 32);
      BatchProgram pr = progs[p];
      long long p_end = __ldg(coff + p + 1);
      for (long long i = i0; i < i1; i++) {
        const long long c0 = cell_base + i * 32;
        while (c0 >= p_end) {
          ++p;
          pr = progs[p];
          p_end = __ldg(coff + p + 1);
        }
        const long long lc = c0 + lane - pr.state0;
        a.X0[c0 + lane] = batch_m0(__ldg(a.row_tag + pr.row0 + (lc >> pr.log2W)), (int)(lc & (pr.W - 1)));
      }
    }
  }
  if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) return;

  // ---- 2. lock-step fixpoint over the active programs' tasks, balanced over the warps
  bool all_done = false;
  for (int it = 0; it < a.max_iters; ++it) {
    const uint64_t* src = (it & 1) ? a.X1 : a.X0;
    uint64_t* dst = (it & 1) ? a.X0 : a.X1;
    const int slot = it % kSlots, prev = (it + kSlots - 1) % kSlots, next = (it + 1) % kSlots;
    // slot `next` was last read at the start of iteration it - 1: clear it for iteration it + 1
    for (long long q = gtid; q < a.n; q += nthreads) a.pflag[(a.p0 + q) * kSlots + next] = 0u;
    if (gtid == 0) a.gflag[next] = 0u;
    active_prefix(a, it, prev, s_cnt, s_pre, s_wsum);
    const long long total = s_pre[a.n];
    const long long i0 = total * gwarp / nwarps, i1 = total * (gwarp + 1) / nwarps;
    if (i0 < i1) {
      int p = last_le(s_pre, a.n, i0);
      BatchProgram pr = progs[p];
      long long p_hi = s_pre[p + 1], t_base = ((pr.state0 - cell_base) >> 5) - s_pre[p];
      bool flagged = false;
      for (long long i = i0; i < i1; i++) {
        if (i >= p_hi) {  // next active program
          do {
            ++p;
          } while (s_pre[p + 1] <= i);
          pr = progs[p];
          p_hi = s_pre[p + 1];
          t_base = ((pr.state0 - cell_base) >> 5) - s_pre[p];
          flagged = false;
        }
        const long long c = cell_base + (t_base + i) * 32 + lane;
        const long long lc = c - pr.state0;
        const long long gr = pr.row0 + (lc >> pr.log2W);
        const int w = (int)(lc & (pr.W - 1));
        const long long beg = __ldg(a.row_ptr + gr), end = __ldg(a.row_ptr + gr + 1);
        const bool any = (__ldg(a.any_mask + (gr >> 5)) >> (gr & 31)) & 1u;
        const uint64_t old = src[c];
        const uint64_t ident = any ? 0ull : ~0ull;  // identity of the row's OR / AND
        uint64_t acc = end > beg ? ident : 0ull;
        const uint64_t* base = src + pr.state0 + w;
        // four entries at a time: all column loads, then all gathers
        for (long long e = beg; e < end; e += 4) {
          int cc[4];
#pragma unroll
          for (int j = 0; j < 4; j++) cc[j] = e + j < end ? __ldg(a.col + e + j) : -1;
          uint64_t vv[4];
#pragma unroll
          for (int j = 0; j < 4; j++) vv[j] = cc[j] >= 0 ? base[(long long)(cc[j] - pr.row0) << pr.log2W] : ident;
          const uint64_t o = vv[0] | vv[1] | vv[2] | vv[3], n = vv[0] & vv[1] & vv[2] & vv[3];
          acc = any ? (acc | o) : (acc & n);
        }
        dst[c] = acc;
        if (__any_sync(FULL, acc != old) && !flagged) {
          flagged = true;
          if (lane == 0) {
            a.pflag[(long long)(a.p0 + p) * kSlots + slot] = 1u;
            a.gflag[slot] = 1u;
          }
        }
      }
    }
    if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) return;
    // programs that were active in iteration it and did not change have converged
    for (long long q = gtid; q < a.n; q += nthreads) {
      const unsigned* f = a.pflag + (a.p0 + q) * kSlots;
      if ((it == 0 || ld_volatile(f + prev) != 0u) && ld_volatile(f + slot) == 0u) a.iters[a.p0 + q] = it + 1;
    }
    if (ld_volatile(a.gflag + slot) == 0u) {
      all_done = true;
      break;
    }
  }
  if (!all_done && gtid == 0) atomicCAS(&ctl->status, 0, LP_ERR_NO_FIXPOINT);
  if (!grid_barrier(ctl, ++round, LP_ERR_TIMEOUT)) return;

  // ---- 3. Algorithm 3 on every program's guess words (either buffer holds the fixpoint)
  const int64_t* moff = a.mask_off + a.p0;
  const long long m_base = __ldg(moff), n_mask = __ldg(moff + a.n) - m_base;
  for (long long m = gtid; m < n_mask; m += nthreads) {
    const int p = last_le(moff, a.n, m_base + m);
    const BatchProgram pr = progs[p];
    const int w = (int)(m_base + m - pr.mask0);
    const long long first = 64ll * w, ng = 1ll << pr.k;
    uint64_t st = ng - first >= 64 ? ~0ull : ((1ull << (ng - first)) - 1ull);
    const uint64_t* fin = a.X0 + pr.state0 + w;
    for (int j = 0; j < pr.n_neg; j++) {
      const long long q = __ldg(a.neg_row + pr.neg0 + j), qb = __ldg(a.bar_row + pr.neg0 + j);
      st &= fin[q << pr.log2W] ^ fin[qb << pr.log2W];
    }
    if (ld_volatile(reinterpret_cast<const unsigned*>(a.iters + a.p0 + p)) == 0u) st = 0;
    a.stable_mask[m_base + m] = st;
    if (st)
      atomicAdd(reinterpret_cast<unsigned long long*>(a.n_stable + a.p0 + p), (unsigned long long)__popcll(st));
  }
}

}  // namespace lp

using namespace lp;

struct lp_batch {
  int device = 0, sm_count = 0;
  int32_t n_programs = 0;
  int32_t n_groups = 0;             // launches: consecutive programs, at most kBatchGroup of them
  std::vector<int32_t> group_start;  // n_groups + 1 program boundaries
  std::vector<lp_info> infos;           // per program
  std::vector<BatchProgram> table;      // host copy
  int64_t total_rows = 0, total_nnz = 0, total_state = 0, total_mask_words = 0;
  BatchProgram* d_table = nullptr;
  int64_t* d_cell_off = nullptr;
  int64_t* d_mask_off = nullptr;
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  uint32_t* d_any = nullptr;
  int32_t* d_tag = nullptr;
  int32_t* d_neg = nullptr;
  int32_t* d_bar = nullptr;
  uint64_t* d_x0 = nullptr;
  uint64_t* d_x1 = nullptr;
  int64_t* d_nstable = nullptr;
  int32_t* d_iters = nullptr;
  unsigned* d_pflag = nullptr;
  DeviceCtl* d_ctl = nullptr;
  uint64_t* d_stage = nullptr;  // staging for a host stable_mask
  int64_t device_bytes = 0;
  double compile_ms = 0;
  int64_t launches = 0;
};

namespace {

lp_status bfail(lp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

void batch_release(lp_batch* b) {
  void* ptrs[] = {b->d_table, b->d_cell_off, b->d_mask_off, b->d_row_ptr, b->d_col, b->d_any, b->d_tag,
                  b->d_neg,   b->d_bar,      b->d_x0,       b->d_x1,      b->d_nstable, b->d_iters,
                  b->d_pflag, b->d_ctl,      b->d_stage};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

template <typename T>
lp_status bupload(lp_batch* b, T** ptr, const T* src, size_t count, cudaStream_t s) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  cudaError_t e = device_malloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return bfail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
                 std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b->device_bytes += (int64_t)bytes;
  if (src && count) {
    e = cudaMemcpyAsync(*ptr, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bfail(LP_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
  }
  return LP_OK;
}

}  // namespace

extern "C" {

lp_status lp_compile_batch(int32_t n_programs, const int32_t* n_atoms, const int64_t* rule_off, const int32_t* head,
                           const int64_t* body_off, const int32_t* body_atom, const uint8_t* body_neg, uint32_t flags,
                           void* cuda_stream, lp_batch** out) {
  NvtxRange nvtx("lp_compile_batch");
  if (!out) return bfail(LP_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  if (flags != 0) return bfail(LP_ERR_INVALID, "flags must be 0");
  if (n_programs < 0 || (n_programs > 0 && (!n_atoms || !rule_off))) return bfail(LP_ERR_INVALID, "bad program list");
  if (n_programs > 0 && rule_off[0] != 0) return bfail(LP_ERR_INVALID, "rule_off[0] must be 0");
  for (int32_t p = 0; p < n_programs; p++)
    if (rule_off[p + 1] < rule_off[p]) return bfail(LP_ERR_INVALID, "rule_off decreases");
  auto t0 = std::chrono::steady_clock::now();
  std::vector<HostMatrix> hms(n_programs);
  std::vector<std::string> errs(n_programs);
  std::vector<int> rcs(n_programs, LP_OK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t p = 0; p < n_programs; p++) {
    const int64_t r0 = rule_off[p], nr = rule_off[p + 1] - r0;
    std::vector<int64_t> off((size_t)nr + 1);
    for (int64_t r = 0; r <= nr; r++) off[r] = body_off[r0 + r] - body_off[r0];
    const int64_t b0 = body_off[r0];
    rcs[p] = compile_host(n_atoms[p], nr, head + r0, off.data(), body_atom ? body_atom + b0 : nullptr,
                          body_neg ? body_neg + b0 : nullptr, hms[p], errs[p]);
  }
  for (int32_t p = 0; p < n_programs; p++)
    if (rcs[p] != LP_OK) return bfail((lp_status)rcs[p], "program " + std::to_string(p) + ": " + errs[p]);
  lp_batch* b = new (std::nothrow) lp_batch();
  if (!b) return bfail(LP_ERR_OOM, "host allocation failed");
  b->n_programs = n_programs;
  b->infos.resize(n_programs);
  b->table.resize(n_programs);
  int64_t row = 0, state = 0, mask = 0, nnz = 0, neg = 0;
  for (int32_t p = 0; p < n_programs; p++) {
    const HostMatrix& hm = hms[p];
    if (hm.k > 16) {
      delete b;
      return bfail(LP_ERR_TOO_MANY_GUESSES, "program " + std::to_string(p) + ": k > 16 guessed atoms");
    }
    BatchProgram& t = b->table[p];
    t.row0 = row;
    t.n_pad = hm.n_pad;
    t.log2W = hm.k > 6 ? hm.k - 6 : 0;
    t.W = 1 << t.log2W;
    t.k = hm.k;
    t.pad_ = 0;
    t.state0 = state;
    t.mask0 = mask;
    t.n_neg = (int32_t)hm.neg_row.size();
    t.neg0 = neg;
    row += hm.n_pad;
    state += (int64_t)hm.n_pad * t.W;
    mask += t.W;
    nnz += hm.nnz;
    neg += t.n_neg;
    lp_info& in = b->infos[p];
    std::memset(&in, 0, sizeof(in));
    in.n_atoms = hm.n;
    in.n_rules = hm.n_rules;
    in.n_prime = hm.n_prime;
    in.nnz = hm.nnz;
    in.n_barred = hm.n_barred;
    in.n_aux = hm.n_aux;
    in.k = hm.k;
    in.n_fact_rows = hm.n_fact_rows;
    in.n_and_rows = hm.n_rule_rows;
    in.n_or_rows = hm.n_or_rows;
  }
  b->total_rows = row;
  b->total_nnz = nnz;
  b->total_state = state;
  b->total_mask_words = mask;
  // block-diagonal concatenation (global row = program row offset + internal row)
  std::vector<int64_t> rp((size_t)row + 1, 0);
  std::vector<int32_t> cl((size_t)std::max<int64_t>(nnz, 1)), tag((size_t)std::max<int64_t>(row, 1)),
      ng((size_t)std::max<int64_t>(neg, 1)), br((size_t)std::max<int64_t>(neg, 1));
  std::vector<uint32_t> any((size_t)std::max<int64_t>(row / 32, 1), 0u);
  if (row >= (int64_t(1) << 31) - 64) {
    delete b;
    return bfail(LP_ERR_INVALID, "batch too large (rows must be < 2^31)");
  }
  {
    int64_t c = 0;
    for (int32_t p = 0; p < n_programs; p++) {
      const HostMatrix& hm = hms[p];
      const int64_t r0 = b->table[p].row0;
      for (int32_t r = 0; r < hm.n_pad; r++) {
        rp[r0 + r] = c + hm.row_ptr[r];
        tag[r0 + r] = hm.row_tag[r];
      }
      for (int64_t e = 0; e < hm.nnz; e++) cl[c + e] = (int32_t)(hm.col[e] + r0);
      for (size_t w = 0; w < hm.any_mask.size(); w++) any[(r0 >> 5) + w] = hm.any_mask[w];
      for (int32_t j = 0; j < b->table[p].n_neg; j++) {
        ng[b->table[p].neg0 + j] = (int32_t)(hm.neg_row[j] + 0);
        br[b->table[p].neg0 + j] = (int32_t)(hm.bar_row[j] + 0);
      }
      c += hm.nnz;
    }
    rp[row] = c;
  }
  std::vector<int64_t> cell_off((size_t)n_programs + 1), mask_off((size_t)n_programs + 1);
  for (int32_t p = 0; p < n_programs; p++) {
    cell_off[p] = b->table[p].state0;
    mask_off[p] = b->table[p].mask0;
  }
  cell_off[n_programs] = state;
  mask_off[n_programs] = mask;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  lp_status st = e == cudaSuccess ? LP_OK : bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (st == LP_OK) st = bupload(b, &b->d_table, b->table.data(), b->table.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_cell_off, cell_off.data(), cell_off.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_mask_off, mask_off.data(), mask_off.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_row_ptr, rp.data(), rp.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_col, cl.data(), (size_t)nnz, s);
  if (st == LP_OK) st = bupload(b, &b->d_any, any.data(), any.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_tag, tag.data(), (size_t)row, s);
  if (st == LP_OK) st = bupload(b, &b->d_neg, ng.data(), (size_t)neg, s);
  if (st == LP_OK) st = bupload(b, &b->d_bar, br.data(), (size_t)neg, s);
  if (st == LP_OK) st = bupload<uint64_t>(b, &b->d_x0, nullptr, (size_t)state, s);
  if (st == LP_OK) st = bupload<uint64_t>(b, &b->d_x1, nullptr, (size_t)state, s);
  if (st == LP_OK) st = bupload<int64_t>(b, &b->d_nstable, nullptr, (size_t)n_programs, s);
  if (st == LP_OK) st = bupload<int32_t>(b, &b->d_iters, nullptr, (size_t)n_programs, s);
  // Groups: consecutive programs whose matrix and iterates together fit the group budget (and
  // at most kBatchGroup of them), so that a group's data stays in L2 across its iterations.
  int64_t budget = kGroupBytes;
  if (const char* env = std::getenv("LP_BATCH_GROUP_BYTES")) budget = std::max<int64_t>(1, std::atoll(env));
  b->group_start.assign(1, 0);
  {
    int64_t bytes = 0;
    for (int32_t p = 0; p < n_programs; p++) {
      const BatchProgram& t = b->table[p];
      const int64_t pb = 8 * ((int64_t)t.n_pad + 1) + 4 * hms[p].nnz + 16 * (int64_t)t.n_pad * t.W;
      const int32_t in_group = p - b->group_start.back();
      if (in_group > 0 && (bytes + pb > budget || in_group == kBatchGroup)) {
        b->group_start.push_back(p);
        bytes = 0;
      }
      bytes += pb;
    }
    b->group_start.push_back(n_programs);
    if (n_programs == 0) b->group_start.assign(1, 0);
  }
  b->n_groups = (int32_t)b->group_start.size() - 1;
  if (st == LP_OK)
    st = bupload<unsigned>(b, &b->d_pflag, nullptr, ((size_t)n_programs + (size_t)b->n_groups) * kSlots, s);
  if (st == LP_OK) st = bupload<DeviceCtl>(b, &b->d_ctl, nullptr, (size_t)b->n_groups, s);
  if (st == LP_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (st != LP_OK) {
    batch_release(b);
    delete b;
    return st;
  }
  b->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = b;
  return LP_OK;
}

lp_status lp_batch_info(const lp_batch* b, int64_t* n_programs, int64_t* total_rows, int64_t* total_nnz,
                        int64_t* total_mask_words, int64_t* device_bytes) {
  if (!b) return bfail(LP_ERR_INVALID, "NULL batch");
  if (n_programs) *n_programs = b->n_programs;
  if (total_rows) *total_rows = b->total_rows;
  if (total_nnz) *total_nnz = b->total_nnz;
  if (total_mask_words) *total_mask_words = b->total_mask_words;
  if (device_bytes) *device_bytes = b->device_bytes;
  return LP_OK;
}

lp_status lp_batch_program_info(const lp_batch* b, int32_t program, lp_info* info, int64_t* mask_word_offset) {
  if (!b || program < 0 || program >= b->n_programs) return bfail(LP_ERR_INVALID, "bad program index");
  if (info) *info = b->infos[program];
  if (mask_word_offset) *mask_word_offset = b->table[program].mask0;
  return LP_OK;
}

lp_status lp_batch_stable_models(lp_batch* b, uint64_t* stable_mask, int64_t* n_stable, int32_t* iters,
                                 int32_t max_iters, void* cuda_stream) {
  NvtxRange nvtx("lp_batch_stable_models");
  if (!b) return bfail(LP_ERR_INVALID, "NULL batch");
  if (!stable_mask) return bfail(LP_ERR_INVALID, "stable_mask must not be NULL");
  if (max_iters < 1) return bfail(LP_ERR_INVALID, "max_iters must be >= 1");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const bool host_mask = !is_device_ptr(stable_mask);
  uint64_t* d_mask = stable_mask;
  if (host_mask) {
    if (!b->d_stage) {
      lp_status st = bupload<uint64_t>(b, &b->d_stage, nullptr, (size_t)b->total_mask_words, s);
      if (st != LP_OK) return st;
    }
    d_mask = b->d_stage;
  }
  cudaError_t e = cudaMemsetAsync(b->d_ctl, 0, std::max<size_t>(b->n_groups, 1) * sizeof(DeviceCtl), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_pflag, 0, ((size_t)b->n_programs + (size_t)b->n_groups) * kSlots * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_nstable, 0, std::max<size_t>(b->n_programs, 1) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_iters, 0, std::max<size_t>(b->n_programs, 1) * 4, s);
  if (e != cudaSuccess) return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  int per_sm = 0;
  if (b->n_programs > 0 &&
      (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_stable_kernel, kBatchBlock, 0) != cudaSuccess ||
       per_sm < 1))
    return bfail(LP_ERR_CUDA, "batch kernel cannot be resident");
  for (int32_t g = 0; g < b->n_groups; g++) {
    BatchArgs a{};
    a.progs = b->d_table;
    a.cell_off = b->d_cell_off;
    a.mask_off = b->d_mask_off;
    a.p0 = b->group_start[g];
    a.n = b->group_start[g + 1] - a.p0;
    a.row_ptr = b->d_row_ptr;
    a.col = b->d_col;
    a.any_mask = b->d_any;
    a.row_tag = b->d_tag;
    a.neg_row = b->d_neg;
    a.bar_row = b->d_bar;
    a.X0 = b->d_x0;
    a.X1 = b->d_x1;
    a.stable_mask = d_mask;
    a.n_stable = reinterpret_cast<long long*>(b->d_nstable);
    a.iters = b->d_iters;
    a.pflag = b->d_pflag;
    a.gflag = b->d_pflag + ((size_t)b->n_programs + g) * kSlots;
    a.ctl = b->d_ctl + g;
    a.max_iters = max_iters;
    // resident blocks only (grid barrier); fewer blocks make the barrier cheaper, and a grid
    // larger than the group's work gains nothing
    const int64_t words = b->table[a.p0 + a.n - 1].state0 + (int64_t)b->table[a.p0 + a.n - 1].n_pad *
                                                                b->table[a.p0 + a.n - 1].W -
                          b->table[a.p0].state0;
    const long long want = std::max<long long>(1, (words + kBatchBlock - 1) / kBatchBlock);
    const int grid = (int)std::min<long long>((long long)per_sm * b->sm_count, want);
    void* params[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)batch_stable_kernel, dim3(grid), dim3(kBatchBlock), params, 0, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(LP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    b->launches++;
    count_launches(1);
  }
  const bool sync = host_mask || n_stable || iters;
  if (host_mask && b->total_mask_words)
    if ((e = cudaMemcpyAsync(stable_mask, d_mask, (size_t)b->total_mask_words * 8, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (!sync) return LP_OK;
  int status = 0;
  if (n_stable && b->n_programs)
    if ((e = cudaMemcpyAsync(n_stable, b->d_nstable, (size_t)b->n_programs * 8, cudaMemcpyDefault, s)) != cudaSuccess)
      return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (iters && b->n_programs)
    if ((e = cudaMemcpyAsync(iters, b->d_iters, (size_t)b->n_programs * 4, cudaMemcpyDefault, s)) != cudaSuccess)
      return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  std::vector<DeviceCtl> ctls((size_t)std::max(b->n_groups, 1));
  if (b->n_groups &&
      (e = cudaMemcpyAsync(ctls.data(), b->d_ctl, (size_t)b->n_groups * sizeof(DeviceCtl), cudaMemcpyDeviceToHost,
                           s)) != cudaSuccess)
    return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  for (int32_t g = 0; g < b->n_groups; g++)
    if (ctls[g].status != 0 && (status == 0 || status == LP_ERR_NO_FIXPOINT)) status = ctls[g].status;
  if (status == LP_ERR_NO_FIXPOINT) return bfail(LP_ERR_NO_FIXPOINT, "a program reached max_iters");
  if (status != 0) return bfail((lp_status)status, "batch kernel gave up waiting at a grid barrier");
  return LP_OK;
}

void lp_batch_free(lp_batch* b) {
  if (!b) return;
  batch_release(b);
  delete b;
}

}  // extern "C"

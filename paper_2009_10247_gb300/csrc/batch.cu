// batch.cu -- Algorithms 2 and 3 for many independent normal programs in one launch
// (lp_compile_batch / lp_batch_stable_models in include/lp.h).
//
// Each program is compiled on the host exactly as lp_compile does (compile_host) and laid out
// as the sliced layout of the least-model kernel 2: rows renumbered by length within windows,
// 128-row groups padded to their longest row, entries column-major (program-local row ids), a
// 48-byte header per group. A row of a program's iterate holds its 2^k guess columns (Def. 8)
// in max(2, 2^k / 8) bytes, so programs with few guesses move few bytes.
//
// One cooperative persistent kernel takes the programs as jobs from a queue, largest first. A
// job runs its program's iteration M_{t+1} = theta(M_P M_t) (rule row: AND of its entries'
// rows; OR row / self-loop: OR; both one AND with an XOR mask) to the fixpoint on one block, or
// for the largest programs on several blocks that meet at the job's own barrier, then applies
// Algorithm 3: stable word = AND over the negated atoms q of word(q) XOR word(q-bar). Programs
// progress independently: no grid-wide barrier, and the data of the programs in flight stays
// in L2 across their iterations.
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
  int64_t state0;           // first byte of the program's iterate region (per buffer), 16-byte aligned
  int64_t mask0;            // first 64-bit word of the program's stable mask
  int64_t neg0;             // first entry of the program's negated / barred row pairs
  int64_t row0;             // first row of the program in the row-tag array
  int32_t g0;               // first group of the program (global group index)
  int32_t n_groups;         // 128-row groups of the program
  int32_t n_pad;            // rows (multiple of 64)
  int32_t rb;               // bytes per row of an iterate: max(2, 2^k / 8)
  int32_t k;                // guessed barred atoms
  int32_t n_neg;            // negated atoms (barred rows)
  int64_t tp0;              // frontier: first entry of the program's transposed row pointers
  int64_t seed0;            // frontier: first entry of the program's seed rows
  int32_t n_seed;           // frontier: rows nonzero in M_0 (fact rows, guessed rows)
  int32_t pad_;
};

constexpr int kBatchBlock = 512;          // full sweep: 512 threads, 2 blocks per SM
constexpr int kBatchFrontierBlock = 512;  // frontier: as many threads per program (its M_0 writes and lists)
constexpr int kGroupRows = 128;

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

// A job: one program, run by n_ctas co-resident blocks (ranks 0 .. n_ctas - 1) that meet at
// the job's own barrier once per iteration; a block takes the job's slot `first_slot + rank`.
struct BatchJob {
  int32_t program;
  int32_t n_ctas;
  int32_t first_slot;
  int32_t pad_;
};

struct BatchArgs {
  const BatchProgram* progs;
  const BatchJob* jobs;
  const int32_t* slot_job;    // n_slots: the job of each slot, multi-block jobs first
  int32_t n_slots;
  const int4* hdr;            // 3 per group: {first entry, width, 0, 0}, OR masks, empty masks
  const int32_t* col;         // entries: program-local row ids in the program's sliced numbering
  const int32_t* row_tag;     // per row (sliced numbering): -1 zero, -2 fact, -3 barred atom of a fact, j guess bit
  const int32_t* neg_row;
  const int32_t* bar_row;
  unsigned char* X0;
  unsigned char* X1;
  uint64_t* stable_mask;
  long long* n_stable;        // zeroed before the launch
  int32_t* iters;             // zeroed before the launch; 0 = no fixpoint within max_iters
  unsigned long long* job_bar;  // 4 per job: three rotating barrier counters, zeroed before the launch
  unsigned* queue;            // next slot, zeroed before the launch
  DeviceCtl* ctl;             // status and abort flag, zeroed before the launch
  int max_iters;
  // frontier schedule (programs with rows of at most 32 bytes): per program its transposed
  // matrix (tptr: global offsets into tidx, which holds program-local rows) and seed rows; per
  // row a stamp; two lists of program-local rows per program (list + row0 and
  // list + total_rows + row0); three rotating list sizes per program
  bool frontier;
  const int32_t* tptr;
  const int32_t* tidx;
  const int32_t* seed;
  unsigned* mark;
  int32_t* list;
  unsigned* fcnt;
  int64_t total_rows;
  // the iterate buffers of a frontier program rest between solves in M_0's guess-independent
  // part (fact rows all ones, other rows zero); a bit per row that changed in this solve; per
  // program 1 while its rest state is valid, and its next unused stamp
  unsigned* dirty;
  unsigned* clean;
  unsigned* epoch;
  // From F: the fixpoint every program reaches from its fact rows with every guessed row zero
  // (a bit per row, fbits) is where its columns start and where its buffers rest; the F pass
  // (f_pass) computes it once per batch, from M_0 with the guessed rows kept at zero.
  bool from_f;
  bool f_pass;
  unsigned* fbits;
};

// The value of a non-guessed row at rest (every column alike): its bit of F where F is known,
// else M_0's (ones on a fact row).
__device__ __forceinline__ bool batch_rest_one(const BatchArgs& a, const BatchProgram& pr, int r, int tag, bool use_f) {
  if (use_f) {
    const long long q = pr.row0 + r;
    return (a.fbits[q >> 5] >> (q & 31)) & 1u;
  }
  return tag == -2;
}

// ---- one row of an iterate: 8 RB bits (RB = 2, 4, 8, 16 or 32 bytes), as NW 64-bit words
template <int RB>
struct RowT {
  static constexpr int NW = RB >= 8 ? RB / 8 : 1;
  static constexpr uint64_t MASK = RB >= 8 ? ~0ull : ((1ull << (8 * RB)) - 1ull);
  uint64_t v[NW];
  __device__ __forceinline__ void load(const unsigned char* base, int r) {
    if constexpr (RB == 2) v[0] = *reinterpret_cast<const uint16_t*>(base + 2ll * r);
    else if constexpr (RB == 4) v[0] = *reinterpret_cast<const uint32_t*>(base + 4ll * r);
    else if constexpr (RB == 8) v[0] = *reinterpret_cast<const uint64_t*>(base + 8ll * r);
    else {
      const ulonglong2* q = reinterpret_cast<const ulonglong2*>(base + (long long)RB * r);
#pragma unroll
      for (int i = 0; i < NW / 2; i++) {
        const ulonglong2 t = q[i];
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
      }
    }
  }
  __device__ __forceinline__ void store(unsigned char* base, int r) const {
    if constexpr (RB == 2) *reinterpret_cast<uint16_t*>(base + 2ll * r) = (uint16_t)v[0];
    else if constexpr (RB == 4) *reinterpret_cast<uint32_t*>(base + 4ll * r) = (uint32_t)v[0];
    else if constexpr (RB == 8) *reinterpret_cast<uint64_t*>(base + 8ll * r) = v[0];
    else {
      ulonglong2* q = reinterpret_cast<ulonglong2*>(base + (long long)RB * r);
#pragma unroll
      for (int i = 0; i < NW / 2; i++) q[i] = make_ulonglong2(v[2 * i], v[2 * i + 1]);
    }
  }
};

// Group of 128 rows of one program, rows of up to 32 bytes: lane l owns rows l, 32 + l,
// 64 + l, 96 + l; slot k of the group holds their k-th entries as one int4 at entry
// off + 4 (32 k + l). Rule rows AND their entries, OR rows OR them (an AND of the complements,
// complemented), empty rows are 0. This pass evaluates rows U0 .. U0 + NU - 1 of the four (all
// four for rows of up to 8 bytes, two at a time above, to bound the registers). Returns whether
// one of them changed.
template <int RB, int U0, int NU>
__device__ __forceinline__ bool group_rows(const BatchArgs& a, const int4 h0, const int4 h1, const int4 h2,
                                           const unsigned char* src, unsigned char* dst, int lg, int n_pad, int lane) {
  using Row = RowT<RB>;
  constexpr int NW = Row::NW;
  const int K = h0.y;
  const uint32_t orm[4] = {(uint32_t)h1.x, (uint32_t)h1.y, (uint32_t)h1.z, (uint32_t)h1.w};
  uint64_t inv[NU], acc[NU][NW];
#pragma unroll
  for (int u = 0; u < NU; u++) {
    inv[u] = ((orm[U0 + u] >> lane) & 1u) ? Row::MASK : 0ull;
#pragma unroll
    for (int i = 0; i < NW; i++) acc[u][i] = ~0ull;
  }
  const int4* e = reinterpret_cast<const int4*>(a.col + h0.x) + lane;
  for (int k = 0; k < K; k++) {
    const int4 c = __ldg(e + 32 * k);
    const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
    for (int u = 0; u < NU; u++) {
      Row x;
      x.load(src, cc[U0 + u]);
#pragma unroll
      for (int i = 0; i < NW; i++) acc[u][i] &= x.v[i] ^ inv[u];
    }
  }
  const uint32_t emm[4] = {(uint32_t)h2.x, (uint32_t)h2.y, (uint32_t)h2.z, (uint32_t)h2.w};
  bool changed = false;
#pragma unroll
  for (int u = 0; u < NU; u++) {
    const int r = lg * kGroupRows + 32 * (U0 + u) + lane;
    if (r >= n_pad) break;  // the last group of a program may end 64 rows early (uniform in the warp)
    const uint64_t keep = ((emm[U0 + u] >> lane) & 1u) ? 0ull : Row::MASK;
    Row old, nw;
    old.load(src, r);
#pragma unroll
    for (int i = 0; i < NW; i++) {
      nw.v[i] = (acc[u][i] ^ inv[u]) & keep;
      changed |= nw.v[i] != old.v[i];
    }
    nw.store(dst, r);
  }
  return changed;
}

template <int RB>
__device__ __forceinline__ bool group_narrow(const BatchArgs& a, const int4 h0, const int4 h1, const int4 h2,
                                             const unsigned char* src, unsigned char* dst, int lg, int n_pad, int lane) {
  if constexpr (RB <= 8) {
    return group_rows<RB, 0, 4>(a, h0, h1, h2, src, dst, lg, n_pad, lane);
  } else {
    const bool c0 = group_rows<RB, 0, 2>(a, h0, h1, h2, src, dst, lg, n_pad, lane);
    const bool c1 = group_rows<RB, 2, 2>(a, h0, h1, h2, src, dst, lg, n_pad, lane);
    return c0 || c1;
  }
}

// Group of 128 rows whose rows hold more than 32 bytes (k > 8): the rows one after another,
// the lanes over a row's 64-bit words.
__device__ __forceinline__ bool group_wide(const BatchArgs& a, const int4 h0, const int4 h1, const int4 h2,
                                           const uint64_t* src, uint64_t* dst, int lg, int NW, int n_pad, int lane) {
  const int K = h0.y;
  bool changed = false;
  for (int t = 0; t < kGroupRows && lg * kGroupRows + t < n_pad; t++) {
    const int u = t >> 5, l = t & 31;
    const uint32_t orm = u == 0 ? (uint32_t)h1.x : u == 1 ? (uint32_t)h1.y : u == 2 ? (uint32_t)h1.z : (uint32_t)h1.w;
    const uint32_t emm = u == 0 ? (uint32_t)h2.x : u == 1 ? (uint32_t)h2.y : u == 2 ? (uint32_t)h2.z : (uint32_t)h2.w;
    const uint64_t inv = ((orm >> l) & 1u) ? ~0ull : 0ull;
    const uint64_t keep = ((emm >> l) & 1u) ? 0ull : ~0ull;
    const long long r = (long long)lg * kGroupRows + t;
    for (int w = lane; w < NW; w += 32) {
      uint64_t acc = ~0ull;
      for (int k = 0; k < K; k++) {
        const int c = __ldg(a.col + h0.x + 4 * (32 * k + l) + u);
        acc &= src[(long long)c * NW + w] ^ inv;
      }
      const uint64_t nw = (acc ^ inv) & keep;
      changed |= nw != src[r * NW + w];
      dst[r * NW + w] = nw;
    }
  }
  return changed;
}

// Barrier of the c blocks of one job (c > 1), carrying an OR of one flag: as grid_barrier_or,
// on the job's own counters. Returns false if the launch is aborting.
__device__ __forceinline__ bool job_barrier_or(const BatchArgs& a, int job, int rank, int c, unsigned long long round,
                                               bool flag, bool* any_flag) {
  __shared__ unsigned s_state;
  const int mine = __syncthreads_or(flag);
  if (threadIdx.x == 0) {
    unsigned long long* base = a.job_bar + 4ll * job;
    unsigned long long* slot = base + round % 3;
    if (rank == 0) base[(round + 1) % 3] = 0ull;
    red_release_add64(slot, mine ? (1ull << 32) + 1ull : 1ull);
    unsigned polls = 0;
    unsigned long long t0 = 0, v;
    unsigned ab = 0;
    while (((v = ld_acquire64(slot)) & 0xffffffffull) < (unsigned long long)c) {
      if (++polls == 1024) t0 = global_ns();
      if (polls > 1024 && (polls & 63) == 0) {
        if ((ab = ld_volatile(&a.ctl->abort)) != 0) break;
        __nanosleep(32);
        if (global_ns() - t0 > kWaitLimitNs) {
          atomicExch(&a.ctl->abort, 1u);
          atomicCAS(&a.ctl->status, 0, LP_ERR_TIMEOUT);
          atomicExch(&a.ctl->timeout_site, round);
          ab = 1;
          break;
        }
      }
    }
    s_state = (ab ? 1u : 0u) | ((v >> 32) ? 2u : 0u);
  }
  __syncthreads();
  const unsigned st = s_state;
  *any_flag = (st & 2u) != 0;
  return (st & 1u) == 0;
}

// Frontier schedule of one job (rows of RB <= 32 bytes: a lane per row). Row i of M_{t+1} depends
// only on the rows that row i of M_P refers to, so iteration t evaluates only the rows of a list:
// those that changed in iteration t - 1 and the rows that refer to them (the transposed matrix,
// deduplicated by a per-row stamp); with two buffers an unevaluated row keeps the right value
// (dst held M_{t-1}, equal to M_t and M_{t+1} on it). Iteration 0 starts from the rows nonzero in
// M_0 (fact rows, guessed rows) and the rows that refer to them: theta of a row whose inputs are
// all zero is zero. The iterates, the iteration count and the fixpoint are the full sweep's.
// Returns false if the launch is aborting; *it and *converged as the full sweep's.
template <int RB>
__device__ bool frontier_job(const BatchArgs& a, const BatchProgram& pr, int program, int j, int rank, int c,
                             int r_lo, int r_hi, unsigned long long& round, int* it_out, bool* converged_out,
                             int (*s_push)[3][32], unsigned* epoch_out) {
  using Row = RowT<RB>;
  constexpr int NW = Row::NW;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* const s_incl = s_push[warp][0];  // this warp's prefix sums, transposed row starts, rows
  int* const s_tb = s_push[warp][1];
  int* const s_row = s_push[warp][2];
  const unsigned lt = (1u << lane) - 1u;
  unsigned char* const xs[2] = {a.X0 + pr.state0, a.X1 + pr.state0};
  unsigned* const mark = a.mark + pr.row0;
  unsigned* const cnt = a.fcnt + 3ll * program;
  int32_t* const lists[2] = {a.list + pr.row0, a.list + a.total_rows + pr.row0};
  const int32_t* const tptr = a.tptr + pr.tp0;
  const long long tid = (long long)rank * blockDim.x + threadIdx.x, nth = (long long)c * blockDim.x;
  const long long warp0 = tid - lane;  // first item index of this warp in each round
  unsigned n_rows = 0, n_ent = 0;
  unsigned long long n_bytes = 0;  // bytes the schedule touches (lp_batch_last_stats)
  bool dummy;
  auto barrier = [&]() -> bool {
    if (c > 1) return job_barrier_or(a, j, rank, c, ++round, false, &dummy);
    __syncthreads();
    return true;
  };
  // appends `value` of every lane whose flag is set to the list (one atomic per warp)
  auto append = [&](int32_t* list, unsigned* counter, bool flag, int value) {
    const unsigned m = __ballot_sync(FULL, flag);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned)__popc(m));
    base = __shfl_sync(FULL, base, leader);
    if (flag) list[base + __popc(m & lt)] = value;
  };
  // Every lane with `ch` pushes its row and the rows referring to it (stamp `stamp`): the
  // warp's (row, dependent) pairs are spread over its lanes, 32 per round, a lane finding its
  // pair's row by binary search over the warp's prefix sums.
  auto push = [&](bool ch, int row, unsigned stamp, int32_t* list, unsigned* counter) {
    int tb = 0, per = 0;
    if (ch) {
      tb = __ldg(tptr + row);
      per = 1 + __ldg(tptr + row + 1) - tb;
      n_bytes += 8ull + 12ull * (unsigned)per;  // row pointers; per item its id, stamp, list slot
    }
    int incl = per;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    if (total == 0) return;
    s_incl[lane] = incl;
    s_tb[lane] = tb;
    s_row[lane] = row;
    __syncwarp();
    for (int q0 = 0; q0 < total; q0 += 32) {
      const int q = q0 + lane;
      bool win = false;
      int item = 0;
      if (q < total) {
        int lo = 0, hi = 31;  // first lane whose inclusive sum exceeds q
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_incl[mid] > q) hi = mid;
          else lo = mid + 1;
        }
        const int first = lo == 0 ? 0 : s_incl[lo - 1];
        const int d = q - first;
        item = d == 0 ? s_row[lo] : __ldg(a.tidx + s_tb[lo] + d - 1);
        win = atomicExch(mark + item, stamp) != stamp;
      }
      append(list, counter, win, item);
    }
    __syncwarp();
  };

  // ---- 1. M_0 (Def. 8). In the rest state only the guessed rows differ from it: write those into
  // X0 (iteration 0 evaluates them, so X1 need not hold them). Otherwise (first solve, a solve
  // that did not finish, stamps about to wrap) the block writes M_0 for its rows into both
  // buffers, four rows per thread (rows come in 128-row groups, so a thread's four are whole),
  // and clears their stamps and changed bits.
  // From F (not in the F pass) the rows rest at F and the columns start from F; the F pass keeps
  // the guessed rows at zero and starts from M_0's other rows.
  const bool at_f = a.from_f && !a.f_pass;
  unsigned e = ld_volatile(a.epoch + program);
  const bool clean = ld_volatile(a.clean + program) != 0u && e < 0xF0000000u - (unsigned)a.max_iters;
  if (!clean) e = 0u;
  if (clean) {
    if (!a.f_pass)
      for (long long i = tid; i < pr.n_seed; i += nth) {
        const int row = __ldg(a.seed + pr.seed0 + i);
        const int tag = __ldg(a.row_tag + pr.row0 + row);
        if (tag >= 0) {
          Row m0;
#pragma unroll
          for (int w = 0; w < NW; w++) m0.v[w] = batch_m0(tag, w) & Row::MASK;
          m0.store(xs[0], row);
        }
      }
  } else {
    for (int r = r_lo + 4 * threadIdx.x; r < r_hi; r += 4 * blockDim.x) {
      const int4 tag4 = *reinterpret_cast<const int4*>(a.row_tag + pr.row0 + r);
      const int tags[4] = {tag4.x, tag4.y, tag4.z, tag4.w};
#pragma unroll
      for (int i = 0; i < 4; i++) {
        Row m0;
        const bool one = tags[i] < 0 && batch_rest_one(a, pr, r + i, tags[i], at_f);
#pragma unroll
        for (int w = 0; w < NW; w++)
          m0.v[w] = (tags[i] >= 0 ? (a.f_pass ? 0ull : batch_m0(tags[i], w)) : (one ? ~0ull : 0ull)) & Row::MASK;
        m0.store(xs[0], r + i);
        m0.store(xs[1], r + i);
      }
      *reinterpret_cast<uint4*>(mark + r) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int w = r_lo / 32 + threadIdx.x; w < r_hi / 32; w += blockDim.x) a.dirty[pr.row0 / 32 + w] = 0u;
  }
  if (rank == 0 && threadIdx.x < 3) cnt[threadIdx.x] = 0u;
  if (!barrier()) return false;
  if (rank == 0 && threadIdx.x == 0) a.clean[program] = 0u;  // every block has read it: in use
  // ---- 2. the first list: seed rows and the rows referring to them (from F the guessed rows
  // alone; in the F pass the fact rows alone, the guessed rows staying zero)
  for (long long base = warp0; base < pr.n_seed; base += nth) {  // uniform in the warp
    const long long i = base + lane;
    bool ok = i < pr.n_seed;
    const int row = ok ? __ldg(a.seed + pr.seed0 + i) : 0;
    if (ok && a.from_f) {
      const int tag = __ldg(a.row_tag + pr.row0 + row);
      ok = a.f_pass ? tag < 0 : tag >= 0;
    }
    push(ok, row, e + 1u, lists[0], cnt);
  }
  if (!barrier()) return false;
  // ---- 3. the iterations
  int t = 0;
  bool converged = false;
  for (; t < a.max_iters; ++t) {
    const unsigned char* src = xs[t & 1];
    unsigned char* dst = xs[(t + 1) & 1];
    const int32_t* cur = lists[t & 1];
    int32_t* nxt = lists[(t + 1) & 1];
    unsigned* nxt_cnt = cnt + (t + 1) % 3;
    if (rank == 0 && threadIdx.x == 0) cnt[(t + 2) % 3] = 0u;  // last read as iteration t - 1's size
    const long long n_cur = ld_volatile(cnt + t % 3);
    for (long long base = warp0; base < n_cur; base += nth) {  // uniform in the warp
      const long long i = base + lane;
      bool ch = false;
      int r = 0;
      if (i < n_cur) {
        r = cur[i];
        const int gg = pr.g0 + (r >> 7), tt = r & 127, u = tt >> 5, l = tt & 31;
        Row old;
        old.load(src, r);  // independent of the header: in flight with it
        const int4 h0 = __ldg(a.hdr + 3 * gg), h1 = __ldg(a.hdr + 3 * gg + 1), h2 = __ldg(a.hdr + 3 * gg + 2);
        const uint32_t orm = u == 0 ? (uint32_t)h1.x : u == 1 ? (uint32_t)h1.y : u == 2 ? (uint32_t)h1.z : (uint32_t)h1.w;
        const uint32_t emm = u == 0 ? (uint32_t)h2.x : u == 1 ? (uint32_t)h2.y : u == 2 ? (uint32_t)h2.z : (uint32_t)h2.w;
        const uint64_t inv = ((orm >> l) & 1u) ? Row::MASK : 0ull, keep = ((emm >> l) & 1u) ? 0ull : Row::MASK;
        const int K = h0.y;
        uint64_t acc[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) acc[w] = ~0ull;
        const int32_t* e = a.col + h0.x + 4 * l + u;
        for (int k = 0; k < K; k += 4) {  // four entries' ids, then their rows
          int cc[4];
#pragma unroll
          for (int q = 0; q < 4; q++) cc[q] = k + q < K ? __ldg(e + 128 * (k + q)) : -1;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            if (cc[q] >= 0) {
              Row x;
              x.load(src, cc[q]);
#pragma unroll
              for (int w = 0; w < NW; w++) acc[w] &= x.v[w] ^ inv;
            }
          }
        }
        Row nw;
#pragma unroll
        for (int w = 0; w < NW; w++) {
          nw.v[w] = (acc[w] ^ inv) & keep;
          ch |= nw.v[w] != old.v[w];
        }
        nw.store(dst, r);
        if (ch) atomicOr(a.dirty + ((pr.row0 + r) >> 5), 1u << ((pr.row0 + r) & 31));
        n_rows++;
        n_ent += (unsigned)K;
        // list slot, header, entries and their gathered rows, the row's old and new words
        n_bytes += 4ull + 48ull + (unsigned long long)K * (4 + RB) + 2ull * RB;
      }
      push(ch, r, e + (unsigned)t + 2u, nxt, nxt_cnt);
    }
    if (!barrier()) return false;
    if (ld_volatile(nxt_cnt) == 0u) {
      converged = true;
      ++t;
      break;
    }
  }
  n_rows = __reduce_add_sync(FULL, n_rows);
  n_ent = __reduce_add_sync(FULL, n_ent);
  for (int o = 16; o > 0; o >>= 1) n_bytes += __shfl_xor_sync(FULL, n_bytes, o);
  if (lane == 0) {
    if (n_rows) atomicAdd(&a.ctl->fr_rows, (unsigned long long)n_rows);
    if (n_ent) atomicAdd(&a.ctl->fr_entries, (unsigned long long)n_ent);
    if (n_bytes) atomicAdd(&a.ctl->fr_list, n_bytes);  // the batch keeps its byte count here
  }
  *it_out = t;
  *converged_out = converged;
  *epoch_out = e + (unsigned)t + 2u;  // the next solve's first stamp
  return true;
}

// After Algorithm 3: the rows of [r_lo, r_hi) that changed in this solve, and (rank 0) the
// guessed rows, back to the rest state in both buffers (from F, and after the F pass, F; else
// M_0's guess-independent part); their changed bits cleared.
template <int RB>
__device__ void frontier_reset(const BatchArgs& a, const BatchProgram& pr, int rank, int c, int r_lo, int r_hi) {
  using Row = RowT<RB>;
  constexpr int NW = Row::NW;
  unsigned char* const xs[2] = {a.X0 + pr.state0, a.X1 + pr.state0};
  for (int w = r_lo / 32 + threadIdx.x; w < r_hi / 32; w += blockDim.x) {
    unsigned bits = a.dirty[pr.row0 / 32 + w];
    if (bits == 0u) continue;
    a.dirty[pr.row0 / 32 + w] = 0u;
    while (bits) {
      const int r = 32 * w + __ffs(bits) - 1;
      bits &= bits - 1;
      const int tag = __ldg(a.row_tag + pr.row0 + r);
      const bool one = tag < 0 && batch_rest_one(a, pr, r, tag, a.from_f);  // F: known by now
      Row v;
#pragma unroll
      for (int i = 0; i < NW; i++) v.v[i] = one ? Row::MASK : 0ull;
      v.store(xs[0], r);
      v.store(xs[1], r);
    }
  }
  if (rank == 0)
    for (int i = threadIdx.x; i < pr.n_seed; i += blockDim.x) {
      const int row = __ldg(a.seed + pr.seed0 + i);
      if (__ldg(a.row_tag + pr.row0 + row) >= 0) {
        Row z;
#pragma unroll
        for (int k = 0; k < NW; k++) z.v[k] = 0ull;
        z.store(xs[0], row);
        z.store(xs[1], row);
      }
    }
  (void)c;
}

// Algorithms 2 and 3 for every program, one job at a time per block: a block takes the next
// slot of the queue, runs its share of that job's program (a contiguous range of its 128-row
// groups; the block's warps claim them from a shared counter) to the program's fixpoint, and
// takes the next slot. Programs progress independently, so the data of the programs being
// solved at any moment stays in L2 across their iterations.
template <int BLOCK, bool FRONTIER>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) batch_stable_kernel(BatchArgs a) {
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ int s_slot, s_next;
  __shared__ int s_push[FRONTIER ? BLOCK / 32 : 1][3][32];  // frontier pushes: per-warp scratch
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_slot = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int slot = s_slot;
    if (slot >= a.n_slots) return;
    const int j = __ldg(a.slot_job + slot);
    const BatchJob job = a.jobs[j];
    const int rank = slot - job.first_slot, c = job.n_ctas;
    const BatchProgram pr = a.progs[job.program];
    if (a.f_pass && !(FRONTIER && pr.rb <= 32)) {  // the F pass serves the frontier programs only
      __syncthreads();
      continue;
    }
    const int g_lo = (int)((long long)pr.n_groups * rank / c), g_hi = (int)((long long)pr.n_groups * (rank + 1) / c);
    const int r_lo = g_lo * kGroupRows, r_hi = min(g_hi * kGroupRows, pr.n_pad);
    unsigned long long round = 0;
    int it = 0;
    bool converged = false;
    unsigned next_epoch = 0u;
    if (FRONTIER && pr.rb <= 32) {  // phases 1 and 2 under the frontier schedule
      bool ok = false;
      switch (pr.rb) {
        case 2: ok = frontier_job<2>(a, pr, job.program, j, rank, c, r_lo, r_hi, round, &it, &converged, s_push, &next_epoch); break;
        case 4: ok = frontier_job<4>(a, pr, job.program, j, rank, c, r_lo, r_hi, round, &it, &converged, s_push, &next_epoch); break;
        case 8: ok = frontier_job<8>(a, pr, job.program, j, rank, c, r_lo, r_hi, round, &it, &converged, s_push, &next_epoch); break;
        case 16: ok = frontier_job<16>(a, pr, job.program, j, rank, c, r_lo, r_hi, round, &it, &converged, s_push, &next_epoch); break;
        default: ok = frontier_job<32>(a, pr, job.program, j, rank, c, r_lo, r_hi, round, &it, &converged, s_push, &next_epoch); break;
      }
      if (!ok) return;
    } else {
    // ---- 1. M_0 (Def. 8) of this block's rows: all 2^k guesses as columns
    {
      unsigned char* x0 = a.X0 + pr.state0;
      const int nw = pr.rb >= 8 ? pr.rb / 8 : 1;
      for (int r = r_lo + threadIdx.x; r < r_hi; r += blockDim.x) {
        const int tag = __ldg(a.row_tag + pr.row0 + r);
        if (pr.rb == 2) reinterpret_cast<uint16_t*>(x0)[r] = (uint16_t)batch_m0(tag, 0);
        else if (pr.rb == 4) reinterpret_cast<uint32_t*>(x0)[r] = (uint32_t)batch_m0(tag, 0);
        else
          for (int w = 0; w < nw; w++) reinterpret_cast<uint64_t*>(x0)[(long long)r * nw + w] = batch_m0(tag, w);
      }
    }
    bool dummy;
    if (c > 1) {
      if (!job_barrier_or(a, j, rank, c, ++round, false, &dummy)) return;
    } else {
      __syncthreads();
    }

    // ---- 2. M_{t+1} = theta(M_P M_t) until no row of the program changes
    for (; it < a.max_iters; ++it) {
      const unsigned char* src = ((it & 1) ? a.X1 : a.X0) + pr.state0;
      unsigned char* dst = ((it & 1) ? a.X0 : a.X1) + pr.state0;
      if (threadIdx.x == 0) s_next = g_lo;
      __syncthreads();
      bool changed = false;
      int g = 0;
      if (lane == 0) g = atomicAdd(&s_next, 1);
      g = __shfl_sync(FULL, g, 0);
      while (g < g_hi) {  // uniform in the warp
        const int gg = pr.g0 + g;
        const int4 h0 = __ldg(a.hdr + 3 * gg), h1 = __ldg(a.hdr + 3 * gg + 1), h2 = __ldg(a.hdr + 3 * gg + 2);
        bool ch;
        switch (pr.rb) {
          case 2: ch = group_narrow<2>(a, h0, h1, h2, src, dst, g, pr.n_pad, lane); break;
          case 4: ch = group_narrow<4>(a, h0, h1, h2, src, dst, g, pr.n_pad, lane); break;
          case 8: ch = group_narrow<8>(a, h0, h1, h2, src, dst, g, pr.n_pad, lane); break;
          case 16: ch = group_narrow<16>(a, h0, h1, h2, src, dst, g, pr.n_pad, lane); break;
          case 32: ch = group_narrow<32>(a, h0, h1, h2, src, dst, g, pr.n_pad, lane); break;
          default:
            ch = group_wide(a, h0, h1, h2, reinterpret_cast<const uint64_t*>(src), reinterpret_cast<uint64_t*>(dst), g,
                            pr.rb / 8, pr.n_pad, lane);
        }
        changed |= ch;
        if (lane == 0) g = atomicAdd(&s_next, 1);
        g = __shfl_sync(FULL, g, 0);
      }
      bool any;
      if (c > 1) {
        if (!job_barrier_or(a, j, rank, c, ++round, changed, &any)) return;
      } else {
        any = __syncthreads_or(changed) != 0;
      }
      if (!any) {
        converged = true;
        ++it;
        break;
      }
    }
    }  // full sweep

    // ---- the F pass: F = column 0 (the all-zero guess) of each row of this block's range
    if (a.f_pass) {
      const unsigned char* fin = a.X0 + pr.state0;
      for (int w32 = r_lo / 32 + (threadIdx.x >> 5); w32 < r_hi / 32; w32 += blockDim.x >> 5) {
        const int r = 32 * w32 + lane;
        const unsigned word = __ballot_sync(FULL, fin[(long long)pr.rb * r] & 1u);
        if (lane == 0) a.fbits[(pr.row0 >> 5) + w32] = word;
      }
    }
    // ---- 3. Algorithm 3 (rank 0): stable word = AND over the negated atoms q of (word of q)
    // XOR (word of q-bar); both buffers hold the fixpoint
    if (rank == 0) {
      if (threadIdx.x == 0) {
        if (!a.f_pass) a.iters[job.program] = converged ? it : 0;
        if (!converged) atomicCAS(&a.ctl->status, 0, LP_ERR_NO_FIXPOINT);
      }
      const int nw = a.f_pass ? 0 : (pr.rb >= 8 ? pr.rb / 8 : 1);
      const unsigned char* fin = a.X0 + pr.state0;
      for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        const long long first = 64ll * w, ng = 1ll << pr.k;
        uint64_t st = ng - first >= 64 ? ~0ull : ((1ull << (ng - first)) - 1ull);
        for (int q = 0; q < pr.n_neg; q++) {
          const int r = __ldg(a.neg_row + pr.neg0 + q), rb = __ldg(a.bar_row + pr.neg0 + q);
          uint64_t vq, vb;
          if (pr.rb == 2) {
            vq = reinterpret_cast<const uint16_t*>(fin)[r];
            vb = reinterpret_cast<const uint16_t*>(fin)[rb];
          } else if (pr.rb == 4) {
            vq = reinterpret_cast<const uint32_t*>(fin)[r];
            vb = reinterpret_cast<const uint32_t*>(fin)[rb];
          } else {
            vq = reinterpret_cast<const uint64_t*>(fin)[(long long)r * nw + w];
            vb = reinterpret_cast<const uint64_t*>(fin)[(long long)rb * nw + w];
          }
          st &= vq ^ vb;
        }
        if (!converged) st = 0;
        a.stable_mask[pr.mask0 + w] = st;
        if (st) atomicAdd(reinterpret_cast<unsigned long long*>(a.n_stable + job.program), (unsigned long long)__popcll(st));
      }
    }
    if (FRONTIER && pr.rb <= 32) {
      // the rest state again, once Algorithm 3 has read the fixpoint; no wait follows, so every
      // block of the job finishes its share once it passes this barrier
      if (c > 1) {
        bool dummy2;
        if (!job_barrier_or(a, j, rank, c, ++round, false, &dummy2)) return;
      } else {
        __syncthreads();
      }
      switch (pr.rb) {
        case 2: frontier_reset<2>(a, pr, rank, c, r_lo, r_hi); break;
        case 4: frontier_reset<4>(a, pr, rank, c, r_lo, r_hi); break;
        case 8: frontier_reset<8>(a, pr, rank, c, r_lo, r_hi); break;
        case 16: frontier_reset<16>(a, pr, rank, c, r_lo, r_hi); break;
        default: frontier_reset<32>(a, pr, rank, c, r_lo, r_hi); break;
      }
      if (rank == 0 && threadIdx.x == 0) {
        a.epoch[job.program] = next_epoch;
        a.clean[job.program] = a.f_pass && !converged ? 0u : 1u;  // an unfinished F pass leaves no F
      }
    }
    __syncthreads();  // s_slot and s_next are reused by the next job
  }
}

}  // namespace lp

using namespace lp;

struct lp_batch {
  int device = 0, sm_count = 0;
  int32_t n_programs = 0;
  int32_t n_jobs = 0, n_slots = 0, grid = 0;  // the launch: jobs, their block slots, resident blocks
  std::vector<lp_info> infos;           // per program
  std::vector<BatchProgram> table;      // host copy
  int64_t total_rows = 0, total_nnz = 0, total_state = 0, total_mask_words = 0, total_entries = 0;
  BatchProgram* d_table = nullptr;
  int4* d_hdr = nullptr;
  int32_t* d_col = nullptr;
  int32_t* d_tag = nullptr;
  int32_t* d_neg = nullptr;
  int32_t* d_bar = nullptr;
  unsigned char* d_x0 = nullptr;
  unsigned char* d_x1 = nullptr;
  int64_t* d_nstable = nullptr;
  int32_t* d_iters = nullptr;
  BatchJob* d_jobs = nullptr;
  int32_t* d_slot_job = nullptr;
  unsigned long long* d_job_bar = nullptr;  // 4 per job, then the queue counter
  DeviceCtl* d_ctl = nullptr;
  uint64_t* d_stage = nullptr;  // staging for a host stable_mask
  bool frontier = false;         // frontier schedule for the programs with rows of <= 32 bytes
  int block = 512;               // threads per block of the launch
  int32_t* d_tptr = nullptr;     // frontier: transposed row pointers (global offsets into d_tidx)
  int32_t* d_tidx = nullptr;
  int32_t* d_seed = nullptr;
  unsigned* d_mark = nullptr;
  int32_t* d_list = nullptr;     // 2 x total_rows
  unsigned* d_fcnt = nullptr;    // 3 per program
  unsigned* d_dirty = nullptr;   // a bit per row
  unsigned* d_clean = nullptr;   // per program: rest state valid (zeroed at compile)
  unsigned* d_epoch = nullptr;   // per program: next unused stamp
  int64_t device_bytes = 0;
  double compile_ms = 0;
  int64_t launches = 0;
  bool from_f = false;           // frontier programs start from F (unless LP_BATCH_FROM_M0)
  bool f_ready = false;          // F has been computed (the F pass ran to its end)
  unsigned* d_fbits = nullptr;   // F: a bit per row
};

namespace {

const void* batch_entry(bool frontier) {
  return frontier ? (const void*)batch_stable_kernel<kBatchFrontierBlock, true>
                  : (const void*)batch_stable_kernel<kBatchBlock, false>;
}

lp_status bfail(lp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

void batch_release(lp_batch* b) {
  void* ptrs[] = {b->d_table, b->d_hdr, b->d_col, b->d_tag, b->d_neg,     b->d_bar, b->d_x0,
                  b->d_x1,    b->d_nstable, b->d_iters, b->d_jobs, b->d_slot_job, b->d_job_bar, b->d_ctl, b->d_stage,
                  b->d_tptr,  b->d_tidx, b->d_seed, b->d_mark, b->d_list, b->d_fcnt, b->d_dirty, b->d_clean,
                  b->d_epoch, b->d_fbits};
  device_free_all(ptrs, sizeof(ptrs) / sizeof(ptrs[0]));
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

// One program's sliced layout (the layout of the least-model kernel 2, built on the host here):
// rows renumbered by length within windows of 1024, 128-row groups padded to their longest row,
// entries column-major so that lane l of a warp reads the k-th entries of rows l, 32 + l,
// 64 + l, 96 + l as one int4; a shorter row repeats its first entry, an empty row is masked.
struct ProgSlices {
  std::vector<int4> hdr;     // 3 per group: {first entry (program-local), width, 0, 0}, OR masks, empty masks
  std::vector<int32_t> ent;  // entries, columns in the new numbering
  std::vector<int32_t> tag;  // Def. 8 initial-column tag per row, new numbering
  std::vector<int32_t> neg, bar;
  // frontier schedule: per row (new numbering) the rows that refer to it, and the rows nonzero in
  // M_0 (fact rows, guessed rows)
  std::vector<int32_t> tptr, tidx, seed;
};

void build_slices(const HostMatrix& hm, ProgSlices& out, bool frontier) {
  constexpr int kWin = 1024;
  const int32_t np = hm.n_pad;
  std::vector<int32_t> q((size_t)np), qinv((size_t)np);
  std::vector<std::pair<int32_t, int32_t>> key;
  for (int32_t lo = 0; lo < np; lo += kWin) {
    const int32_t hi = std::min(np, lo + kWin);
    key.clear();
    for (int32_t r = lo; r < hi; r++) key.emplace_back(hm.row_ptr[r + 1] - hm.row_ptr[r], r);
    std::stable_sort(key.begin(), key.end(), [](const std::pair<int32_t, int32_t>& x, const std::pair<int32_t, int32_t>& y) {
      return x.first < y.first;
    });
    for (int32_t i = 0; i < hi - lo; i++) {
      qinv[lo + i] = key[i].second;
      q[key[i].second] = lo + i;
    }
  }
  const int32_t ng = (np + kGroupRows - 1) / kGroupRows;
  out.hdr.assign(3 * (size_t)ng, make_int4(0, 0, 0, 0));
  int64_t off = 0;
  std::vector<int32_t> K((size_t)ng, 0);
  for (int32_t g = 0; g < ng; g++) {
    int32_t k = 0;
    uint32_t orm[4] = {0, 0, 0, 0}, emm[4] = {0, 0, 0, 0};
    for (int t = 0; t < kGroupRows; t++) {
      const int32_t row = g * kGroupRows + t;
      int32_t len = 0;
      bool anyb = false;
      if (row < np) {
        const int32_t r = qinv[row];
        len = hm.row_ptr[r + 1] - hm.row_ptr[r];
        anyb = (hm.any_mask[r >> 5] >> (r & 31)) & 1u;
      }
      k = std::max(k, len);
      if (anyb) orm[t >> 5] |= 1u << (t & 31);
      if (len == 0) emm[t >> 5] |= 1u << (t & 31);
    }
    K[g] = k;
    out.hdr[3 * (size_t)g] = make_int4((int)off, k, 0, 0);
    out.hdr[3 * (size_t)g + 1] = make_int4((int)orm[0], (int)orm[1], (int)orm[2], (int)orm[3]);
    out.hdr[3 * (size_t)g + 2] = make_int4((int)emm[0], (int)emm[1], (int)emm[2], (int)emm[3]);
    off += (int64_t)kGroupRows * k;
  }
  out.ent.assign((size_t)off, 0);
  for (int32_t g = 0; g < ng; g++) {
    const int64_t base = out.hdr[3 * (size_t)g].x;
    for (int t = 0; t < kGroupRows; t++) {
      const int32_t row = g * kGroupRows + t;
      if (row >= np) continue;
      const int32_t r = qinv[row];
      const int32_t b = hm.row_ptr[r], len = hm.row_ptr[r + 1] - b;
      const int32_t first = len > 0 ? q[hm.col[b]] : 0;
      const int u = t >> 5, l = t & 31;
      for (int32_t k = 0; k < K[g]; k++) out.ent[base + 4 * (32 * k + l) + u] = k < len ? q[hm.col[b + k]] : first;
    }
  }
  out.tag.assign((size_t)np, -1);
  for (int32_t r = 0; r < np; r++) out.tag[q[r]] = hm.row_tag[r];
  out.neg.resize(hm.neg_row.size());
  out.bar.resize(hm.bar_row.size());
  for (size_t j = 0; j < hm.neg_row.size(); j++) {
    out.neg[j] = q[hm.neg_row[j]];
    out.bar[j] = q[hm.bar_row[j]];
  }
  if (!frontier) return;
  out.tptr.assign((size_t)np + 1, 0);
  for (int32_t r = 0; r < np; r++)
    for (int32_t e = hm.row_ptr[r]; e < hm.row_ptr[r + 1]; e++) out.tptr[q[hm.col[e]] + 1]++;
  for (int32_t j = 0; j < np; j++) out.tptr[j + 1] += out.tptr[j];
  out.tidx.assign((size_t)out.tptr[np], 0);
  std::vector<int32_t> cur(out.tptr.begin(), out.tptr.end() - 1);
  for (int32_t r = 0; r < np; r++)
    for (int32_t e = hm.row_ptr[r]; e < hm.row_ptr[r + 1]; e++) out.tidx[cur[q[hm.col[e]]]++] = q[r];
  out.seed.clear();
  for (int32_t j = 0; j < np; j++)
    if (out.tag[j] == -2 || out.tag[j] >= 0) out.seed.push_back(j);
}

}  // namespace

extern "C" {

lp_status lp_compile_batch(int32_t n_programs, const int32_t* n_atoms, const int64_t* rule_off, const int32_t* head,
                           const int64_t* body_off, const int32_t* body_atom, const uint8_t* body_neg, uint32_t flags,
                           void* cuda_stream, lp_batch** out) {
  NvtxRange nvtx("lp_compile_batch");
  if (!out) return bfail(LP_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  if (flags & ~(LP_BATCH_FULL_SWEEP | LP_BATCH_FROM_M0)) return bfail(LP_ERR_INVALID, "unknown flags");
  const bool frontier = !(flags & LP_BATCH_FULL_SWEEP);
  if (n_programs < 0 || (n_programs > 0 && (!n_atoms || !rule_off))) return bfail(LP_ERR_INVALID, "bad program list");
  if (n_programs > 0 && rule_off[0] != 0) return bfail(LP_ERR_INVALID, "rule_off[0] must be 0");
  for (int32_t p = 0; p < n_programs; p++)
    if (rule_off[p + 1] < rule_off[p]) return bfail(LP_ERR_INVALID, "rule_off decreases");
  auto t0 = std::chrono::steady_clock::now();
  std::vector<HostMatrix> hms(n_programs);
  std::vector<ProgSlices> sl(n_programs);
  std::vector<std::string> errs(n_programs);
  std::vector<int> rcs(n_programs, LP_OK);
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t p = 0; p < n_programs; p++) {
    const int64_t r0 = rule_off[p], nr = rule_off[p + 1] - r0;
    std::vector<int64_t> off((size_t)nr + 1);
    for (int64_t r = 0; r <= nr; r++) off[r] = body_off[r0 + r] - body_off[r0];
    const int64_t b0 = body_off[r0];
    try {
      rcs[p] = compile_host(n_atoms[p], nr, head + r0, off.data(), body_atom ? body_atom + b0 : nullptr,
                            body_neg ? body_neg + b0 : nullptr, hms[p], errs[p]);
      if (rcs[p] == LP_OK && hms[p].k <= 16) build_slices(hms[p], sl[p], frontier);
    } catch (const std::bad_alloc&) {
      rcs[p] = LP_ERR_OOM;
      errs[p] = "host allocation failed";
    }
  }
  for (int32_t p = 0; p < n_programs; p++)
    if (rcs[p] != LP_OK) return bfail((lp_status)rcs[p], "program " + std::to_string(p) + ": " + errs[p]);
  lp_batch* b = new (std::nothrow) lp_batch();
  if (!b) return bfail(LP_ERR_OOM, "host allocation failed");
  b->n_programs = n_programs;
  b->frontier = frontier;
  b->from_f = frontier && !(flags & LP_BATCH_FROM_M0);
  b->infos.resize(n_programs);
  b->table.resize(n_programs);
  int64_t row = 0, state = 0, mask = 0, nnz = 0, neg = 0, ent = 0, groups = 0, tp = 0, ti = 0, seeds = 0;
  for (int32_t p = 0; p < n_programs; p++) {
    const HostMatrix& hm = hms[p];
    if (hm.k > 16) {
      delete b;
      return bfail(LP_ERR_TOO_MANY_GUESSES, "program " + std::to_string(p) + ": k > 16 guessed atoms");
    }
    BatchProgram& t = b->table[p];
    t.row0 = row;
    t.n_pad = hm.n_pad;
    t.rb = std::max(2, (1 << hm.k) / 8);
    t.k = hm.k;
    t.state0 = state;
    t.mask0 = mask;
    t.n_neg = (int32_t)hm.neg_row.size();
    t.neg0 = neg;
    t.g0 = (int32_t)groups;
    t.n_groups = (int32_t)(sl[p].hdr.size() / 3);
    t.tp0 = tp;
    t.seed0 = seeds;
    t.n_seed = (int32_t)sl[p].seed.size();
    tp += (int64_t)sl[p].tptr.size();
    ti += (int64_t)sl[p].tidx.size();
    seeds += (int64_t)sl[p].seed.size();
    row += hm.n_pad;
    state += (int64_t)hm.n_pad * t.rb;
    mask += t.rb >= 8 ? t.rb / 8 : 1;
    nnz += hm.nnz;
    neg += t.n_neg;
    ent += (int64_t)sl[p].ent.size();
    groups += t.n_groups;
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
  b->total_entries = ent;
  if (row >= (int64_t(1) << 31) - 64 || ent >= (int64_t(1) << 31) - 64 || groups >= (int64_t(1) << 29) ||
      ti >= (int64_t(1) << 31) - 64) {
    delete b;
    return bfail(LP_ERR_INVALID, "batch too large (rows and stored entries must be < 2^31)");
  }
  // concatenation: group headers with global entry offsets, entries, row tags, negated pairs
  std::vector<int4> hdr(3 * (size_t)std::max<int64_t>(groups, 1));
  std::vector<int32_t> cl((size_t)std::max<int64_t>(ent, 1)), tag((size_t)std::max<int64_t>(row, 1)),
      ng((size_t)std::max<int64_t>(neg, 1)), br((size_t)std::max<int64_t>(neg, 1));
  {
    int64_t e0 = 0;
    for (int32_t p = 0; p < n_programs; p++) {
      const BatchProgram& t = b->table[p];
      const ProgSlices& ps = sl[p];
      for (int32_t g = 0; g < t.n_groups; g++) {
        int4 h = ps.hdr[3 * (size_t)g];
        h.x = (int)(h.x + e0);
        hdr[3 * ((size_t)t.g0 + g)] = h;
        hdr[3 * ((size_t)t.g0 + g) + 1] = ps.hdr[3 * (size_t)g + 1];
        hdr[3 * ((size_t)t.g0 + g) + 2] = ps.hdr[3 * (size_t)g + 2];
      }
      std::copy(ps.ent.begin(), ps.ent.end(), cl.begin() + e0);
      std::copy(ps.tag.begin(), ps.tag.end(), tag.begin() + t.row0);
      std::copy(ps.neg.begin(), ps.neg.end(), ng.begin() + t.neg0);
      std::copy(ps.bar.begin(), ps.bar.end(), br.begin() + t.neg0);
      e0 += (int64_t)ps.ent.size();
    }
  }
  // frontier: transposed matrices (row pointers made global), seed rows
  std::vector<int32_t> tptr((size_t)std::max<int64_t>(tp, 1)), tidx((size_t)std::max<int64_t>(ti, 1)),
      seed((size_t)std::max<int64_t>(seeds, 1));
  if (frontier) {
    int64_t i0 = 0;
    for (int32_t p = 0; p < n_programs; p++) {
      const BatchProgram& t = b->table[p];
      const ProgSlices& ps = sl[p];
      for (size_t x = 0; x < ps.tptr.size(); x++) tptr[t.tp0 + x] = (int32_t)(ps.tptr[x] + i0);
      std::copy(ps.tidx.begin(), ps.tidx.end(), tidx.begin() + i0);
      std::copy(ps.seed.begin(), ps.seed.end(), seed.begin() + t.seed0);
      i0 += (int64_t)ps.tidx.size();
    }
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  lp_status st = e == cudaSuccess ? LP_OK : bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (st == LP_OK) st = bupload(b, &b->d_table, b->table.data(), b->table.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_hdr, hdr.data(), 3 * (size_t)groups, s);
  if (st == LP_OK) st = bupload(b, &b->d_col, cl.data(), (size_t)ent, s);
  if (st == LP_OK) st = bupload(b, &b->d_tag, tag.data(), (size_t)row, s);
  if (st == LP_OK) st = bupload(b, &b->d_neg, ng.data(), (size_t)neg, s);
  if (st == LP_OK) st = bupload(b, &b->d_bar, br.data(), (size_t)neg, s);
  if (st == LP_OK) st = bupload<unsigned char>(b, &b->d_x0, nullptr, (size_t)state, s);
  if (st == LP_OK) st = bupload<unsigned char>(b, &b->d_x1, nullptr, (size_t)state, s);
  if (st == LP_OK) st = bupload<int64_t>(b, &b->d_nstable, nullptr, (size_t)n_programs, s);
  if (st == LP_OK) st = bupload<int32_t>(b, &b->d_iters, nullptr, (size_t)n_programs, s);
  if (frontier) {
    if (st == LP_OK) st = bupload(b, &b->d_tptr, tptr.data(), (size_t)tp, s);
    if (st == LP_OK) st = bupload(b, &b->d_tidx, tidx.data(), (size_t)ti, s);
    if (st == LP_OK) st = bupload(b, &b->d_seed, seed.data(), (size_t)seeds, s);
    if (st == LP_OK) st = bupload<unsigned>(b, &b->d_mark, nullptr, (size_t)row, s);
    if (st == LP_OK) st = bupload<int32_t>(b, &b->d_list, nullptr, 2 * (size_t)row, s);
    if (st == LP_OK) st = bupload<unsigned>(b, &b->d_fcnt, nullptr, 3 * (size_t)n_programs, s);
    if (st == LP_OK) st = bupload<unsigned>(b, &b->d_dirty, nullptr, (size_t)row / 32 + 1, s);
    if (st == LP_OK) st = bupload<unsigned>(b, &b->d_clean, nullptr, (size_t)n_programs, s);
    if (st == LP_OK) st = bupload<unsigned>(b, &b->d_epoch, nullptr, (size_t)n_programs, s);
    if (st == LP_OK && (e = cudaMemsetAsync(b->d_clean, 0, std::max<size_t>(n_programs, 1) * 4, s)) != cudaSuccess)
      st = bfail(LP_ERR_CUDA, cudaGetErrorString(e));
    if (st == LP_OK && b->from_f) st = bupload<unsigned>(b, &b->d_fbits, nullptr, (size_t)row / 32 + 1, s);
  }
  // Jobs: one per program, largest first. A program whose share of the work exceeds one block's
  // share of the whole batch runs on several co-resident blocks (at most 16, and all multi-block
  // jobs together on at most half of the grid, so that every one of them is fully staffed by
  // the first blocks to start); the others run on one block each.
  int per_sm = 0;
  b->block = frontier ? kBatchFrontierBlock : kBatchBlock;
  if (st == LP_OK && (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_entry(frontier), b->block, 0)) !=
                         cudaSuccess)
    st = bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if (st == LP_OK && n_programs > 0 && per_sm < 1) st = bfail(LP_ERR_CUDA, "batch kernel cannot be resident");
  std::vector<BatchJob> jobs;
  std::vector<int32_t> slot_job;
  if (st == LP_OK) {
    b->grid = std::max(1, per_sm * b->sm_count);
    std::vector<double> work((size_t)n_programs);
    double total_work = 0;
    for (int32_t p = 0; p < n_programs; p++) {
      const BatchProgram& t = b->table[p];
      work[p] = 4.0 * (double)sl[p].ent.size() + 3.0 * (double)t.n_pad * t.rb + 48.0 * t.n_groups;
      total_work += work[p];
    }
    std::vector<int32_t> order((size_t)n_programs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return work[x] > work[y]; });
    const double share = total_work / b->grid;
    const int multi_cap = std::max(1, b->grid / 2);
    int multi = 0;
    for (int32_t p : order) {
      int c = 1;
      // a frontier program evaluates a small share of its rows: at most two blocks
      const bool fr_prog = frontier && b->table[p].rb <= 32;
      if (share > 0 && work[p] > share) c = (int)std::min<double>(fr_prog ? 2.0 : 16.0, std::ceil(work[p] / share));
      c = std::min(c, std::max(1, b->table[p].n_groups));
      if (c > 1 && multi + c > multi_cap) c = 1;
      if (c > 1) multi += c;
      BatchJob jb{p, c, (int32_t)slot_job.size(), 0};
      jobs.push_back(jb);
      for (int r = 0; r < c; r++) slot_job.push_back((int32_t)jobs.size() - 1);
    }
    b->n_jobs = (int32_t)jobs.size();
    b->n_slots = (int32_t)slot_job.size();
  }
  if (st == LP_OK) st = bupload(b, &b->d_jobs, jobs.data(), jobs.size(), s);
  if (st == LP_OK) st = bupload(b, &b->d_slot_job, slot_job.data(), slot_job.size(), s);
  if (st == LP_OK) st = bupload<unsigned long long>(b, &b->d_job_bar, nullptr, 4 * (size_t)b->n_jobs + 1, s);
  if (st == LP_OK) st = bupload<DeviceCtl>(b, &b->d_ctl, nullptr, 1, s);
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

lp_status lp_batch_last_stats(const lp_batch* b, int64_t* rows_evaluated, int64_t* entries_evaluated,
                              int64_t* bytes_touched, void* cuda_stream) {
  if (!b) return bfail(LP_ERR_INVALID, "NULL batch");
  DeviceCtl ctl;
  std::memset(&ctl, 0, sizeof(ctl));
  if (b->n_programs > 0) {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemcpyAsync(&ctl, b->d_ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rows_evaluated) *rows_evaluated = (int64_t)ctl.fr_rows;
  if (entries_evaluated) *entries_evaluated = (int64_t)ctl.fr_entries;
  if (bytes_touched) *bytes_touched = (int64_t)ctl.fr_list;
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
  cudaError_t e = cudaSuccess;
  // one launch over all jobs; the F pass (from F, before the first solve) computes F
  auto launch = [&](bool f_pass) -> lp_status {
    e = cudaMemsetAsync(b->d_ctl, 0, sizeof(DeviceCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_job_bar, 0, (4 * (size_t)b->n_jobs + 1) * 8, s);
    if (!f_pass) {
      if (e == cudaSuccess) e = cudaMemsetAsync(b->d_nstable, 0, std::max<size_t>(b->n_programs, 1) * 8, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(b->d_iters, 0, std::max<size_t>(b->n_programs, 1) * 4, s);
    }
    if (e != cudaSuccess) return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
    if (b->n_programs == 0) return LP_OK;
    BatchArgs a{};
    a.progs = b->d_table;
    a.jobs = b->d_jobs;
    a.slot_job = b->d_slot_job;
    a.n_slots = b->n_slots;
    a.hdr = b->d_hdr;
    a.col = b->d_col;
    a.row_tag = b->d_tag;
    a.neg_row = b->d_neg;
    a.bar_row = b->d_bar;
    a.X0 = b->d_x0;
    a.X1 = b->d_x1;
    a.stable_mask = d_mask;
    a.n_stable = reinterpret_cast<long long*>(b->d_nstable);
    a.iters = b->d_iters;
    a.job_bar = b->d_job_bar;
    a.queue = reinterpret_cast<unsigned*>(b->d_job_bar + 4 * (size_t)b->n_jobs);
    a.ctl = b->d_ctl;
    // from the fact rows every iteration adds a row, so the F pass always ends
    a.max_iters = f_pass ? (1 << 30) : max_iters;
    a.frontier = b->frontier;
    a.tptr = b->d_tptr;
    a.tidx = b->d_tidx;
    a.seed = b->d_seed;
    a.mark = b->d_mark;
    a.list = b->d_list;
    a.fcnt = b->d_fcnt;
    a.total_rows = b->total_rows;
    a.dirty = b->d_dirty;
    a.clean = b->d_clean;
    a.epoch = b->d_epoch;
    a.from_f = b->from_f;
    a.f_pass = f_pass;
    a.fbits = b->d_fbits;
    // every block resident (multi-block jobs meet at their own barriers); no more blocks than slots
    const int grid = std::max(1, std::min(b->grid, b->n_slots));
    void* params[] = {&a};
    e = cudaLaunchCooperativeKernel(batch_entry(b->frontier), dim3(grid), dim3(b->block), params, 0, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(LP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    b->launches++;
    count_launches(1);
    return LP_OK;
  };
  lp_status lst;
  if (b->from_f && !b->f_ready && b->n_programs > 0) {
    if ((lst = launch(true)) != LP_OK) return lst;
    DeviceCtl fctl;
    std::memset(&fctl, 0, sizeof(fctl));
    if ((e = cudaMemcpyAsync(&fctl, b->d_ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
    if (fctl.status != 0) return bfail((lp_status)fctl.status, "the fixpoint from the fact rows did not finish");
    b->f_ready = true;
  }
  if ((lst = launch(false)) != LP_OK) return lst;
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
  DeviceCtl ctl;
  std::memset(&ctl, 0, sizeof(ctl));
  if (b->n_programs && (e = cudaMemcpyAsync(&ctl, b->d_ctl, sizeof(DeviceCtl), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bfail(LP_ERR_CUDA, cudaGetErrorString(e));
  status = ctl.status;
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

// kernels.h -- launch interfaces of liblp's kernels (host side).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lp {

struct DeviceCtl;

// Sets a kernel's dynamic shared-memory limit and L1 / shared carveout preference on the current
// device only when they differ from the last values set there: the attribute call costs far more
// host time than a launch, and it would sit inside every solve's timed window.
cudaError_t set_kernel_smem(const void* kernel, int dyn_bytes, int carveout);

// Algorithm 1 on one bit-packed vector (persistent cooperative kernel).
struct FixArgs {
  const int32_t* row_ptr;   // n_pad + 1, internal order
  const int32_t* col;       // nnz, internal column ids
  const uint32_t* any_mask; // n_pad / 32: OR-rule rows
  uint32_t* x0;             // n_pad / 32 words: initial vector / even iterates
  uint32_t* x1;             // n_pad / 32 words: odd iterates
  int32_t n_words;          // n_pad / 32
  int32_t max_iters;
  DeviceCtl* ctl;
  // initial vector, default mode (x0 zeroed by the caller): facts of the selected atoms
  const uint64_t* init;        // ceil(n/64) words or NULL (= every fact)
  const int32_t* fact_row;     // internal rows of the fact rows
  const int32_t* fact_owner;   // their original atoms
  int32_t n_facts;
  const uint64_t* fact_mask;   // ceil(n/64): atoms that have a fact rule
  int32_t n_atom_words;        // ceil(n/64)
  // initial vector, LP_ROWS mode: canonical rows
  const uint64_t* rows_init;   // ceil(n'/64) words or NULL (default mode)
  const int32_t* inv;          // internal row -> canonical row (LP_ROWS only)
  int32_t n_prime;
  // output: bit a of out = final bit of internal row perm[a], a < n_out
  uint64_t* out;
  const int32_t* perm;         // canonical -> internal
  int32_t n_out;
  int32_t n_sec_a;             // leading rows that rule rows refer to (used by the streamed kernel)
};

// Threads per block of the least-model kernel: 512 for row map 0 (40 registers, 3 blocks per
// SM), 1024 for the thread-per-row maps (up to 64 registers, one block per SM, so half as many
// blocks meet at each grid barrier as with two 512-thread blocks).
constexpr int kFixBlockMap0 = 512, kFixBlockRows = 1024;
inline int fix_block(int row_map) { return row_map == 0 ? kFixBlockMap0 : kFixBlockRows; }
// row_map 0 (a warp per 32-row word, entries in 32-entry chunks): row_split = warps per word
// (1, 2, 4 or 8), chunk_batch = chunks whose loads a warp issues together (1 or 4). row_map 1,
// 2, 3 (a thread per row: two words per warp step with 8 column ids per pass, four words, or
// loads pipelined over the warp's words with 5 ids staged per row) take row_split =
// chunk_batch = 1.
cudaError_t launch_fixpoint(const FixArgs& a, int grid, int row_split, int chunk_batch, int row_map, cudaStream_t s);
int fixpoint_blocks_per_sm(int row_split, int chunk_batch, int row_map);

// The same loop with the matrix streamed through shared memory (fixpoint_stream.cu).
struct StreamLayout {
  const uint32_t* desc;     // n_pad row descriptors
  const int32_t* word_hdr;  // 2 * (n_pad / 32 + 1)
  const int32_t* and_col;   // rule-row entries (+ padding)
  const int32_t* groups;    // kGroupInts per group (device)
  int32_t n_groups;
  int32_t n_sec_a;          // leading rows that rule rows refer to (staged in shared memory)
  const int32_t* host_groups;  // the same group records on the host (launch geometry)
};
cudaError_t launch_fixpoint_stream(const FixArgs& a, const StreamLayout& layout, int grid, cudaStream_t s);
int fixpoint_stream_blocks_per_sm();

// The same loop on a sliced layout of M_P (fixpoint_sliced.cu): rows renumbered by (gather
// class, length) within windows, 32-row slices stored column-major at the slice's width.
struct SlicedLayout {
  const int4* hdr;          // 3 per 128-row group: {first entry, width | staged flag}, OR masks, empty masks
  const int32_t* col;       // entries, renumbered columns
  const int32_t* q;         // internal row -> new row
  const int32_t* fact_row;  // fact rows, renumbered
  const int32_t* perm;      // canonical row -> new row (n' entries)
  int32_t n_groups;         // ceil(n_pad / 128)
  int64_t total_entries;    // stored entries (the groups' offsets end there)
  int32_t n_stage_words;    // vector words staged in shared memory (covers the leading n_sec_a rows)
};
constexpr int kSlicedBlock = 1024;
int sliced_windows(int32_t n_sec_a, int32_t n_pad);
int sliced_groups(int32_t n_pad);
// Build from the device CSR. Pass 1: renumbering q / qinv, group headers (3 int4 per group), and
// *total_dev = entries to store (cnt: sliced_groups ints of scratch). Pass 2 (after scol of *total_dev ints is allocated):
// the entries, and the fact rows and output permutation renumbered.
cudaError_t build_sliced_pass1(const int32_t* row_ptr, const int32_t* col, const uint32_t* any_mask, int32_t n_sec_a,
                               int32_t n_pad, int32_t* q, int32_t* qinv, int4* hdr, int32_t* cnt, long long* total_dev,
                               cudaStream_t s);
cudaError_t build_sliced_pass2(const int32_t* row_ptr, const int32_t* col, const int32_t* q, const int32_t* qinv,
                               const int4* hdr, int32_t n_pad, int32_t* scol, const int32_t* fact_row, int32_t n_facts,
                               int32_t* fact_row_out, const int32_t* perm, int32_t n_perm, int32_t* perm_out,
                               cudaStream_t s);
cudaError_t launch_fixpoint_sliced(const FixArgs& a, const SlicedLayout& L, bool stage, int grid, cudaStream_t s);
int fixpoint_sliced_blocks_per_sm(bool stage, int stage_words);

// The same loop in one block with kernel 2's sliced layout and both vectors in shared memory
// (fixpoint_block.cu), for programs whose layout fits: block_kernel_smem_bytes at most the
// device's per-block limit.
constexpr int kBlockThreads = 1024;
long long block_kernel_smem_bytes(int n_words, int n_groups, long long entries);
cudaError_t launch_fixpoint_block(const FixArgs& a, const SlicedLayout& S, cudaStream_t s);

// Algorithms 2 + 3 over tiles of 64-bit guess words (persistent cooperative kernel).
struct StableArgs {
  const int32_t* row_ptr;
  const int32_t* col;
  const uint32_t* any_mask;
  const int32_t* row_tag;   // n_pad: -1 zero, -2 fact, -3 barred atom of a fact, j >= 0 guess bit j
  int32_t n_pad;
  uint64_t* X0;             // n_pad * W words: iterate buffers of one tile
  uint64_t* X1;
  int32_t W;                // guess words per tile (1, 2, 4, 8, 16 or 32)
  int32_t log2W;
  int64_t n_guesses;
  int64_t n_gwords;         // ceil(n_guesses / 64)
  int64_t n_tiles;
  const uint64_t* guesses;  // n_guesses k-bit words, or NULL = all 2^k in order
  int32_t k;
  const int32_t* neg_row;   // per negated atom: internal row of q
  const int32_t* bar_row;   // ... and of q-bar
  int32_t n_barred;
  const int32_t* perm;      // canonical -> internal (first n entries: original atoms)
  int32_t n;
  uint64_t* stable_mask;    // n_gwords words
  uint64_t* models;         // max_models x ceil(n/64) words or NULL
  int64_t max_models;
  int32_t n_atom_words;
  int32_t max_iters;
  DeviceCtl* ctl;
  // frontier schedule (stable_frontier.cu): the transposed matrix, and per wave of fr_tiles
  // tiles (item = tile * n_pad + row; X0 / X1 above then hold fr_tiles tiles each) a stamp per
  // item, two work lists, a changed-item bitmap and each tile's last changing iteration
  const int32_t* t_ptr;     // n_pad + 1: rows referring to column j are t_idx[t_ptr[j] .. t_ptr[j + 1])
  const int32_t* t_idx;     // nnz
  unsigned* mark;           // fr_tiles * n_pad
  int32_t* fr_list;         // 2 x fr_tiles * n_pad
  unsigned* fr_dirty;       // ceil(fr_tiles * n_pad / 32)
  int32_t* fr_last;         // fr_tiles
  unsigned* fr_cnt;         // kFrontierCounters: rest-state record (slots 3 to 7), per iteration the
                            // list sizes and wide-item count (16 to 27, rotating)
  const unsigned* long_mask;  // ceil(n_pad / 32): rows of at least kLongRow entries (a warp evaluates
                              // them); NULL if there are none
  int32_t* fr_wide;         // wide_cap: items whose dependents the whole grid pushes
  int32_t wide_cap;
  int32_t fr_tiles;         // tiles per wave (the buffers' capacity)
  unsigned fr_key;          // nonzero tag of the buffers' layout
  const int32_t* fr_seed;   // n_seed rows the first list starts from: the fact rows, then the
  int32_t n_seed;           // guessed rows (only the guessed rows when starting from fr_F)
  const uint32_t* fr_F;     // ceil(n_pad / 32) or NULL: the guess-independent fixpoint to start from
  const int32_t* guess_rows;  // n_guess_rows: the guessed barred rows (row_tag >= 0)
  int32_t n_guess_rows;
};

constexpr int kStableBlock = 256;
// row_split: one row per warp, its entries split over the warp's 32 / W lane groups
cudaError_t launch_stable(const StableArgs& a, int grid, bool row_split, cudaStream_t s);
int stable_blocks_per_sm(bool row_split);
// Frontier schedule (needs the t_ptr ... wide_cap fields)
cudaError_t launch_stable_frontier(const StableArgs& a, int grid, cudaStream_t s);
int stable_frontier_blocks_per_sm(int W);
// rows with at least this many entries are evaluated by a whole warp under the frontier schedule
constexpr int kLongRow = 64;
// counters of the frontier schedule (StableArgs::fr_cnt)
constexpr int kFrontierCounters = 32;
// mask (ceil(n_pad / 32) words): bit r set iff row r has at least kLongRow entries; *any (zeroed
// by the caller) becomes nonzero if one is
cudaError_t build_long_rows(const int32_t* row_ptr, int32_t n_pad, unsigned* mask, unsigned* any, cudaStream_t s);
// Transposed matrix for the frontier schedule, built on the device: cnt (n_pad + 1 ints of
// scratch, zeroed by the caller) becomes the cursor of the fill.
cudaError_t build_transpose(const int32_t* row_ptr, const int32_t* col, int32_t n_pad, int32_t* t_ptr, int32_t* t_idx,
                            int32_t* cnt, cudaStream_t s);

}  // namespace lp

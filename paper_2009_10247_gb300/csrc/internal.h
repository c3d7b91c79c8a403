// internal.h -- liblp's private types, shared by its host compiler, kernels and C ABI glue.
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/lp.h"

namespace lp {

// Allocator whose argument-less construct() default-initializes: resize() of a vector of plain
// integers leaves the new elements unwritten, so the host compiler sizes its large arrays
// without a serial zero fill and writes them in parallel loops (which also spreads the first
// touch of their pages over the threads).
template <class T>
struct uninit_alloc : std::allocator<T> {
  using value_type = T;
  template <class U>
  struct rebind {
    using other = uninit_alloc<U>;
  };
  uninit_alloc() noexcept = default;
  template <class U>
  uninit_alloc(const uninit_alloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using hvec = std::vector<T, uninit_alloc<T>>;

// Releases a vector's storage.
template <class V>
void free_vec(V& v) {
  V().swap(v);
}

// Canonical row kinds (the values lp_export_matrix reports).
enum RowKind : int8_t { K_EMPTY = 0, K_RULE = 1, K_OR = 2, K_FACT = 3, K_BARRED = 4 };

// Result of the host compile (Sec. 2.1/2.2 standardization + Def. 2/7 matrix), already in the
// internal row order the kernels use. Every "row" is also a column (M_P is square).
struct HostMatrix {
  int32_t n = 0;          // original atoms
  int64_t n_rules = 0;
  int32_t n_prime = 0;    // rows of M_P
  int32_t n_pad = 0;      // rows padded to a multiple of 64 (padding rows are empty)
  int64_t nnz = 0;
  int32_t n_barred = 0, n_aux = 0, k = 0;
  int32_t n_fact_rows = 0, n_rule_rows = 0, n_or_rows = 0;

  hvec<int32_t> row_ptr;    // internal CSR, n_pad + 1
  hvec<int32_t> col;        // internal column ids, nnz
  hvec<uint32_t> any_mask;  // n_pad / 32 words: bit set = OR-rule row (threshold 1)
  hvec<int32_t> perm;       // canonical row -> internal row (n_prime)
  hvec<int8_t> canon_kind;  // canonical row kinds (n_prime)
  hvec<int32_t> canon_rule; // canonical row -> original rule of a rule row, else -1
  hvec<int32_t> fact_row;   // internal rows with a_ii = 1 from a fact (Def. 2 item 3)
  hvec<int32_t> fact_owner; // original atom of each fact row
  std::vector<uint64_t> fact_mask; // ceil(n/64) words: atoms with at least one fact rule
  std::vector<int32_t> neg_row;    // per negated atom q (ascending id): internal row of q
  std::vector<int32_t> bar_row;    // ... and internal row of q-bar
  std::vector<int32_t> guess_row;  // internal rows of the k guessed barred atoms, bit order
  hvec<int32_t> row_tag;    // n_pad: -1 zero, -2 fact, j >= 0 guessed barred atom j,
                                   //        -3 barred atom of a fact (initial column of Def. 8)

  // Streamed layout of the least-model kernel (see fixpoint_stream.cu). Row kinds: 0 = rule
  // row (entries listed in and_col), 1 = OR-rule row (its entries are the next `length` new
  // atoms after those of the OR rows before it, so they are not stored), 2 = self-loop (fact
  // or barred atom: its own bit). Per 32-row word a header {first and_col index of the word,
  // first new atom of the word's OR rows | kLongWord}. In a word whose rows all have at most
  // 32 entries a row's descriptor is kind << 30 | offset << 6 | length, the offset counted
  // from the word's first rule entry (rule rows) or first new atom (OR rows); in a "long"
  // word (header bit kLongWord) it is kind << 30 | length and offsets come from prefix sums.
  // Groups are consecutive word ranges whose headers, descriptors and and_col entries fit
  // one shared-memory stage.
  std::vector<uint32_t> desc;      // n_pad
  std::vector<int32_t> word_hdr;   // 2 * (n_pad / 32 + 1)
  std::vector<int32_t> and_col;    // entries of rule rows, in row order (+ padding)
  std::vector<int32_t> groups;     // kGroupInts per group (see below)
  int32_t n_groups = 0;
  int32_t n_sec_a = 0;  // leading rows referenced by rule rows: every rule-row entry is below it
};

// Stage geometry of the streamed least-model kernel (shared by compile_host and the kernel):
// word headers | row descriptors | slice of the vector for OR rows | rule-row entries.
constexpr int kGroupWordsMax = 62;                 // words (x32 rows) per group: 2 per consumer warp
constexpr int kStageHdrBytes = 64 * 8;             // room for 64 word headers
constexpr int kStageDescBytes = 64 * 128;          // room for 64 words of row descriptors
constexpr int kStageXWords = 512;                  // vector words for the OR rows of a group
constexpr int kStageXBytes = kStageXWords * 4;
constexpr int kStageColInts = 5504;
constexpr int kStageBytes = kStageHdrBytes + kStageDescBytes + kStageXBytes + kStageColInts * 4;  // 32 KiB
static_assert(kStageBytes == 32768, "stage layout");
constexpr int kGroupInts = 8;  // w0, w1, col0, ncol (-1: global), xw0, nxw (-1: global), 0, 0

enum StreamKind : uint32_t { SK_RULE = 0, SK_OR = 1, SK_SELF = 2 };
constexpr uint32_t kLongWord = 0x80000000u;  // header (second int) flag: descriptors hold lengths only
constexpr uint32_t kHasOr = 0x80000000u;     // header (first int) flag: the word has OR-rule rows
constexpr uint32_t kHasSelf = 0x40000000u;   // header (first int) flag: the word has self-loops

// Builds the matrix; returns LP_OK or LP_ERR_INVALID / LP_ERR_OOM with a message in err.
lp_status compile_host(int32_t n_atoms, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                       const int32_t* body_atom, const uint8_t* body_neg, HostMatrix& hm, std::string& err);
// compile_host on the calling thread alone (its parallel regions get teams of one): for small
// programs, where waking a thread team costs more than the work. Same result.
lp_status compile_host_serial(int32_t n_atoms, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                              const int32_t* body_atom, const uint8_t* body_neg, HostMatrix& hm, std::string& err);
// Programs with at most this many rules plus body literals are standardized by
// compile_host_serial unless lp_compile is asked for the device.
constexpr int64_t kSmallCompile = 1 << 14;
// The streamed layout (desc, word_hdr, and_col, groups) from hm.row_ptr / hm.col, which the
// caller fills with the internal CSR first.
lp_status build_stream_layout(HostMatrix& hm, std::string& err);

// Thread-local error message used by the C ABI.
void set_error(const std::string& msg);

}  // namespace lp

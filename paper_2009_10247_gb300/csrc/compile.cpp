// compile.cpp -- host compiler of liblp: rules -> program matrix M_P in the internal layout.
//
// Sec. 2.1 / 2.2 of the paper (Nguyen, Inoue, Sakama, ICLP 2020): the literal "not q" becomes
// a new atom q-bar (Eq. 4), bodies are sets (footnote of Eq. 2), heads with several rules are
// standardized into an OR-rule over one new atom per rule, and M_P follows Def. 2 and Def. 7.
// The values 1/m are never stored: a rule row fires when all its body atoms hold, an OR row
// when one does, which is theta(M_P v) of Def. 5 evaluated exactly.
//
// Internal order (what the kernels see; outputs are mapped back):
//   section A: original and barred atoms, by descending number of rows that reference them,
//              so that the most gathered bits share a few cache lines;
//   section B: the new atoms, grouped by the OR row that references them (in section-A order
//              of that row, then rule order), so that an OR row gathers one contiguous range;
//   padding:   empty rows up to a multiple of 64.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>

#include "internal.h"

#ifdef _OPENMP
#include <omp.h>
#endif
#if defined(_OPENMP) && defined(__GLIBCXX__)
#include <parallel/algorithm>
#endif

namespace lp {

namespace {

// Wall time of each compile phase, printed to stderr at the end when LP_COMPILE_TRACE is set.
struct PhaseTrace {
  bool on = std::getenv("LP_COMPILE_TRACE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  std::string line;
  void mark(const char* name) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    char buf[64];
    std::snprintf(buf, sizeof buf, "%s=%.2f ", name, std::chrono::duration<double, std::milli>(now - t).count());
    line += buf;
    t = now;
  }
  ~PhaseTrace() {
    if (on && !line.empty()) std::fprintf(stderr, "lp_compile phases (ms): %s\n", line.c_str());
  }
};

inline void sort_small(int32_t* a, int64_t m) {
  if (m > 24) {
    std::sort(a, a + m);
    return;
  }
  for (int64_t i = 1; i < m; i++) {
    int32_t x = a[i];
    int64_t j = i - 1;
    while (j >= 0 && a[j] > x) {
      a[j + 1] = a[j];
      j--;
    }
    a[j + 1] = x;
  }
}

inline int omp_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Sort of 64-bit keys, in parallel where libstdc++'s parallel mode is available.
inline void parallel_sort(hvec<uint64_t>& v) {
#if defined(_OPENMP) && defined(__GLIBCXX__)
  __gnu_parallel::sort(v.begin(), v.end());
#else
  std::sort(v.begin(), v.end());
#endif
}

// v = n copies of x, written by the team.
template <class T>
void par_fill(hvec<T>& v, size_t n, T x) {
  v.resize(n);
  T* d = v.data();
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; i++) d[i] = x;
}

// Blocked exclusive scan over [0, m) on the OpenMP team that actually runs (one thread when
// the caller is itself inside a parallel region, as lp_compile_batch's compiles are): each
// thread counts its contiguous range (count(i0, i1)), one thread sizes the outputs for the
// total (prepare(total)), then each thread writes its range from its offset (emit(i0, i1,
// base)). The output order is the sequential one. Returns the total.
template <typename Count, typename Prepare, typename Emit>
int64_t blocked_scan(int64_t m, Count count, Prepare prepare, Emit emit) {
  std::vector<int64_t> part;
  int nt = 1;
#pragma omp parallel
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#pragma omp single
    nt = omp_get_num_threads();
#endif
#pragma omp single
    part.assign((size_t)nt + 1, 0);
    const int64_t i0 = m * t / nt, i1 = m * (t + 1) / nt;
    part[t + 1] = count(i0, i1);
#pragma omp barrier
#pragma omp single
    {
      for (int q = 0; q < nt; q++) part[q + 1] += part[q];
      prepare(part[nt]);
    }
    emit(i0, i1, part[t]);
  }
  return part[nt];
}

}  // namespace

lp_status compile_host(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                       const int32_t* body_atom, const uint8_t* body_neg, HostMatrix& hm, std::string& err) {
  PhaseTrace trace;
  // ---- validation
  if (n < 0 || n_rules < 0) {
    err = "negative atom or rule count";
    return LP_ERR_INVALID;
  }
  if (n_rules > 0 && (!head || !body_off)) {
    err = "head/body_off must not be NULL when n_rules > 0";
    return LP_ERR_INVALID;
  }
  if (n_rules > 0 && body_off[0] != 0) {
    err = "body_off[0] must be 0";
    return LP_ERR_INVALID;
  }
  int64_t first_bad = n_rules;  // first rule with a bad head or a decreasing body_off
#pragma omp parallel for reduction(min : first_bad) schedule(static)
  for (int64_t r = 0; r < n_rules; r++)
    if (head[r] < 0 || head[r] >= n || body_off[r + 1] < body_off[r]) first_bad = std::min(first_bad, r);
  if (first_bad < n_rules) {
    const int64_t r = first_bad;
    err = (head[r] < 0 || head[r] >= n) ? "head atom out of range at rule " + std::to_string(r)
                                        : "body_off decreases at rule " + std::to_string(r);
    return LP_ERR_INVALID;
  }
  const int64_t total = n_rules > 0 ? body_off[n_rules] : 0;
  if (total > 0 && !body_atom) {
    err = "body_atom must not be NULL when there are body literals";
    return LP_ERR_INVALID;
  }
  if (total >= (int64_t(1) << 31)) {
    err = "too many body literals (must be < 2^31)";
    return LP_ERR_INVALID;
  }
  int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
  for (int64_t e = 0; e < total; e++) bad |= (body_atom[e] < 0 || body_atom[e] >= n);
  if (bad) {
    err = "body atom out of range";
    return LP_ERR_INVALID;
  }

  if (n_rules >= (int64_t(1) << 31) - 1) {
    err = "too many rules (must be < 2^31 - 1)";
    return LP_ERR_INVALID;
  }

  try {
    trace.mark("validate");
    // ---- rules per head, negated atoms, barred ids (canonical: n + rank of q)
    hvec<int32_t> cnt, bar_id;
    par_fill(cnt, (size_t)n, 0);
    par_fill(bar_id, (size_t)n, -1);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n_rules; r++) {
      if (r + 16 < n_rules) __builtin_prefetch(&cnt[head[r + 16]], 1);
      __atomic_fetch_add(&cnt[head[r]], 1, __ATOMIC_RELAXED);
    }
    if (body_neg) {
#pragma omp parallel for schedule(static)
      for (int64_t e = 0; e < total; e++)
        if (body_neg[e]) bar_id[body_atom[e]] = 0;  // every writer stores the same value
    }
    // barred ids n, n + 1, ... in ascending atom order
    const int32_t nb = (int32_t)blocked_scan(
        n,
        [&](int64_t a0, int64_t a1) {
          int64_t c = 0;
          for (int64_t a = a0; a < a1; a++) c += bar_id[a] == 0;
          return c;
        },
        [](int64_t) {},
        [&](int64_t a0, int64_t a1, int64_t k) {
          for (int64_t a = a0; a < a1; a++)
            if (bar_id[a] == 0) bar_id[a] = (int32_t)(n + k++);
        });
    // new atoms for the rules of multi-rule heads, in rule order (blocked prefix count)
    hvec<int32_t> aux;
    par_fill(aux, (size_t)n_rules, -1);
    int64_t naux = 0;
    {
      // ranges follow the team that actually runs (one thread when this compile is itself
      // inside a parallel region, as in lp_compile_batch)
      std::vector<int64_t> part;
      int nt = 1;
#pragma omp parallel
      {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#pragma omp single
        nt = omp_get_num_threads();
#endif
#pragma omp single
        part.assign((size_t)nt + 1, 0);
        const int64_t r0 = n_rules * t / nt, r1 = n_rules * (t + 1) / nt;
        int64_t c = 0;
        for (int64_t r = r0; r < r1; r++) c += cnt[head[r]] >= 2;
        part[t + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int q = 0; q < nt; q++) part[q + 1] += part[q];
        int64_t k = part[t];
        for (int64_t r = r0; r < r1; r++)
          if (cnt[head[r]] >= 2) aux[r] = (int32_t)std::min<int64_t>(INT32_MAX, (int64_t)n + nb + k++);
      }
      naux = part[nt];
    }
    const int64_t n_prime64 = (int64_t)n + nb + naux;
    if (n_prime64 >= (int64_t(1) << 31) - 128) {
      err = "standardized program too large (n' must be < 2^31 - 128)";
      return LP_ERR_INVALID;
    }
    const int32_t np = (int32_t)n_prime64;
    trace.mark("heads");

    // ---- body sets in canonical columns (sorted, duplicates removed), in place per rule
    hvec<int32_t> rb(total);  // every rule writes its whole range
    hvec<int32_t> setlen(n_rules);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t r = 0; r < n_rules; r++) {
      int64_t b = body_off[r], m = body_off[r + 1] - b;
      int32_t* s = rb.data() + b;
      for (int64_t i = 0; i < m; i++) {
        int32_t a = body_atom[b + i];
        s[i] = (body_neg && body_neg[b + i]) ? bar_id[a] : a;
      }
      sort_small(s, m);
      int64_t u = 0;
      for (int64_t i = 0; i < m; i++)
        if (u == 0 || s[u - 1] != s[i]) s[u++] = s[i];
      setlen[r] = (int32_t)u;
    }

    trace.mark("bodies");
    // ---- canonical rows: kind, defining rule, rules of each head (in rule order)
    // hr_off: first position of each head's rules in the grouped order (a scan of the counts).
    hvec<int64_t> hr_off((size_t)n + 1);
    hr_off[0] = 0;
    blocked_scan(
        n,
        [&](int64_t a0, int64_t a1) {
          int64_t c = 0;
          for (int64_t a = a0; a < a1; a++) c += cnt[a];
          return c;
        },
        [](int64_t) {},
        [&](int64_t a0, int64_t a1, int64_t off) {
          for (int64_t a = a0; a < a1; a++) hr_off[a + 1] = off += cnt[a];
        });
    // Rules grouped by head, in rule order within a head: a counting sort over contiguous rule
    // ranges, one per thread (per-thread head counts, a scan over the threads per head, then
    // each thread writes its range in order).
    hvec<int32_t> by_head(n_rules);
    {
      hvec<int32_t> tcnt;
      int nt = 1;
#pragma omp parallel num_threads(std::min(16, std::max(1, omp_max_threads())))
      {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#pragma omp single
        nt = omp_get_num_threads();
#endif
#pragma omp single
        tcnt.resize((size_t)nt * n);
        const int64_t r0 = n_rules * t / nt, r1 = n_rules * (t + 1) / nt;
        int32_t* c = tcnt.data() + (size_t)t * n;
        std::fill(c, c + n, 0);  // each thread clears its own counts
        for (int64_t r = r0; r < r1; r++) {
          if (r + 16 < r1) __builtin_prefetch(&c[head[r + 16]], 1);
          c[head[r]]++;
        }
#pragma omp barrier
#pragma omp for schedule(static)
        for (int32_t a = 0; a < n; a++) {  // exclusive offsets of each thread within head a
          int64_t off = hr_off[a];
          for (int q = 0; q < nt; q++) {
            const int32_t k = tcnt[(size_t)q * n + a];
            tcnt[(size_t)q * n + a] = (int32_t)(off - hr_off[a]);
            off += k;
          }
        }
        for (int64_t r = r0; r < r1; r++) {
          if (r + 16 < r1) {
            __builtin_prefetch(&hr_off[head[r + 16]]);
            __builtin_prefetch(&c[head[r + 16]], 1);
          }
          const int32_t h = head[r];
          by_head[hr_off[h] + c[h]++] = (int32_t)r;
        }
      }
    }
    trace.mark("group");
    auto rule_at = [&](int64_t t) -> int32_t { return by_head[t]; };
    hvec<int8_t> kind;
    hvec<int32_t> row_rule;  // rule defining a RULE/FACT row
    par_fill(kind, (size_t)np, (int8_t)K_EMPTY);
    par_fill(row_rule, (size_t)np, -1);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n_rules; r++)
      if (aux[r] >= 0) {  // a rule of a multi-rule head defines its new atom's row
        kind[aux[r]] = setlen[r] == 0 ? K_FACT : K_RULE;
        row_rule[aux[r]] = (int32_t)r;
      }
#pragma omp parallel for schedule(static)
    for (int32_t a = 0; a < n; a++) {
      if (cnt[a] >= 2) {
        kind[a] = K_OR;
      } else if (cnt[a] == 1) {
        const int32_t r = rule_at(hr_off[a]);
        kind[a] = setlen[r] == 0 ? K_FACT : K_RULE;
        row_rule[a] = r;
      }
    }
#pragma omp parallel for schedule(static)
    for (int32_t a = 0; a < n; a++)
      if (bar_id[a] >= 0) kind[bar_id[a]] = K_BARRED;

    auto row_len = [&](int32_t c) -> int64_t {
      switch (kind[c]) {
        case K_RULE: return setlen[row_rule[c]];
        case K_OR: return hr_off[c + 1] - hr_off[c];
        case K_FACT:
        case K_BARRED: return 1;
        default: return 0;
      }
    };

    trace.mark("kinds");
    // ---- references per canonical column (for the internal order)
    int64_t nnz = 0;
#pragma omp parallel for reduction(+ : nnz) schedule(static)
    for (int32_t c = 0; c < np; c++) nnz += row_len(c);
    if (nnz >= (int64_t(1) << 31)) {
      err = "too many matrix entries (nnz must be < 2^31)";
      return LP_ERR_INVALID;
    }
    const int32_t nA = n + nb;
    // Only rule-row entries count as references (gathers): OR entries point at new atoms,
    // which are placed by their OR row, and self-loops read their own bit. Every body atom is
    // an original or barred atom (< nA); per-thread histograms are summed at the end.
    hvec<int64_t> deg(nA);  // every entry is written below
    {
      hvec<int32_t> local;
      int nt = 1;
#pragma omp parallel
      {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#pragma omp single
        nt = omp_get_num_threads();
#endif
#pragma omp single
        local.resize((size_t)nt * nA);
        int32_t* h = local.data() + (size_t)t * nA;
        std::fill(h, h + nA, 0);  // each thread clears its own histogram
#pragma omp for schedule(static)
        for (int64_t r = 0; r < n_rules; r++) {
          if (setlen[r] == 0) continue;  // facts define self-loop rows
          const int32_t* s = rb.data() + body_off[r];
          for (int32_t i = 0; i < setlen[r]; i++) h[s[i]]++;
        }
#pragma omp for schedule(static)
        for (int32_t c = 0; c < nA; c++) {
          int64_t d = 0;
          for (int q = 0; q < nt; q++) d += local[(size_t)q * nA + c];
          deg[c] = d;
        }
      }
    }

    trace.mark("refs");
    // ---- internal order
    hvec<int32_t> inv(np);  // internal -> canonical (a permutation: every entry is written)
    // bpos[i]: first section-B position (relative to nA) of the new atoms of the OR row at
    // internal position i < nA; an OR row's entries are the run [nA + bpos[i], nA + bpos[i + 1])
    std::vector<int64_t> bpos((size_t)nA + 1, 0);
    {
      // section A by descending references, ties by canonical id: unique keys, so any sort
      // gives the same order
      int64_t maxdeg = 0;
#pragma omp parallel for reduction(max : maxdeg) schedule(static)
      for (int32_t c = 0; c < nA; c++) maxdeg = std::max(maxdeg, deg[c]);
      hvec<uint64_t> key(nA);
#pragma omp parallel for schedule(static)
      for (int32_t c = 0; c < nA; c++) key[c] = ((uint64_t)(maxdeg - deg[c]) << 32) | (uint32_t)c;
      parallel_sort(key);
#pragma omp parallel for schedule(static)
      for (int32_t i = 0; i < nA; i++) inv[i] = (int32_t)(key[i] & 0xffffffffu);
      // section B: each OR row's new atoms, OR rows in section-A order
      auto n_new = [&](int64_t i) -> int64_t {
        const int32_t c = inv[i];
        return kind[c] == K_OR ? hr_off[c + 1] - hr_off[c] : 0;
      };
      blocked_scan(
          nA,
          [&](int64_t i0, int64_t i1) {
            int64_t c = 0;
            for (int64_t i = i0; i < i1; i++) c += n_new(i);
            return c;
          },
          [](int64_t) {},
          [&](int64_t i0, int64_t i1, int64_t off) {
            for (int64_t i = i0; i < i1; i++) bpos[i + 1] = off += n_new(i);
          });
      if (nA + bpos[nA] != np) {
        err = "internal error: new atoms not covered by OR rows";
        return LP_ERR_INVALID;
      }
#pragma omp parallel for schedule(dynamic, 4096)
      for (int32_t i = 0; i < nA; i++) {
        const int32_t c = inv[i];
        if (kind[c] != K_OR) continue;
        int64_t pos = nA + bpos[i];
        for (int64_t t = hr_off[c]; t < hr_off[c + 1]; t++) inv[pos++] = aux[rule_at(t)];
      }
    }
    hm.perm.resize(np);  // inv is a permutation
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < np; i++) {
      if (i + 16 < np) __builtin_prefetch(&hm.perm[inv[i + 16]], 1);
      hm.perm[inv[i]] = i;
    }
    const int32_t npad = (int32_t)(((int64_t)np + 63) / 64 * 64);
    trace.mark("order");

    // ---- internal CSR
    // Row lengths and kinds moved to internal order (sequential reads, one scattered write per
    // row), their running sum into row_ptr, then the rows' entries.
    hm.row_ptr.resize((size_t)npad + 1);
    hm.row_ptr[0] = 0;
    hvec<int8_t> ikind(np);  // kind of internal row i
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < np; c++) {
      if (c + 16 < np) {
        __builtin_prefetch(&hm.row_ptr[hm.perm[c + 16] + 1], 1);
        __builtin_prefetch(&ikind[hm.perm[c + 16]], 1);
      }
      const int32_t i = hm.perm[c];
      hm.row_ptr[i + 1] = (int32_t)row_len(c);
      ikind[i] = kind[c];
    }
    blocked_scan(
        np,
        [&](int64_t i0, int64_t i1) {
          int64_t c = 0;
          for (int64_t i = i0; i < i1; i++) c += hm.row_ptr[i + 1];
          return c;
        },
        [](int64_t) {},
        [&](int64_t i0, int64_t i1, int64_t base) {
          for (int64_t i = i0; i < i1; i++) {
            base += hm.row_ptr[i + 1];
            hm.row_ptr[i + 1] = (int32_t)base;  // nnz < 2^31 was checked
          }
        });
    for (int32_t i = np; i < npad; i++) hm.row_ptr[i + 1] = hm.row_ptr[i];  // empty padding rows
    trace.mark("row_ptr");
    hm.col.resize((size_t)nnz);  // the passes below write every entry of every row
    // rule rows: walk the rules in order (sequential reads of the body sets) and scatter each
    // body, mapped to internal ids and sorted, into its row
    // (the target row's position and entry range are random accesses: they are prefetched a
    // few rules ahead)
    constexpr int64_t kAhead = 16;
    auto target = [&](int64_t r) { return aux[r] >= 0 ? aux[r] : head[r]; };
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t r = 0; r < n_rules; r++) {
      if (r + kAhead < n_rules) __builtin_prefetch(&hm.perm[target(r + kAhead)]);
      if (r + kAhead / 2 < n_rules) __builtin_prefetch(&hm.row_ptr[hm.perm[target(r + kAhead / 2)]]);
      if (setlen[r] == 0) continue;  // a fact: its row is a self-loop
      const int32_t i = hm.perm[target(r)];
      int32_t* d = hm.col.data() + hm.row_ptr[i];
      const int32_t* sb = rb.data() + body_off[r];
      for (int32_t t = 0; t < setlen[r]; t++) d[t] = hm.perm[sb[t]];
      sort_small(d, setlen[r]);
    }
    trace.mark("scatter");
    // self-loop rows (facts, barred atoms) hold their own column; OR rows list their new
    // atoms, which sit consecutively in section B in rule order
#pragma omp parallel for schedule(dynamic, 4096)
    for (int32_t i = 0; i < np; i++) {
      int32_t* d = hm.col.data() + hm.row_ptr[i];
      if (ikind[i] == K_FACT || ikind[i] == K_BARRED) {
        *d = i;
      } else if (ikind[i] == K_OR) {
        for (int64_t t = bpos[i]; t < bpos[i + 1]; t++) *d++ = (int32_t)(nA + t);
      }
    }
    hm.any_mask.resize((size_t)npad / 32);
#pragma omp parallel for schedule(static)
    for (int32_t w = 0; w < npad / 32; w++) {
      uint32_t bits = 0;
      for (int l = 0; l < 32; l++) {
        const int32_t i = 32 * w + l;
        if (i < np && ikind[i] == K_OR) bits |= 1u << l;
      }
      hm.any_mask[w] = bits;
    }

    trace.mark("or_rows");
    // ---- facts, negated atoms, guesses (Def. 4 and Def. 8)
    hvec<int32_t> owner_of_row(np);
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < np; c++) owner_of_row[c] = c < n ? c : -1;
#pragma omp parallel for schedule(static)
    for (int32_t a = 0; a < n; a++)
      if (bar_id[a] >= 0) owner_of_row[bar_id[a]] = a;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n_rules; r++)
      if (aux[r] >= 0) owner_of_row[aux[r]] = head[r];
    hm.fact_mask.assign(((size_t)n + 63) / 64, 0ull);
    int64_t n_rule_rows = 0, n_or_rows = 0;
#pragma omp parallel for reduction(+ : n_rule_rows, n_or_rows) schedule(static)
    for (int32_t c = 0; c < np; c++) {
      n_rule_rows += kind[c] == K_RULE;
      n_or_rows += kind[c] == K_OR;
    }
    // fact rows in canonical order, with their atoms
    blocked_scan(
        np,
        [&](int64_t c0, int64_t c1) {
          int64_t f = 0;
          for (int64_t c = c0; c < c1; c++) f += kind[c] == K_FACT;
          return f;
        },
        [&](int64_t n_fact_rows) {
          hm.fact_row.resize((size_t)n_fact_rows);
          hm.fact_owner.resize((size_t)n_fact_rows);
        },
        [&](int64_t c0, int64_t c1, int64_t f) {
          for (int64_t c = c0; c < c1; c++)
            if (kind[c] == K_FACT) {
              const int32_t a = owner_of_row[c];
              hm.fact_row[f] = hm.perm[c];
              hm.fact_owner[f++] = a;
              __atomic_fetch_or(&hm.fact_mask[a >> 6], 1ull << (a & 63), __ATOMIC_RELAXED);
            }
        });
    par_fill(hm.row_tag, (size_t)npad, -1);
    const int64_t n_fact = (int64_t)hm.fact_row.size();
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < n_fact; f++) hm.row_tag[hm.fact_row[f]] = -2;
    hm.neg_row.clear();
    hm.bar_row.clear();
    hm.guess_row.clear();
    for (int32_t a = 0; a < n; a++) {
      if (bar_id[a] < 0) continue;
      hm.neg_row.push_back(hm.perm[a]);
      hm.bar_row.push_back(hm.perm[bar_id[a]]);
      bool is_fact = (hm.fact_mask[a >> 6] >> (a & 63)) & 1ull;
      if (is_fact) {
        hm.row_tag[hm.perm[bar_id[a]]] = -3;
      } else {
        hm.row_tag[hm.perm[bar_id[a]]] = (int32_t)hm.guess_row.size();
        hm.guess_row.push_back(hm.perm[bar_id[a]]);
      }
    }
    // rule rows refer only to the leading section-A rows that have references
    {
      int32_t ng_atoms = 0;
      while (ng_atoms < nA && deg[inv[ng_atoms]] > 0) ng_atoms++;
      hm.n_sec_a = ng_atoms;
    }

    hm.n = n;
    hm.n_rules = n_rules;
    hm.n_prime = np;
    hm.n_pad = npad;
    hm.nnz = nnz;
    hm.n_barred = nb;
    hm.n_aux = (int32_t)naux;
    hm.k = (int32_t)hm.guess_row.size();
    hm.n_fact_rows = (int32_t)hm.fact_row.size();
    hm.n_rule_rows = (int32_t)n_rule_rows;
    hm.n_or_rows = (int32_t)n_or_rows;
    par_fill(hm.canon_rule, (size_t)np, -1);
#pragma omp parallel for schedule(static)
    for (int32_t c = 0; c < np; c++)
      if (kind[c] == K_RULE) hm.canon_rule[c] = row_rule[c];
    hm.canon_kind.swap(kind);
    trace.mark("facts");
  } catch (const std::bad_alloc&) {
    err = "host allocation failed in lp_compile";
    return LP_ERR_OOM;
  }
  return LP_OK;
}

// Streamed layout of the least-model kernel (row descriptors, word headers, rule-row entries,
// stage groups), from the internal CSR in hm.row_ptr / hm.col. Built on first use of that
// kernel only.
lp_status build_stream_layout(HostMatrix& hm, std::string& err) {
  const int32_t np = hm.n_prime, npad = hm.n_pad, nA = hm.n + hm.n_barred;
  std::vector<int32_t> inv(np);
  for (int32_t c = 0; c < np; c++) inv[hm.perm[c]] = c;
  const hvec<int8_t>& kind = hm.canon_kind;
  try {
    {
      const int32_t nw = npad / 32;
      hm.desc.assign(npad, 0u);
      hm.word_hdr.assign(2 * ((size_t)nw + 1), 0);
      int64_t n_and = 0;
      for (int32_t i = 0; i < np; i++) {
        const int8_t kd = kind[inv[i]];
        const int64_t len = hm.row_ptr[i + 1] - hm.row_ptr[i];
        if (len >= (int64_t(1) << 30)) {
          err = "row too long for the streamed layout";
          return LP_ERR_INVALID;
        }
        uint32_t sk = (kd == K_OR) ? SK_OR : (kd == K_FACT || kd == K_BARRED) ? SK_SELF : SK_RULE;
        hm.desc[i] = (sk << 30) | (uint32_t)len;
        if (sk == SK_RULE) n_and += len;
      }
      hm.and_col.assign((size_t)n_and + 8, 0);
      int64_t ca = 0, oa = nA;  // OR rows' new atoms are section B in OR-row order
      for (int32_t i = 0; i < npad; i++) {
        if ((i & 31) == 0) {
          hm.word_hdr[2 * (i >> 5)] = (int32_t)ca;
          hm.word_hdr[2 * (i >> 5) + 1] = (int32_t)oa;
        }
        if (i >= np) continue;
        const uint32_t sk = hm.desc[i] >> 30;
        const int32_t b = hm.row_ptr[i], e = hm.row_ptr[i + 1];
        if (sk == SK_RULE) {
          for (int32_t t = b; t < e; t++) hm.and_col[ca++] = hm.col[t];
        } else if (sk == SK_OR) {
          for (int32_t t = b; t < e; t++)
            if (hm.col[t] != oa + (t - b)) {
              err = "internal error: OR row entries are not the next new atoms";
              return LP_ERR_INVALID;
            }
          oa += e - b;
        } else if (e - b != 1 || hm.col[b] != i) {
          err = "internal error: self-loop row expected";
          return LP_ERR_INVALID;
        }
      }
      hm.word_hdr[2 * nw] = (int32_t)ca;
      hm.word_hdr[2 * nw + 1] = (int32_t)oa;
      if (ca >= (int64_t(1) << 30)) {
        err = "too many rule entries for the streamed layout (must be < 2^30)";
        return LP_ERR_INVALID;
      }
      // which row kinds a word holds (header bits kHasOr / kHasSelf)
      for (int32_t wd = 0; wd < nw; wd++) {
        uint32_t fl = 0;
        for (int l = 0; l < 32; l++) {
          const uint32_t sk = hm.desc[32 * wd + l] >> 30;
          if (sk == SK_OR) fl |= kHasOr;
          if (sk == SK_SELF) fl |= kHasSelf;
        }
        hm.word_hdr[2 * wd] = (int32_t)((uint32_t)hm.word_hdr[2 * wd] | fl);
      }
      // words whose rows all have <= 32 entries carry each row's offset in its descriptor
      for (int32_t wd = 0; wd < nw; wd++) {
        bool small = true;
        for (int l = 0; l < 32; l++) small &= (hm.desc[32 * wd + l] & 0x3fffffffu) <= 32u;
        if (!small) {
          hm.word_hdr[2 * wd + 1] = (int32_t)((uint32_t)hm.word_hdr[2 * wd + 1] | kLongWord);
          continue;
        }
        uint32_t ao = 0, oo = 0;
        for (int l = 0; l < 32; l++) {
          uint32_t& d = hm.desc[32 * wd + l];
          const uint32_t sk = d >> 30, len = d & 0x3fffffffu;
          const uint32_t off = sk == SK_RULE ? ao : (sk == SK_OR ? oo : 0u);
          if (sk == SK_RULE) ao += len;
          if (sk == SK_OR) oo += len;
          d = (sk << 30) | (off << 6) | len;
        }
      }
      // groups of an even number of words whose entries fit a stage (with alignment slack)
      hm.groups.clear();
      const int32_t cap = kStageColInts - 8;
      int32_t w = 0;
      while (w < nw) {
        int32_t w1 = w;
        auto hdr_col = [&](int32_t wd) { return (int32_t)((uint32_t)hm.word_hdr[2 * wd] & ~(kHasOr | kHasSelf)); };
        auto words_cols = [&](int32_t a, int32_t b2) { return hdr_col(b2) - hdr_col(a); };
        while (w1 < nw && w1 - w < kGroupWordsMax && words_cols(w, std::min(w1 + 2, nw)) <= cap)
          w1 = std::min(w1 + 2, nw);
        int32_t ncol;
        const int32_t c0 = hdr_col(w) & ~3;
        if (w1 == w) {  // one pair of words alone exceeds a stage: its entries stay in global memory
          w1 = std::min(w + 2, nw);
          ncol = -1;
        } else {
          const int32_t c1 = (hdr_col(w1) + 3) & ~3;
          ncol = c1 - c0;
        }
        // the slice of the vector holding the group's OR rows' new atoms (whole 4-word units)
        const int64_t ob0 = (uint32_t)hm.word_hdr[2 * w + 1] & ~kLongWord;
        const int64_t ob1 = (uint32_t)hm.word_hdr[2 * w1 + 1] & ~kLongWord;
        int32_t xw0 = 0, nxw = 0;
        if (ob1 > ob0) {
          xw0 = (int32_t)((ob0 >> 5) & ~int64_t(3));
          const int32_t xw1 = (int32_t)((((ob1 + 31) >> 5) + 3) & ~int64_t(3));
          nxw = xw1 - xw0 <= kStageXWords ? xw1 - xw0 : -1;  // -1: read from global memory
        }
        const int32_t rec[kGroupInts] = {w, w1, c0, ncol, xw0, nxw, 0, 0};
        hm.groups.insert(hm.groups.end(), rec, rec + kGroupInts);
        w = w1;
      }
      hm.n_groups = (int32_t)(hm.groups.size() / kGroupInts);
    }

  } catch (const std::bad_alloc&) {
    err = "host allocation failed building the streamed layout";
    return LP_ERR_OOM;
  }
  return LP_OK;
}

lp_status compile_host_serial(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                              const int32_t* body_atom, const uint8_t* body_neg, HostMatrix& hm, std::string& err) {
  lp_status st = LP_OK;
#ifdef _OPENMP
#pragma omp parallel num_threads(1)
  {
    omp_set_num_threads(1);  // this task's regions (and the parallel sort) run on one thread
    st = compile_host(n, n_rules, head, body_off, body_atom, body_neg, hm, err);
  }
#else
  st = compile_host(n, n_rules, head, body_off, body_atom, body_neg, hm, err);
#endif
  return st;
}

}  // namespace lp

/*
 * oracle.c -- plain CPU oracle (test infrastructure only; see oracle.h).
 *
 * Every function follows one passage of the paper and does nothing beyond it: no row
 * reordering, no bit packing, no blocking. Truth values are one byte per atom, matrix entries
 * are exact rationals num/den, and theta compares the exact row sum with 1.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Input check shared by the two standardization entry points. */
static int check_program(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                         const int32_t* body_atom) {
  if (n < 0 || n_rules < 0) return ORC_ERR_INVALID;
  if (n_rules > 0 && (!head || !body_off)) return ORC_ERR_INVALID;
  if (n_rules > 0 && body_off[0] != 0) return ORC_ERR_INVALID;
  for (int64_t r = 0; r < n_rules; r++) {
    if (head[r] < 0 || head[r] >= n) return ORC_ERR_INVALID;
    if (body_off[r + 1] < body_off[r]) return ORC_ERR_INVALID;
  }
  int64_t total = n_rules > 0 ? body_off[n_rules] : 0;
  if (total > 0 && !body_atom) return ORC_ERR_INVALID;
  for (int64_t e = 0; e < total; e++)
    if (body_atom[e] < 0 || body_atom[e] >= n) return ORC_ERR_INVALID;
  return 0;
}

/*
 * The transformation of Sec. 2.1/2.2 as one pass over the rules:
 *  - positive form (Eq. 4): the literal "not q" becomes the new atom q-bar;
 *  - the footnote of Eq. 2 assumes distinct body atoms, so each body is reduced to its set;
 *  - standardization (Sec. 2.1, Algorithm 1 step 1): a head with k >= 2 rules gets the OR-rule
 *    h <- b_1 | ... | b_k and one new atom b_i <- body(r_i) per rule; a head with one rule keeps it.
 * Atom order: the n original atoms, then the barred atoms by ascending atom id (Def. 7 puts
 * them after p_1..p_n), then the new atoms in rule order (Example 1 puts u, v after p..t).
 * A fact stays a fact: its row is the self-loop a_ii = 1 of Def. 2 item 3.
 */
typedef struct {
  int64_t* cnt;       /* rules per head                          */
  int64_t* barred;    /* column of q-bar, or -1 if q never negated */
  int64_t* aux;       /* new atom of rule r, or -1                  */
  int64_t* setlen;    /* size of the body set of rule r             */
  int64_t n_barred, n_aux;
} std_plan;

static void plan_free(std_plan* p) {
  free(p->cnt);
  free(p->barred);
  free(p->aux);
  free(p->setlen);
}

/* Columns of the body set of rule r, ascending, written to buf; returns the count. */
static int64_t body_set(const std_plan* p, const int64_t* body_off, const int32_t* body_atom,
                        const uint8_t* body_neg, int64_t r, int64_t* buf) {
  int64_t m = 0;
  for (int64_t e = body_off[r]; e < body_off[r + 1]; e++) {
    int neg = body_neg ? body_neg[e] != 0 : 0;
    buf[m++] = neg ? p->barred[body_atom[e]] : (int64_t)body_atom[e];
  }
  qsort(buf, (size_t)m, sizeof(int64_t), cmp_i64);
  int64_t u = 0;
  for (int64_t i = 0; i < m; i++)
    if (u == 0 || buf[u - 1] != buf[i]) buf[u++] = buf[i];
  return u;
}

static int make_plan(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                     const int32_t* body_atom, const uint8_t* body_neg, std_plan* p) {
  memset(p, 0, sizeof(*p));
  int rc = check_program(n, n_rules, head, body_off, body_atom);
  if (rc) return rc;
  p->cnt = calloc((size_t)n + 1, sizeof(int64_t));
  p->barred = malloc(((size_t)n + 1) * sizeof(int64_t));
  p->aux = malloc(((size_t)n_rules + 1) * sizeof(int64_t));
  p->setlen = malloc(((size_t)n_rules + 1) * sizeof(int64_t));
  if (!p->cnt || !p->barred || !p->aux || !p->setlen) {
    plan_free(p);
    return ORC_ERR_INVALID;
  }
  for (int32_t a = 0; a < n; a++) p->barred[a] = -1;
  for (int64_t r = 0; r < n_rules; r++) {
    p->cnt[head[r]]++;
    if (body_neg)
      for (int64_t e = body_off[r]; e < body_off[r + 1]; e++)
        if (body_neg[e]) p->barred[body_atom[e]] = 0;
  }
  for (int32_t a = 0; a < n; a++)
    if (p->barred[a] == 0) p->barred[a] = (int64_t)n + p->n_barred++;
  int64_t maxlen = 0;
  for (int64_t r = 0; r < n_rules; r++) {
    p->aux[r] = p->cnt[head[r]] >= 2 ? (int64_t)n + p->n_barred + p->n_aux++ : -1;
    if (body_off[r + 1] - body_off[r] > maxlen) maxlen = body_off[r + 1] - body_off[r];
  }
  int64_t* buf = malloc(((size_t)maxlen + 1) * sizeof(int64_t));
  if (!buf) {
    plan_free(p);
    return ORC_ERR_INVALID;
  }
  for (int64_t r = 0; r < n_rules; r++) p->setlen[r] = body_set(p, body_off, body_atom, body_neg, r, buf);
  free(buf);
  return 0;
}

/* Row length: a fact row is one self-loop; a single rule is its body set; an OR row has
 * one entry per rule of its head. */
static int64_t rule_row_len(const std_plan* p, int64_t r) { return p->setlen[r] == 0 ? 1 : p->setlen[r]; }

int orc_standardize_size(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                         const int32_t* body_atom, const uint8_t* body_neg, int64_t* sizes) {
  std_plan p;
  int rc = make_plan(n, n_rules, head, body_off, body_atom, body_neg, &p);
  if (rc) return rc;
  int64_t nnz = p.n_barred; /* one self-loop per barred atom (Def. 7 item 1) */
  for (int64_t r = 0; r < n_rules; r++) {
    if (p.cnt[head[r]] >= 2) nnz += 1 + rule_row_len(&p, r); /* OR entry + the new atom's row */
    else nnz += rule_row_len(&p, r);
  }
  sizes[0] = (int64_t)n + p.n_barred + p.n_aux;
  sizes[1] = nnz;
  sizes[2] = p.n_barred;
  sizes[3] = p.n_aux;
  plan_free(&p);
  return 0;
}

int orc_standardize_fill(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                         const int32_t* body_atom, const uint8_t* body_neg, int64_t* row_ptr,
                         int64_t* col, int32_t* num, int32_t* den, int8_t* kind, int64_t* owner) {
  std_plan p;
  int rc = make_plan(n, n_rules, head, body_off, body_atom, body_neg, &p);
  if (rc) return rc;
  int64_t np = (int64_t)n + p.n_barred + p.n_aux;
  int64_t* len = calloc((size_t)np + 1, sizeof(int64_t));
  int64_t maxlen = 1;
  for (int64_t r = 0; r < n_rules; r++)
    if (body_off[r + 1] - body_off[r] > maxlen) maxlen = body_off[r + 1] - body_off[r];
  int64_t* buf = malloc(((size_t)maxlen + 1) * sizeof(int64_t));
  if (!len || !buf) {
    free(len);
    free(buf);
    plan_free(&p);
    return ORC_ERR_INVALID;
  }
  /* kind, owner and row lengths */
  for (int64_t i = 0; i < np; i++) {
    kind[i] = ORC_EMPTY;
    owner[i] = i < n ? i : -1;
  }
  for (int32_t a = 0; a < n; a++)
    if (p.barred[a] >= 0) {
      kind[p.barred[a]] = ORC_BARRED;
      owner[p.barred[a]] = a;
      len[p.barred[a]] = 1;
    }
  for (int64_t r = 0; r < n_rules; r++) {
    int64_t h = head[r];
    if (p.cnt[h] >= 2) {
      kind[h] = ORC_OR;
      len[h] += 1;
      int64_t x = p.aux[r];
      kind[x] = p.setlen[r] == 0 ? ORC_FACT : ORC_AND;
      owner[x] = h;
      len[x] = rule_row_len(&p, r);
    } else {
      kind[h] = p.setlen[r] == 0 ? ORC_FACT : ORC_AND;
      len[h] = rule_row_len(&p, r);
    }
  }
  row_ptr[0] = 0;
  for (int64_t i = 0; i < np; i++) row_ptr[i + 1] = row_ptr[i] + len[i];
  /* entries: cursor per row */
  int64_t* cur = len; /* reuse as write cursor */
  for (int64_t i = 0; i < np; i++) cur[i] = row_ptr[i];
  for (int64_t i = 0; i < np; i++) {
    /* Def. 2 item 4: every row starts all-zero; den = 1 unless set below */
    den[i] = 1;
  }
  for (int32_t a = 0; a < n; a++)
    if (p.barred[a] >= 0) { /* Def. 7 items 1-2: a_ii = 1 on a barred row, nothing else */
      int64_t i = p.barred[a];
      col[cur[i]] = i;
      num[cur[i]++] = 1;
    }
  for (int64_t r = 0; r < n_rules; r++) {
    int64_t h = head[r];
    int64_t row = p.cnt[h] >= 2 ? p.aux[r] : h;
    if (p.cnt[h] >= 2) { /* Def. 2 item 2: the OR-rule h <- b_1 | ... | b_k, a_ij = 1 */
      col[cur[h]] = p.aux[r];
      num[cur[h]++] = 1;
    }
    if (p.setlen[r] == 0) { /* Def. 2 item 3: a fact, a_ii = 1 */
      col[cur[row]] = row;
      num[cur[row]++] = 1;
      den[row] = 1;
    } else { /* Def. 2 item 1: a_ij = 1/m over the m distinct body atoms */
      int64_t m = body_set(&p, body_off, body_atom, body_neg, r, buf);
      for (int64_t j = 0; j < m; j++) {
        col[cur[row]] = buf[j];
        num[cur[row]++] = 1;
      }
      den[row] = (int32_t)m;
    }
  }
  free(len);
  free(buf);
  plan_free(&p);
  return 0;
}

/* Def. 5 applied to M v: u_i = 1 iff sum_j a_ij v_j >= 1. With a_ij = num_ij / den_i and
 * den_i > 0 the comparison is sum_j num_ij v_j >= den_i, exact in integers. */
static void theta_rows(int64_t lo, int64_t hi, const int64_t* row_ptr, const int64_t* col,
                       const int32_t* num, const int32_t* den, const uint8_t* v, uint8_t* u) {
  for (int64_t i = lo; i < hi; i++) {
    int64_t s = 0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) s += (int64_t)num[e] * v[col[e]];
    u[i] = s >= den[i] ? 1 : 0;
  }
}

void orc_theta_step(int64_t n_prime, const int64_t* row_ptr, const int64_t* col, const int32_t* num,
                    const int32_t* den, const uint8_t* v, uint8_t* u) {
#ifdef _OPENMP
#pragma omp parallel
  {
    int t = omp_get_thread_num(), nt = omp_get_num_threads();
    int64_t lo = n_prime * t / nt, hi = n_prime * (t + 1) / nt;
    theta_rows(lo, hi, row_ptr, col, num, den, v, u);
  }
#else
  theta_rows(0, n_prime, row_ptr, col, num, den, v, u);
#endif
}

/* Algorithm 1, steps 4-10: v = v0; u = theta(M v); while u != v: v = u; u = theta(M v). */
static int alg1_core(int64_t n_prime, const int64_t* row_ptr, const int64_t* col, const int32_t* num,
                     const int32_t* den, uint8_t* v, uint8_t* u, int64_t max_iters, int parallel,
                     int64_t* iters_out) {
  int64_t iters = 0;
  for (;;) {
    if (iters >= max_iters) {
      *iters_out = iters;
      return ORC_ERR_NO_FIXPOINT;
    }
    if (parallel) orc_theta_step(n_prime, row_ptr, col, num, den, v, u);
    else theta_rows(0, n_prime, row_ptr, col, num, den, v, u);
    iters++;
    if (memcmp(u, v, (size_t)n_prime) == 0) break;
    memcpy(v, u, (size_t)n_prime);
  }
  *iters_out = iters;
  return 0;
}

int orc_alg1(int64_t n_prime, const int64_t* row_ptr, const int64_t* col, const int32_t* num,
             const int32_t* den, const uint8_t* v0, int64_t max_iters, uint8_t* v_out,
             int64_t* iters_out) {
  uint8_t* u = malloc((size_t)n_prime + 1);
  if (!u) return ORC_ERR_INVALID;
  memcpy(v_out, v0, (size_t)n_prime);
  int rc = alg1_core(n_prime, row_ptr, col, num, den, v_out, u, max_iters, 1, iters_out);
  free(u);
  return rc;
}

/* T_P of Sec. 2.1: T_P(I) = { h | h <- b_1 & ... & b_m in P and {b_1..b_m} subset of I },
 * iterated from the empty set; T_P^n(empty) is the least model (van Emden-Kowalski). With
 * assume_true it runs on the Gelfond-Lifschitz reduct P^I of a normal program. */
int orc_tp_least_model(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                       const int32_t* body_atom, const uint8_t* body_neg, const uint8_t* keep_fact,
                       const uint8_t* assume_true, uint8_t* out, int64_t* iters_out) {
  int rc = check_program(n, n_rules, head, body_off, body_atom);
  if (rc) return rc;
  uint8_t* next = calloc((size_t)n + 1, 1);
  if (!next) return ORC_ERR_INVALID;
  memset(out, 0, (size_t)n);
  int64_t iters = 0;
  for (;;) {
    memset(next, 0, (size_t)n);
    for (int64_t r = 0; r < n_rules; r++) {
      if (body_off[r + 1] == body_off[r] && keep_fact && !keep_fact[head[r]]) continue;
      int fires = 1;
      for (int64_t e = body_off[r]; e < body_off[r + 1] && fires; e++) {
        if (body_neg && body_neg[e]) {
          if (!assume_true) {
            free(next);
            return ORC_ERR_NEGATION;
          }
          if (assume_true[body_atom[e]]) fires = 0; /* rule deleted from the reduct */
        } else if (!out[body_atom[e]]) {
          fires = 0;
        }
      }
      if (fires) next[head[r]] = 1;
    }
    iters++;
    int same = memcmp(next, out, (size_t)n) == 0;
    memcpy(out, next, (size_t)n);
    if (same) break;
  }
  free(next);
  *iters_out = iters;
  return 0;
}

/* Algorithm 3 on one column v: keep it iff a_q + a_qbar = 1 for every barred row. */
static int alg3_column(int64_t n_prime, const int8_t* kind, const int64_t* owner, const uint8_t* v) {
  for (int64_t j = 0; j < n_prime; j++)
    if (kind[j] == ORC_BARRED && v[owner[j]] + v[j] != 1) return 0;
  return 1;
}

int orc_alg23_batch(int32_t n_atoms, int64_t n_prime, const int64_t* row_ptr, const int64_t* col,
                    const int32_t* num, const int32_t* den, const int8_t* kind, const int64_t* owner,
                    int64_t k, const int64_t* guess_rows, int64_t n_guesses, const uint64_t* guesses,
                    int64_t max_iters, uint8_t* stable_out, uint8_t* models_out, int64_t* iters_out) {
  if (k < 0 || k > 64) return ORC_ERR_INVALID;
  for (int64_t j = 0; j < k; j++)
    if (guess_rows[j] < 0 || guess_rows[j] >= n_prime || kind[guess_rows[j]] != ORC_BARRED)
      return ORC_ERR_INVALID;
  int err = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    uint8_t* v = malloc((size_t)n_prime + 1);
    uint8_t* u = malloc((size_t)n_prime + 1);
    if (!v || !u) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = ORC_ERR_INVALID;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int64_t g = 0; g < n_guesses; g++) {
      if (!v || !u) continue;
      /* Def. 8: a column of M_0. Fact rows are 1; a barred row is 0 when its atom is a fact
       * (item 3) or is not guessed; the guessed barred rows take the bits of the guess. */
      for (int64_t i = 0; i < n_prime; i++) v[i] = kind[i] == ORC_FACT ? 1 : 0;
      for (int64_t j = 0; j < k; j++) v[guess_rows[j]] = (uint8_t)((guesses[g] >> j) & 1u);
      int64_t it = 0;
      /* Algorithm 2 steps 4-7 on this column: M = M_0; U = theta(M_P M) until U = M. */
      int rc = alg1_core(n_prime, row_ptr, col, num, den, v, u, max_iters, 0, &it);
      if (iters_out) iters_out[g] = it;
      stable_out[g] = rc == 0 ? (uint8_t)alg3_column(n_prime, kind, owner, v) : 0;
      if (rc) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
        err = rc;
      }
      if (models_out) memcpy(models_out + (size_t)g * (size_t)n_atoms, v, (size_t)n_atoms);
    }
    free(v);
    free(u);
  }
  return err;
}

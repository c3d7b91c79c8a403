/*
 * oracle.h -- plain, slow CPU oracle for the sparse linear-algebraic fixpoint of logic
 * programs (Nguyen, Inoue, Sakama, "Enhancing Linear Algebraic Computation of Logic Programs
 * Using Sparse Representation", ICLP 2020).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load this library. It shares no code, header, table or helper with the CUDA
 * library; the two meet only in the seeded input generators.
 *
 * Program format taken by every function (plain host arrays, never modified):
 *   atoms are 0..n-1; rule r in [0, n_rules) has head[r] and the body literals
 *   body_atom[body_off[r] .. body_off[r+1]); body_neg[e] != 0 marks the literal "not b"
 *   (body_neg may be NULL for a definite program). A rule with an empty body is a fact.
 *
 * Return codes: 0 = ok, ORC_ERR_INVALID = malformed input, ORC_ERR_NO_FIXPOINT = the
 * iteration cap was reached with u != v, ORC_ERR_NEGATION = a negated literal where the
 * function needs a definite program.
 */
#ifndef LP_ORACLE_H
#define LP_ORACLE_H
#include <stdint.h>

#define ORC_ERR_INVALID 1
#define ORC_ERR_NO_FIXPOINT 4
#define ORC_ERR_NEGATION 7

/* Row kinds of the standardized program matrix. */
#define ORC_EMPTY 0  /* atom that heads no rule: all-zero row                       */
#define ORC_AND 1    /* single rule h <- b1 & ... & bm : a_ij = 1/m   (Def. 2 item 1) */
#define ORC_OR 2     /* OR-rule h <- b1 | ... | bl   : a_ij = 1     (Def. 2 item 2)   */
#define ORC_FACT 3   /* fact h <-                    : a_ii = 1     (Def. 2 item 3)   */
#define ORC_BARRED 4 /* new atom q-bar               : a_ii = 1     (Def. 7 items 1-2)*/

/* Sizes of the standardized positive form: sizes[0] = n' (rows), sizes[1] = nnz,
 * sizes[2] = number of barred atoms, sizes[3] = number of new (auxiliary) atoms. */
int orc_standardize_size(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                         const int32_t* body_atom, const uint8_t* body_neg, int64_t* sizes);

/* Fill the CSR of M_P: row_ptr (n'+1), col (nnz), num (nnz), den (n'), kind (n'), owner (n').
 * Entry e of row i has value num[e] / den[i]. owner[i] is the original atom a row stands for
 * (itself for originals, q for q-bar, the rule's head for a new atom). */
int orc_standardize_fill(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                         const int32_t* body_atom, const uint8_t* body_neg, int64_t* row_ptr,
                         int64_t* col, int32_t* num, int32_t* den, int8_t* kind, int64_t* owner);

/* One application u = theta(M v) (Def. 5) with the row sums compared exactly. */
void orc_theta_step(int64_t n_prime, const int64_t* row_ptr, const int64_t* col, const int32_t* num,
                    const int32_t* den, const uint8_t* v, uint8_t* u);

/* Algorithm 1 from v0: returns the fixpoint in v_out and the number of theta applications
 * (the last one shows no change) in *iters_out. Parallel over rows when built with OpenMP. */
int orc_alg1(int64_t n_prime, const int64_t* row_ptr, const int64_t* col, const int32_t* num,
             const int32_t* den, const uint8_t* v0, int64_t max_iters, uint8_t* v_out,
             int64_t* iters_out);

/* Naive T_P iteration T_P^k(empty) on the ORIGINAL (unstandardized) rules until
 * T_P(I) = I. keep_fact (n entries or NULL) drops the fact rules whose head is 0 there.
 * assume_true (n entries or NULL): Gelfond-Lifschitz reduct by this set -- a rule with a
 * negated atom in assume_true is deleted, the other negated literals are removed. Without it a
 * negated literal is an error. *iters_out = number of T_P applications. */
int orc_tp_least_model(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                       const int32_t* body_atom, const uint8_t* body_neg, const uint8_t* keep_fact,
                       const uint8_t* assume_true, uint8_t* out, int64_t* iters_out);

/* Algorithms 2 and 3 one guess at a time (parallel over guesses with OpenMP).
 * guess_rows[j] (j < k) is the barred row set by bit j of a guess; every other barred row
 * starts at 0 and every FACT row at 1 (Def. 8). For guess g: fixpoint column of
 * M_{k+1} = theta(M_P M_k), then the check of Algorithm 3 over every barred row.
 * stable_out[g] = 1 iff the column passes; models_out (n_guesses x n_atoms, nullable) gets the
 * column over the original atoms; iters_out (nullable) the theta applications per guess. */
int orc_alg23_batch(int32_t n_atoms, int64_t n_prime, const int64_t* row_ptr, const int64_t* col,
                    const int32_t* num, const int32_t* den, const int8_t* kind, const int64_t* owner,
                    int64_t k, const int64_t* guess_rows, int64_t n_guesses, const uint64_t* guesses,
                    int64_t max_iters, uint8_t* stable_out, uint8_t* models_out, int64_t* iters_out);

/* Number of OpenMP threads the parallel functions use (1 without OpenMP). */
int orc_num_threads(void);

#endif

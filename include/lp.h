/*
 * lp.h -- C ABI of liblp: the fixpoint of the immediate-consequence operator of a logic
 * program in sparse-matrix form, v_{k+1} = theta(M_P v_k), on one NVIDIA GB300 (sm_103a).
 *
 * Method: Nguyen, Inoue, Sakama, "Enhancing Linear Algebraic Computation of Logic Programs
 * Using Sparse Representation" (ICLP 2020). Section, definition and algorithm numbers below
 * refer to that paper.
 *
 * Conventions shared by every call
 *  - Bit vectors are arrays of uint64_t words, little-endian bit order: item i is bit (i % 64)
 *    of word (i / 64). Bits past the last item of the last word are written as 0 and ignored
 *    on input.
 *  - Pointers named *_dev or documented as "device or host" may be device memory (cudaMalloc,
 *    torch tensors) or host memory (pageable or pinned); liblp asks the CUDA runtime which one
 *    and stages host buffers through device memory it owns. Host buffers make the call
 *    synchronous.
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream). Device work of a call is
 *    ordered on that stream.
 *  - Ownership: the caller owns every buffer it passes; liblp owns the lp_program handle and all
 *    device memory behind it (the program matrix and solver scratch), released by lp_free.
 *  - Errors: every call returns an lp_status; nothing is thrown across the ABI. The message of
 *    the last error of the calling thread is returned by lp_last_error().
 *  - A program handle must not be used by two calls at the same time, nor by calls whose device
 *    work may overlap (the same handle on two streams with no ordering between them): its
 *    device scratch (iterate vectors, control block, tiles) is shared by its solves. Distinct
 *    handles share no device scratch (lp_least_model_static excepted, see there).
 */
#ifndef LP_H
#define LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_program lp_program;

typedef enum {
  LP_OK = 0,
  LP_ERR_INVALID = 1,           /* malformed input or unsupported argument           */
  LP_ERR_OOM = 2,               /* device or host allocation failed                   */
  LP_ERR_CUDA = 3,              /* a CUDA runtime call failed                         */
  LP_ERR_NO_FIXPOINT = 4,       /* max_iters theta applications without u == v        */
  LP_ERR_TOO_MANY_GUESSES = 5,  /* guess count or k beyond what the call supports     */
  LP_ERR_TIMEOUT = 6            /* a bounded device-side wait gave up (kernel aborted) */
} lp_status;

/* lp_compile flags */
#define LP_COMPILE_HOST_ONLY 1u /* build M_P on the host only (no GPU needed): the handle then
                                   serves lp_program_info and lp_export_matrix only          */
#define LP_COMPILE_ON_HOST 2u   /* standardize on the host's threads and upload the matrix
                                   (default: the rules are uploaded and standardized on the
                                   GPU; both give the same matrix, array for array)          */
#define LP_COMPILE_ON_DEVICE 4u /* standardize on the GPU even a small program (by default
                                   programs of at most 16,384 rules plus body literals are
                                   standardized on one host thread, which is faster there)   */

/* lp_least_model flags */
#define LP_ROWS 1u   /* init/out are over all n' rows of M_P in canonical order (see below)   */
#define LP_TIMING 2u /* record CUDA events around the fixpoint kernel (lp_last_solve_stats)   */

typedef struct {
  int64_t n_atoms;      /* n = |B_P|, original atoms                                        */
  int64_t n_rules;      /* rules given to lp_compile                                        */
  int64_t n_prime;      /* n' = rows (and columns) of M_P                                    */
  int64_t nnz;          /* stored entries of M_P                                             */
  int64_t n_barred;     /* distinct negated atoms q (one barred atom q-bar each, Eq. 4)      */
  int64_t n_aux;        /* new atoms introduced by standardization (Sec. 2.1)               */
  int64_t k;            /* guessed barred atoms: negated atoms that are not facts (Def. 8)   */
  int64_t n_fact_rows;  /* rows a_ii = 1 of Def. 2 item 3                                    */
  int64_t n_and_rows;   /* rows of single rules (Def. 2 item 1)                              */
  int64_t n_or_rows;    /* rows of OR-rules (Def. 2 item 2)                                  */
  int64_t device_bytes; /* device memory held by the handle right now                         */
  int64_t upload_bytes; /* bytes lp_compile copied host -> device                            */
  double compile_ms;    /* host time of lp_compile (standardize, order, CSR, upload)         */
} lp_info;

typedef struct {
  int32_t iters;         /* theta applications of the last solve (the last shows no change)  */
  int32_t status;        /* lp_status of the last solve as written by the device             */
  float kernel_ms;       /* duration of the fixpoint kernel (LP_TIMING), else -1            */
  int64_t launches;      /* kernels launched by the last call                                 */
  int64_t tiles;         /* stable models: column tiles processed                            */
  int64_t tile_words;    /* stable models: 64-bit guess words per tile                       */
  int64_t max_tile_iters;/* stable models: largest per-tile iteration count (Algorithm 2's
                            from M_0; from F under stable_frontier 2)                        */
  int64_t sum_tile_iters;/* stable models: sum of per-tile iteration counts                  */
  int64_t frontier_rows;   /* stable models, frontier schedule: rows re-evaluated after each
                              tile's first iteration (summed over iterations and tiles)          */
  int64_t frontier_entries;/* ... their matrix entries                                           */
  int64_t frontier_list;   /* ... changed rows whose dependents were visited                    */
  int64_t frontier_deps;   /* ... dependents visited (entries of the transposed matrix)         */
} lp_solve_stats;

/*
 * lp_compile -- build the program matrix M_P of a (normal) logic program.
 *
 * Sec. 2.1 and Sec. 2.2: the literal "not q" becomes the new atom q-bar (positive form, Eq. 4);
 * each body is taken as a set (the paper assumes distinct body atoms); a head with k >= 2 rules
 * is standardized into the OR-rule h <- b_1 | ... | b_k plus one new atom b_i <- body(r_i) per
 * rule, and a head with one rule keeps it (the result is singly-defined, Def. 1). M_P follows
 * Def. 2 (a_ij = 1/m for a rule with m body atoms, 1 for an OR-rule, a_ii = 1 for a fact) and
 * Def. 7 (a_ii = 1 and nothing else on a barred row); it is stored as CSR (Sec. 3.2) with the
 * values implicit: a row's threshold is its body size for a rule and 1 for an OR-rule or a
 * self-loop, which is theta(sum_j a_ij v_j) of Def. 5 evaluated exactly in integers.
 *
 * Canonical atom order (used by LP_ROWS and lp_export_matrix): the n original atoms, then one
 * barred atom per negated atom by ascending atom id, then the new atoms in rule order. The
 * device copy is stored in an internal order of liblp's choosing; results come back in the
 * original (or canonical) order.
 *
 * Arguments (host arrays, read only, copied): n_atoms >= 0; rules r in [0, n_rules) have
 * head[r] in [0, n_atoms) and body literals body_atom[body_off[r] .. body_off[r+1]) with
 * body_off[0] = 0 and body_off non-decreasing; body_neg (nullable) marks negated literals with
 * a non-zero byte. An empty body is a fact. n_rules, the body literals, n_prime and nnz must
 * stay below 2^31. By default the rules are copied to the device as given and standardized
 * there by kernels on cuda_stream, except that a program of at most 16,384 rules plus body
 * literals is standardized on one host thread and uploaded; with LP_COMPILE_ON_HOST (or
 * LP_COMPILE_HOST_ONLY) the host compiler runs on OpenMP threads (one for such a small
 * program), with LP_COMPILE_ON_DEVICE always on the device. All build the same arrays, and none
 * depends on the number of threads.
 * flags: 0, LP_COMPILE_ON_HOST, LP_COMPILE_ON_DEVICE, or LP_COMPILE_HOST_ONLY (no device memory
 * is touched; solves on such a handle return LP_ERR_INVALID); LP_COMPILE_ON_DEVICE with another
 * flag is LP_ERR_INVALID. cuda_stream: stream of the uploads and the device
 * compile; the call returns after it has finished. On success *out receives a new
 * handle (free it with lp_free). Errors: LP_ERR_INVALID (malformed program), LP_ERR_OOM,
 * LP_ERR_CUDA; *out is then NULL.
 */
lp_status lp_compile(int32_t n_atoms, int64_t n_rules, const int32_t* head, const int64_t* body_off,
                     const int32_t* body_atom, const uint8_t* body_neg, uint32_t flags, void* cuda_stream,
                     lp_program** out);

/* Sizes and statistics of a compiled program (host struct, written on success). */
lp_status lp_program_info(const lp_program* prog, lp_info* out);

/*
 * lp_least_model -- Algorithm 1: v = v0; u = theta(M_P v); while u != v: v = u; u = theta(M_P v).
 *
 * Default mode: init (device or host, ceil(n/64) words, nullable) selects original atoms whose
 * facts enter the initial vector of Def. 4; NULL selects every fact. init must be a subset of
 * the atoms that have a fact rule, else LP_ERR_INVALID (checked on the device). Because every
 * fact row and barred row is a self-loop, the iterates grow monotonically and reach the least
 * model of the program restricted to the selected facts (negated literals count as false: the
 * barred atoms start at 0). out (device or host, ceil(n/64) words) receives the fixpoint over
 * the n original atoms in their original order.
 * LP_ROWS: init (required) and out are ceil(n'/64) words over all n' rows in canonical order;
 * any initial vector is accepted and Algorithm 1 is run literally, so the loop may not
 * converge.
 * max_iters >= 1 bounds the theta applications; reaching it with u != v returns
 * LP_ERR_NO_FIXPOINT (out then holds the last iterate). iters_out (host, nullable) receives
 * the number of theta applications, the last of which showed no change; a non-NULL iters_out
 * or a host buffer makes the call wait for the device and report device-side errors
 * (LP_ERR_INVALID for a bad init, LP_ERR_NO_FIXPOINT, LP_ERR_TIMEOUT). Otherwise the call
 * returns after enqueueing the work and lp_last_solve_stats reports the device status later.
 */
lp_status lp_least_model(lp_program* prog, const uint64_t* init, uint64_t* out, int32_t max_iters,
                         uint32_t flags, int32_t* iters_out, void* cuda_stream);

/*
 * lp_stable_models -- Algorithms 2 and 3 over a batch of guesses (Def. 8 initial matrix).
 *
 * A guess is a k-bit word (k from lp_info): bit j is the initial value of the j-th guessed
 * barred atom (the negated atoms that are not facts, by ascending atom id); 1 means "q is
 * assumed false". Barred atoms of facts start at 0 (Def. 8 item 3) and fact rows at 1.
 * guesses (device or host, n_guesses words) lists the guesses; NULL means all 2^k guesses in
 * order g = 0 .. 2^k - 1 (then n_guesses must equal 2^k, k <= 40). Every column is iterated
 * M_{k+1} = theta(M_P M_k) to its fixpoint and kept iff a_q + a_q-bar = 1 for every negated
 * atom q (Algorithm 3; each rejected column is skipped, the others are all returned).
 * stable_mask (device or host, ceil(n_guesses/64) words): bit g set iff guess g gives a stable
 * model. models (device or host, nullable): max_models rows of ceil(n/64) words; row s gets the
 * s-th stable model in guess order over the n original atoms. n_stable_out (host, nullable):
 * number of stable guesses (may exceed max_models); a non-NULL n_stable_out makes the call wait.
 * max_iters bounds each column tile's theta applications (LP_ERR_NO_FIXPOINT otherwise).
 */
lp_status lp_stable_models(lp_program* prog, const uint64_t* guesses, int64_t n_guesses,
                           uint64_t* stable_mask, uint64_t* models, int64_t max_models,
                           int64_t* n_stable_out, int32_t max_iters, void* cuda_stream);

/*
 * Relaxed (differentiable) fixpoint -- not in the paper: a smooth version of Algorithm 1 for
 * gradient-based learning. Each step applies, row by row, a sigmoid of temperature tau to the
 * row sums x = M_P v of the program matrix (Def. 2/7) in place of theta (Def. 5):
 *   rule row of rule r with m body atoms:  u = sigmoid(w_r (x - 1 + 1/(2m)) / tau), x = the mean
 *   OR-rule row:                           u = sigmoid((x - 1/2) / tau),            x = the sum
 *   self-loop (fact or barred atom):       u = v;     empty row: u = 0.
 * For binary inputs the logit is at least w_r/(2 m tau) in magnitude, so as tau -> 0 each step is
 * theta exactly. Vectors are batches of b columns stored row-major: float [n'][b] over all rows in
 * canonical order (lp_compile). weights: float [n_rules], one per rule given to lp_compile (facts
 * have none: their entry is ignored and their gradient is 0). All buffers are device memory.
 *
 * lp_relaxed_workspace: sizes in floats of the checkpoint buffer (forward -> backward) and the
 * backward scratch for a batch of b columns, `steps` steps and a checkpoint every ckpt_every steps.
 */
lp_status lp_relaxed_workspace(lp_program* prog, int32_t batch, int32_t steps, int32_t ckpt_every,
                               int64_t* ckpt_floats, int64_t* scratch_floats);

/* Forward: v_0 = v0 (float [n'][b]), v_{t+1} = step(v_t), t < steps; vT receives v_steps. ckpt
 * (ckpt_floats, written) keeps every ckpt_every-th iterate for lp_relaxed_backward. Asynchronous on
 * cuda_stream. Errors: LP_ERR_INVALID (sizes, tau <= 0, host pointers), LP_ERR_CUDA. */
lp_status lp_relaxed_forward(lp_program* prog, const float* weights, const float* v0, int32_t batch, int32_t steps,
                             float tau, int32_t ckpt_every, float* ckpt, float* vT, void* cuda_stream);

/* Adjoint of lp_relaxed_forward (same weights, batch, steps, tau, ckpt_every, and its ckpt):
 * given gT = dL/dv_steps (float [n'][b]), writes dweights = dL/dweights (float [n_rules]) and
 * dv0 = dL/dv0 (float [n'][b]). Each segment between checkpoints is recomputed from its
 * checkpoint into scratch (scratch_floats). Weight gradients are summed in float over each 256
 * batch columns of a row and accumulated in double across those sums and the steps. */
lp_status lp_relaxed_backward(lp_program* prog, const float* weights, const float* gT, int32_t batch, int32_t steps,
                              float tau, int32_t ckpt_every, const float* ckpt, float* scratch, float* dweights,
                              float* dv0, void* cuda_stream);

/*
 * Many independent normal programs in one launch (batches of uneven sizes; Algorithms 2 and 3
 * over all 2^k guesses of every program).
 *
 * lp_compile_batch: programs p in [0, n_programs); program p has n_atoms[p] atoms (ids local to
 * the program) and the rules [rule_off[p], rule_off[p+1]) of the concatenated rule arrays head,
 * body_off (over all rules, body_off[0] = 0), body_atom, body_neg (nullable), in the format of
 * lp_compile. Each program is compiled exactly as lp_compile would (on the host's threads);
 * every program needs k <= 16.
 * flags: 0, LP_BATCH_FULL_SWEEP, or LP_BATCH_FROM_M0. By default the programs whose iterate rows
 * hold at most 32 bytes (k <= 8) run the frontier schedule: after a first list of rows and the
 * rows referring to them, each iteration evaluates only the rows one of whose inputs changed in
 * the last one (the compile builds each program's transposed matrix for it), and every column
 * starts from F, the fixpoint of the program from its fact rows with every guessed row zero
 * (computed by one extra launch before the first solve, then kept): the first list is the
 * guessed rows. Under LP_BATCH_FROM_M0 the frontier starts from M_0 (the first list: the rows
 * nonzero in M_0), which gives Algorithm 2's iterates and iteration counts; from F the columns
 * reach the same fixpoints in fewer iterations, and `iters` counts those. The programs with
 * wider rows, and every program under LP_BATCH_FULL_SWEEP, evaluate every row in every
 * iteration from M_0. All give the same stable masks. On success *out receives a handle
 * (lp_batch_free).
 */
#define LP_BATCH_FULL_SWEEP 1u
#define LP_BATCH_FROM_M0 2u
typedef struct lp_batch lp_batch;
lp_status lp_compile_batch(int32_t n_programs, const int32_t* n_atoms, const int64_t* rule_off, const int32_t* head,
                           const int64_t* body_off, const int32_t* body_atom, const uint8_t* body_neg,
                           uint32_t flags, void* cuda_stream, lp_batch** out);

/* Totals of a batch (host outputs, each nullable): programs, rows, stored entries, stable-mask
 * words (sum over programs of ceil(2^k / 64)) and device bytes held. */
lp_status lp_batch_info(const lp_batch* batch, int64_t* n_programs, int64_t* total_rows, int64_t* total_nnz,
                        int64_t* total_mask_words, int64_t* device_bytes);

/* Sizes of program `program` (as lp_program_info) and the first word of its stable mask. */
lp_status lp_batch_program_info(const lp_batch* batch, int32_t program, lp_info* info, int64_t* mask_word_offset);

/*
 * lp_batch_stable_models: for every program, all 2^k guesses (guess g = column g of M_0, Def. 8)
 * are iterated M_{k+1} = theta(M_P M_k) to the fixpoint and checked by Algorithm 3.
 * stable_mask (device or host, total_mask_words): program p's bit g (at its mask_word_offset) is
 * set iff guess g gives a stable model. n_stable (device or host, n_programs, nullable): stable
 * guesses per program; iters (device or host, n_programs, nullable): theta applications until
 * the program's fixpoint (from F under the default frontier schedule; 0 if it had none within
 * max_iters). One cooperative launch runs every
 * program as an independent job (the largest on several blocks, the rest on one block each),
 * each iterated until an application changes none of its words. A host buffer or a non-NULL
 * n_stable / iters makes the call wait;
 * LP_ERR_NO_FIXPOINT if a program reaches max_iters (its mask is then zero); LP_ERR_TIMEOUT if a
 * grid barrier wait gave up (2 s).
 */
lp_status lp_batch_stable_models(lp_batch* batch, uint64_t* stable_mask, int64_t* n_stable, int32_t* iters,
                                 int32_t max_iters, void* cuda_stream);

/* Work of the last lp_batch_stable_models call under the frontier schedule (host outputs,
 * nullable): rows evaluated and their stored entries, summed over programs and iterations, and
 * the bytes those evaluations touch (per evaluated row its list slot, group header, entries,
 * gathered rows, old and new row; per changed row its transposed row pointers and per pushed
 * row its id, stamp and list slot); 0 for full-sweep programs. Waits for cuda_stream. */
lp_status lp_batch_last_stats(const lp_batch* batch, int64_t* rows_evaluated, int64_t* entries_evaluated,
                              int64_t* bytes_touched, void* cuda_stream);

/* Release a batch and its device memory (NULL is a no-op; small buffers go to the cache that
 * lp_free describes). */
void lp_batch_free(lp_batch* batch);

/*
 * Schedules and the autotuner. A schedule fixes how the solves of one handle map onto the GPU:
 * which least-model kernel runs and with how many resident CTAs per SM, and how wide the
 * stable-model column tiles are (Algorithm 2 processes the 2^k columns of M_0 a tile at a
 * time). Every schedule computes the same result; only the time differs. A host-only handle
 * starts with all fields 0. A device handle starts with fixpoint_kernel 3 if the program fits
 * one block's shared memory, else 2 with fixpoint_stage 1 (0 where the sliced layout's indices
 * would overflow), and stable_frontier 2; the other fields are 0 (LP_FIXPOINT=stream in the
 * environment makes fixpoint_kernel default to 1).
 */
typedef struct {
  int32_t fixpoint_kernel;        /* least model: 0 = warps over 32-row output words, the words'
                                     entries in 32-entry chunks; 1 = rows streamed through shared
                                     memory in bulk-copy stages (its layout is built from the
                                     device matrix on first use, which downloads the CSR once);
                                     2 = a sliced layout: rows renumbered by length within
                                     windows, 128-row groups padded to their longest row and
                                     stored column-major, a lane per row, blocks given equal
                                     shares of the work (built on the device from the CSR on
                                     first use); 3 = one block with kernel 2's layout and both
                                     vectors in shared memory, a block barrier per iteration
                                     (small programs only: lp_set_schedule builds the layout and
                                     returns LP_ERR_INVALID if it does not fit one block)        */
  int32_t fixpoint_blocks_per_sm; /* least model: resident CTAs per SM; 0 = all that fit        */
  int32_t fixpoint_row_split;     /* least model, kernel 0: warps sharing one 32-row output word
                                     (1, 2, 4 or 8; 0 = 1): more for programs with long rows    */
  int32_t fixpoint_chunk_batch;   /* least model, kernel 0: 32-entry chunks whose loads a warp
                                     issues together (1 or 4; 0 = 1): 4 for long rows            */
  int32_t fixpoint_row_map;       /* least model, kernel 0: 0 = a warp per 32-row word (the
                                     chunks above); a thread per row, for short rows: 1 = two
                                     words per warp step, 2 = four words, 3 = loads pipelined
                                     over the warp's words. 1-3 need row split and chunk batch
                                     0 or 1                                                      */
  int32_t stable_tile_words;      /* stable models: 64-bit guess words per tile, 1, 2, 4, 8, 16
                                     or 32 (capped at the guesses' words); 0 = the widest whose
                                     two iterate buffers fit 1 GiB                               */
  int32_t stable_blocks_per_sm;   /* stable models: resident CTAs per SM; 0 = all that fit      */
  int32_t stable_row_split;       /* stable models: 1 = one row per warp, its entries split over
                                     the warp's lane groups (long rows); 0 = 32 / W rows per warp */
  int32_t stable_frontier;        /* stable models: 1 = all tiles at once, each iteration
                                     evaluating only the rows that changed and the rows that refer
                                     to them, starting from the rows nonzero in M_0 (same iterates
                                     and iteration counts; the transposed matrix is built on the
                                     device on first use; the iterate buffers of up to 8 GiB,
                                     LP_FRONTIER_BYTES, stay allocated and are restored to their
                                     rest state after each solve); 2 = the same from F, the
                                     fixpoint reached from the fact rows with every guessed row 0
                                     (the part of every column's fixpoint no guess changes;
                                     computed once per handle by a least-model solve): the same
                                     stable bits and models in fewer iterations, and the reported
                                     iteration counts are those from F; 0 = a full sweep per tile;
                                     1 and 2 need stable_row_split 0; the autotuner tries all   */
  int32_t fixpoint_stage;         /* least model, kernel 2: 0 = copy the vector prefix that rule
                                     rows gather into shared memory every iteration when it fits
                                     (160 KB); 1 = gather from global memory (through L1)         */
} lp_schedule;

typedef struct {
  lp_schedule schedule;
  int32_t solve;                  /* LP_TUNE_LEAST or LP_TUNE_STABLE: the solve that was timed   */
  float ms;                       /* median time of the timed runs; -1 if the schedule could not
                                     run (e.g. its tiles did not fit in device memory)           */
} lp_tune_record;

#define LP_TUNE_LEAST 1u   /* time lp_least_model from the fact vector                         */
#define LP_TUNE_STABLE 2u  /* time lp_stable_models on all 2^k guesses (k > 16: the first 2^16) */

/* Read / replace the handle's schedule. lp_set_schedule rejects values outside the ranges
 * above with LP_ERR_INVALID and leaves the schedule unchanged. */
lp_status lp_get_schedule(const lp_program* prog, lp_schedule* out);
lp_status lp_set_schedule(lp_program* prog, const lp_schedule* schedule);

/*
 * lp_autotune -- run every candidate schedule of the selected solves (what: LP_TUNE_LEAST
 * and/or LP_TUNE_STABLE) on this program: one warm-up run, then reps (>= 1) runs timed with
 * CUDA events on cuda_stream; keep the fastest for each solve in the handle. Every
 * candidate's result (least model, stable mask) is compared bit for bit with the first
 * candidate's; a difference returns LP_ERR_CUDA. records (host, nullable): up to
 * max_records entries, one per candidate in the order run; *n_records (nullable) = number of
 * candidates. Blocks the calling thread. Candidates: least model, kernel 0 with all / 4 / 2
 * CTAs per SM, kernel 0 with row splits 1, 2, 4, 8 and chunk batches 1, 4, kernel 0 with row
 * maps 1, 2, 3, kernel 1 with all / 1 CTAs per SM, kernel 2 with and without staging, and
 * kernel 3 when the matrix fits one block's shared memory; stable
 * models, tile widths 1..32 with all / half the CTAs per SM, and each width with the row split.
 */
lp_status lp_autotune(lp_program* prog, uint32_t what, int32_t reps, lp_tune_record* records, int32_t max_records,
                      int32_t* n_records, void* cuda_stream);

/*
 * lp_stable_search -- stable models by fixed-budget guess sampling and local search, for k too
 * large to enumerate 2^k columns (the paper's future work, Sec. 5). A population of
 * `population` (1..2048) guesses -- k-bit words as in lp_stable_models -- is drawn from a
 * counter-based generator (SplitMix64 of seed, round, column). Each of `rounds` rounds runs
 * Algorithm 2 on the population (one column tile) and Algorithm 3 on every column. A stable
 * column's guess is recorded, and the column restarts from a fresh random guess. A failed
 * column moves to the guess its fixpoint implies (bit j = 1 iff the j-th guessed atom is false
 * there); if that is the guess it held one round earlier, the bits that step would flip are
 * drawn at random instead.
 * Every reported guess is stable (Algorithm 3 accepted it); the search is not complete.
 * found (device or host, max_found words, nullable if max_found = 0): the distinct stable
 * guesses found, ascending; *n_found (host, required): how many there are (may exceed
 * max_found). Waits for cuda_stream. k <= 64. The handle's schedule is left unchanged.
 */
lp_status lp_stable_search(lp_program* prog, int32_t population, int32_t rounds, uint64_t seed, uint64_t* found,
                           int64_t max_found, int64_t* n_found, void* cuda_stream);

/*
 * lp_check_grid_barrier -- diagnostics, no counterpart in the paper: runs the bounded grid
 * barrier that every persistent kernel of liblp meets once per theta iteration, alone, with
 * `blocks` co-resident CTAs of which the first `absent` never arrive (like a block or rank that
 * has left). The others wait at most limit_us microseconds (1..2e6), then record
 * LP_ERR_TIMEOUT, raise the abort flag and return, so the context stays usable. *status_out
 * (host) receives LP_OK if the barrier completed, else the device status (LP_ERR_TIMEOUT);
 * *ms_out (host, nullable) the kernel's duration. Waits for cuda_stream. LP_ERR_INVALID if
 * `blocks` cannot be co-resident.
 */
lp_status lp_check_grid_barrier(int32_t blocks, int32_t absent, int32_t limit_us, int32_t* status_out, float* ms_out,
                                void* cuda_stream);

/* Statistics and device status of the last solve on this handle; waits for cuda_stream. */
lp_status lp_last_solve_stats(lp_program* prog, lp_solve_stats* out, void* cuda_stream);

/*
 * lp_export_matrix -- the compiled M_P in canonical order, as the CSR of Sec. 3.2, for
 * checking lp_compile. Host arrays: row_ptr (n'+1), col (nnz), threshold (n'): the number of
 * body atoms of a rule row (its entries are 1/threshold), 1 for an OR-rule or a self-loop,
 * 0 for an empty row. kind (n', nullable): 0 empty, 1 rule, 2 OR-rule, 3 fact, 4 barred.
 * Within a row the columns are ascending.
 */
lp_status lp_export_matrix(const lp_program* prog, int64_t* row_ptr, int64_t* col, int32_t* threshold,
                           int8_t* kind, void* cuda_stream);

/*
 * lp_least_model_static -- Algorithm 1 on a matrix the caller already holds in device memory,
 * without allocating anything. The paper has no counterpart: this is a deployment variant of
 * lp_least_model for callers that may not call cudaMalloc or cudaFree, such as code that runs
 * under another framework's fixed device-memory pool or budget, or a latency-critical loop that
 * cannot afford the synchronisation an allocation can cause.
 *
 * Its only scratch (a second iterate vector and a control block) is one fixed array of
 * 256 B + 2 MiB compiled into liblp; every GPU that loads the library holds it until the process
 * exits. Hence n_rows <= 2^24 (16,777,216); larger matrices return LP_ERR_INVALID with a message.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress) and queries the
 * kernel's occupancy; make that first call before any stream capture. Every call on a device
 * shares the array and it keeps the previous call's contents (the control block is cleared
 * at the start of each call): calls that overlap on the GPU -- on different streams or threads
 * -- race and must not be issued.
 *
 * Matrix (device, read only): row_ptr (n_rows + 1 int32, non-decreasing, row_ptr[0] = 0), col
 * (row_ptr[n_rows] int32 column ids in [0, n_rows); an id outside is reported as
 * LP_ERR_INVALID and counts as false), threshold (n_rows int32): row i becomes true when at
 * least threshold[i] of its entries are true. The row pointers themselves are NOT checked: the
 * kernel reads col[row_ptr[0] .. row_ptr[n_rows]), so row_ptr must be non-decreasing and its
 * last value must not exceed the length of the col buffer (a larger one reads past the buffer).
 * For the threshold: row i becomes true when at
 * least threshold[i] of its entries are true -- the body size for a rule (entries 1/m), 1 for an
 * OR-rule or a self-loop; values below 1 count as 1. lp_export_matrix returns this form.
 * v0 (device, ceil(n_rows/64) words): initial vector over the rows; out (device, same size,
 * may be v0 itself): receives the fixpoint (or the last iterate when max_iters is reached).
 * Host pointers are rejected (LP_ERR_INVALID): nothing is staged. iters_out (host, nullable):
 * when given, the call waits for the device and reports the theta applications and the device
 * status (LP_ERR_NO_FIXPOINT, LP_ERR_INVALID, LP_ERR_TIMEOUT); when NULL it only enqueues.
 */
lp_status lp_least_model_static(int32_t n_rows, const int32_t* row_ptr, const int32_t* col, const int32_t* threshold,
                                const uint64_t* v0, uint64_t* out, int32_t max_iters, int32_t* iters_out,
                                void* cuda_stream);

/* Release a handle and its device memory (NULL is a no-op). It waits for the device to finish
 * its work, as cudaFree does; then device buffers of up to 256 KiB go to a per-process cache
 * that later handles reuse (at most 16 MiB in all, never returned before the process exits;
 * LP_ALLOC_CACHE=0 in the environment turns the cache off) and the others back to the driver.
 * The pinned host control block is kept for reuse the same way. */
void lp_free(lp_program* prog);

/* Diagnostics, no counterpart in the paper: checks the invariants the kernels rely on without
 * re-checking them per access -- row pointers start at 0, never decrease and end at nnz; every
 * column index is a row of the matrix; every fact row is a self-loop -- on the device copy
 * (a small kernel; waits for cuda_stream) or, for an LP_COMPILE_HOST_ONLY handle, on the host
 * copy. *n_bad (host) receives the number of violations (0 for every matrix lp_compile builds). */
lp_status lp_check_matrix(const lp_program* prog, int64_t* n_bad, void* cuda_stream);

/* Diagnostics, no counterpart in the paper: copies internal array `which` of a device handle
 * to host memory `out` (the two compilers are compared with it). which: 0 row_ptr (n_pad + 1
 * int32), 1 col (nnz int32), 2 perm (canonical -> internal, n' int32), 3 any_mask (n_pad / 32
 * uint32), 4 row_tag (n_pad int32), 5 fact_row (fact rows int32), 6 fact_owner (same), 7
 * fact_mask (ceil(n / 64) uint64), 8 neg_row (n_barred int32), 9 bar_row (same). *bytes (host)
 * receives the array's size; out may be NULL to ask for it, else it must hold that many bytes.
 * Waits for cuda_stream. Errors: LP_ERR_INVALID (NULL handle or bytes, unknown which, a
 * host-only handle). */
lp_status lp_debug_internal(const lp_program* prog, int32_t which, void* out, int64_t* bytes, void* cuda_stream);

/* Test hook, no counterpart in the paper: after `after` more successful device allocations by
 * liblp, the next one fails (once) as if the device were out of memory, so that the
 * LP_ERR_OOM paths of every call can be exercised without exhausting a GPU. -1 turns it off.
 * Process-wide; not for concurrent use with other liblp calls. */
void lp_debug_fail_alloc(int64_t after);

/* Message of the last failed call on this thread ("" if none). Valid until the next call. */
const char* lp_last_error(void);

/* Number of kernels liblp has launched in this process (all handles). */
int64_t lp_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* LP_H */

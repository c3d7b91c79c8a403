/* A plain C consumer of liblp's ABI that solves on the GPU (no Python in the process): compiles
 * the programs of Example 1 (Sec. 2.1) and Example 2 (Sec. 2.2) and a two-atom even loop, runs
 * lp_least_model (Algorithm 1) and lp_stable_models (Algorithms 2 and 3) with host buffers
 * (liblp stages them through device memory), and prints the results. Built and run by
 * tests/test_c_abi.py on a machine with a GPU. */
#include <stdio.h>

#include "lp.h"

static int compile(int32_t n, int64_t n_rules, const int32_t* head, const int64_t* off, const int32_t* atom,
                   const uint8_t* neg, lp_program** prog) {
  lp_status st = lp_compile(n, n_rules, head, off, atom, neg, 0u, NULL, prog);
  if (st != LP_OK) printf("compile failed: %d %s\n", (int)st, lp_last_error());
  return st == LP_OK;
}

int main(void) {
  /* Example 1: atoms p q r s t = 0..4;  p :- q, r.  p :- s, t.  r :- s.  q :- t.  s.  t. */
  {
    const int32_t head[6] = {0, 0, 2, 1, 3, 4};
    const int64_t off[7] = {0, 2, 4, 5, 6, 6, 6};
    const int32_t atom[6] = {1, 2, 3, 4, 3, 4};
    lp_program* prog = NULL;
    if (!compile(5, 6, head, off, atom, NULL, &prog)) return 1;
    uint64_t out[1] = {0};
    int32_t iters = 0;
    lp_status st = lp_least_model(prog, NULL, out, 100, 0u, &iters, NULL);
    printf("example1 least %d model %llu iters %d\n", (int)st, (unsigned long long)out[0], (int)iters);
    uint64_t init[1] = {1ull << 3}; /* only the fact s */
    st = lp_least_model(prog, init, out, 100, 0u, &iters, NULL);
    printf("example1 facts_s %d model %llu iters %d\n", (int)st, (unsigned long long)out[0], (int)iters);
    lp_free(prog);
  }
  /* Example 2: atoms p q s t u v = 0..5;  p :- q, s.  q :- p, t.  s :- not t.  t.  u :- v. */
  {
    const int32_t head[5] = {0, 1, 2, 3, 4};
    const int64_t off[6] = {0, 2, 4, 5, 5, 6};
    const int32_t atom[6] = {1, 2, 0, 3, 3, 5};
    const uint8_t neg[6] = {0, 0, 0, 0, 1, 0};
    lp_program* prog = NULL;
    if (!compile(6, 5, head, off, atom, neg, &prog)) return 1;
    lp_info info;
    if (lp_program_info(prog, &info) != LP_OK) return 2;
    uint64_t mask[1] = {0}, models[1] = {0};
    int64_t n_stable = -1;
    lp_status st = lp_stable_models(prog, NULL, (int64_t)1 << info.k, mask, models, 1, &n_stable, 1000, NULL);
    printf("example2 stable %d k %d mask %llu n_stable %lld model %llu\n", (int)st, (int)info.k,
           (unsigned long long)mask[0], (long long)n_stable, (unsigned long long)models[0]);
    lp_free(prog);
  }
  /* p :- not q.  q :- not p.  (atoms p q = 0, 1): stable models {p} and {q} */
  {
    const int32_t head[2] = {0, 1};
    const int64_t off[3] = {0, 1, 2};
    const int32_t atom[2] = {1, 0};
    const uint8_t neg[2] = {1, 1};
    lp_program* prog = NULL;
    if (!compile(2, 2, head, off, atom, neg, &prog)) return 1;
    uint64_t mask[1] = {0}, models[4] = {0, 0, 0, 0};
    int64_t n_stable = -1;
    lp_status st = lp_stable_models(prog, NULL, 4, mask, models, 4, &n_stable, 1000, NULL);
    printf("evenloop stable %d mask %llu n_stable %lld models %llu %llu\n", (int)st, (unsigned long long)mask[0],
           (long long)n_stable, (unsigned long long)models[0], (unsigned long long)models[1]);
    lp_free(prog);
  }
  return 0;
}

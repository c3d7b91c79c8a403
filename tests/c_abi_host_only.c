/* A plain C consumer of liblp's ABI (no Python): compiles the program of Example 1 (Sec. 2.1)
 * on the host only, prints its standardized matrix as CSR (Sec. 3.2, Example 4) in canonical
 * order, and checks that a solve on a host-only handle is refused with a message. Built and run
 * by tests/test_c_abi.py. */
#include <stdio.h>
#include <string.h>

#include "lp.h"

int main(void) {
  /* atoms p q r s t = 0..4;  p :- q, r.  p :- s, t.  r :- s.  q :- t.  s.  t. */
  const int32_t head[6] = {0, 0, 2, 1, 3, 4};
  const int64_t body_off[7] = {0, 2, 4, 5, 6, 6, 6};
  const int32_t body_atom[6] = {1, 2, 3, 4, 3, 4};
  lp_program* prog = NULL;
  lp_status st = lp_compile(5, 6, head, body_off, body_atom, NULL, LP_COMPILE_HOST_ONLY, NULL, &prog);
  if (st != LP_OK) {
    printf("compile failed: %d %s\n", (int)st, lp_last_error());
    return 1;
  }
  lp_info info;
  if (lp_program_info(prog, &info) != LP_OK) return 2;
  int64_t row_ptr[16], col[32];
  int32_t threshold[16];
  int8_t kind[16];
  if (info.n_prime > 15 || info.nnz > 32) return 3;
  if (lp_export_matrix(prog, row_ptr, col, threshold, kind, NULL) != LP_OK) return 4;
  printf("n_prime %d nnz %lld\n", (int)info.n_prime, (long long)info.nnz);
  printf("row_ptr");
  for (int i = 0; i <= info.n_prime; i++) printf(" %lld", (long long)row_ptr[i]);
  printf("\ncol");
  for (int64_t e = 0; e < info.nnz; e++) printf(" %lld", (long long)col[e]);
  printf("\nthreshold");
  for (int i = 0; i < info.n_prime; i++) printf(" %d", (int)threshold[i]);
  printf("\n");
  uint64_t out[1] = {0};
  st = lp_least_model(prog, NULL, out, 100, 0u, NULL, NULL);
  printf("host-only solve %d %s\n", (int)st, strlen(lp_last_error()) > 0 ? "with message" : "without message");
  lp_free(prog);
  return 0;
}

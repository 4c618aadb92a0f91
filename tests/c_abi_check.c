/* Compiled as C99 against include/stokesmg.h and linked to the library by
 * tests/test_abi.py: the boundary is plain C.  Without a GPU it exercises
 * only the calls that must fail before touching a device; with one (argv[1]
 * == "gpu") it also sets up a 4^3, k = 2 problem and reads its layout. */
#include <stdio.h>
#include <string.h>

#include "stokesmg.h"

int main(int argc, char** argv) {
  stk_options opt;
  if (stk_default_options(&opt) != STK_OK) return 1;
  if (opt.gmres_restart != 20 || opt.local_cg_iters != 15) return 2;
  stk_problem* P = NULL;
  if (stk_setup(10, 2, 1.0, &opt, &P) != STK_EINVAL || P != NULL) return 3;  /* 10 is not 2 or 3 times 2^L */
  if (strlen(stk_last_error(NULL)) == 0) return 4;
  if (stk_setup(8, 9, 1.0, &opt, &P) != STK_EINVAL) return 5;                 /* degree out of range */
  if (stk_destroy(NULL) != STK_OK) return 6;
  if (stk_solve_batch(NULL, 0, NULL, NULL, 1e-8, NULL) != STK_EINVAL) return 7;
  if (argc > 1 && strcmp(argv[1], "gpu") == 0) {
    if (stk_setup(4, 2, 1.0, &opt, &P) != STK_OK) return 10;
    int n = 0;
    int64_t nv = 0, np = 0, nt = 0;
    if (stk_layout(P, 1, &n, &nv, &np, &nt) != STK_OK || n != 4) return 11;
    printf("layout n=%d total=%lld\n", n, (long long)nt);
    stk_destroy(P);
  }
  printf("c abi ok\n");
  return 0;
}

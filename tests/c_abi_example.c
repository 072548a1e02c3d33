/* The library used from plain C (C11), through include/fock.h alone: the
 * host-only entry points, which need no GPU.  Prints one line per check,
 *   <name> <value ...>
 * and returns 0 when every call returned the status the header documents. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "fock.h"

static int failures = 0;

static void expect(const char* what, fock_status got, fock_status want) {
  if (got != want) {
    printf("unexpected %s %d (%s) %s\n", what, (int)got, fock_status_string(got), fock_last_error(NULL));
    ++failures;
  }
}

int main(void) {
  /* the 24^3 / L = 10 bohr / Ecut = 10 Ha sphere: size query, then the list */
  const int grid[3] = {24, 24, 24};
  const double cell[9] = {10.0, 0.0, 0.0, 0.0, 10.0, 0.0, 0.0, 0.0, 10.0};
  int64_t npw = 0;
  expect("gsphere size", fock_gsphere(grid, cell, 10.0, &npw, NULL, 0), FOCK_OK);
  int32_t* miller = (int32_t*)malloc((size_t)npw * 3 * sizeof(int32_t));
  expect("gsphere list", fock_gsphere(grid, cell, 10.0, &npw, miller, npw), FOCK_OK);
  printf("npw %lld\n", (long long)npw);
  printf("first %d %d %d\n", miller[0], miller[1], miller[2]);
  printf("last %d %d %d\n", miller[3 * (npw - 1)], miller[3 * (npw - 1) + 1], miller[3 * (npw - 1) + 2]);
  expect("gsphere short", fock_gsphere(grid, cell, 10.0, &npw, miller, npw - 1), FOCK_ERR_INVALID_ARG);
  free(miller);

  /* the pair schedule of 10 bands in 3 shards: every unique pair once */
  int64_t total = 0;
  for (int shard = 0; shard < 3; ++shard) {
    int64_t n = 0;
    expect("schedule size", fock_schedule(10, 4, shard, 3, NULL, 0, &n), FOCK_OK);
    int32_t* pairs = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * 2 * sizeof(int32_t));
    expect("schedule list", fock_schedule(10, 4, shard, 3, pairs, n, &n), FOCK_OK);
    for (int64_t k = 0; k < n; ++k)
      if (pairs[2 * k] > pairs[2 * k + 1]) ++failures;
    total += n;
    free(pairs);
  }
  printf("pairs %lld\n", (long long)total);

  /* status strings and the shared argument rules */
  printf("status %s|%s\n", fock_status_string(FOCK_OK), fock_status_string(FOCK_ERR_GRID_TOO_SMALL));
  expect("destroy NULL", fock_destroy(NULL), FOCK_OK);
  expect("npw NULL", fock_plan_npw(NULL, &npw), FOCK_ERR_INVALID_ARG);
  expect("create NULL", fock_plan_create(NULL, grid, cell, 10.0, FOCK_KERNEL_SPENCER_ALAVI, NULL, 0,
                                         FOCK_PREC_FP64, 0u),
         FOCK_ERR_INVALID_ARG);
  printf("failures %d\n", failures);
  return failures == 0 ? 0 : 1;
}

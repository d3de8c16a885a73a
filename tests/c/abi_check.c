/* Plain C99 user of include/ttm.h: compiles against the header alone, links against
 * libttm.so, and exercises the calls that need no GPU (version, argument and option
 * validation, host-side output planning). */
#include <stdio.h>
#include <string.h>

#include "ttm.h"

static int failures = 0;
#define CHECK(cond)                                                \
  do {                                                             \
    if (!(cond)) {                                                 \
      fprintf(stderr, "FAILED %s:%d: %s\n", __FILE__, __LINE__, #cond); \
      ++failures;                                                  \
    }                                                              \
  } while (0)

int main(void) {
  ttm_handle *h = NULL;
  ttm_options opt;
  int64_t bA[3] = {1, 2, 1}, bB[3] = {1, 2, 1};
  double a0[4] = {1, 0, 0, 1}, a1[4] = {1, 2, 3, 4};
  double *coresA[2] = {a0, a1}, *coresB[2] = {a0, a1};
  ttm_tt A, B;

  CHECK(strncmp(ttm_version(), "ttm-gb300", 9) == 0);

  /* NULL arguments are rejected before any CUDA call */
  CHECK(ttm_create(NULL, 0, NULL, NULL) == TTM_ERR_INVALID_ARG);
  CHECK(ttm_multiply(NULL, NULL, NULL, NULL, NULL) == TTM_ERR_INVALID_ARG);

  /* option validation happens before the device is touched */
  memset(&opt, 0, sizeof(opt));
  opt.prec = TTM_PREC_FP64;
  opt.eps = 1.5;
  CHECK(ttm_create(&h, 0, NULL, &opt) == TTM_ERR_INVALID_ARG);
  CHECK(strstr(ttm_last_error(), "eps") != NULL);
  opt.eps = 0.0;
  opt.prec = TTM_PREC_TF32X3;
  CHECK(ttm_create(&h, 0, NULL, &opt) == TTM_ERR_UNSUPPORTED);
  opt.prec = TTM_PREC_FP64;
  opt.f32_block = 5;
  CHECK(ttm_create(&h, 0, NULL, &opt) == TTM_ERR_INVALID_ARG);
  opt.f32_block = 0;

  /* host-side planning: a two-site product of bond-2 trains */
  A.L = 2; A.d = 2; A.on_host = 1; A.reserved = 0; A.bonds = bA; A.cores = coresA;
  B.L = 2; B.d = 2; B.on_host = 1; B.reserved = 0; B.bonds = bB; B.cores = coresB;
  CHECK(ttm_output_capacity(&A, &B, &opt) > 0);
  bA[0] = 2; /* boundary bond must be 1 */
  CHECK(ttm_output_capacity(&A, &B, &opt) < 0);

  if (failures == 0) printf("c abi check ok\n");
  return failures == 0 ? 0 : 1;
}

/* Plain C99 user of include/ttm.h: compiles against the header alone, links against
 * libttm.so, and exercises the calls that need no GPU (version, argument and option
 * validation, host-side output planning). */
#include <stddef.h>
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
  opt.prec = (ttm_precision)1; /* not a precision mode */
  CHECK(ttm_create(&h, 0, NULL, &opt) == TTM_ERR_INVALID_ARG);
  opt.prec = TTM_PREC_BF16_SPLIT;
  opt.split_digits = 9;
  CHECK(ttm_create(&h, 0, NULL, &opt) == TTM_ERR_INVALID_ARG);
  opt.split_digits = 0;
  opt.prec = TTM_PREC_FP64;
  opt.jacobi_kernel = 5;
  CHECK(ttm_create(&h, 0, NULL, &opt) == TTM_ERR_INVALID_ARG);
  opt.jacobi_kernel = 0;

  /* host-side planning: a two-site product of bond-2 trains */
  A.L = 2; A.d = 2; A.on_host = 1; A.reserved = 0; A.bonds = bA; A.cores = coresA;
  B.L = 2; B.d = 2; B.on_host = 1; B.reserved = 0; B.bonds = bB; B.cores = coresB;
  CHECK(ttm_output_capacity(&A, &B, &opt) > 0);
  bA[0] = 2; /* boundary bond must be 1 */
  CHECK(ttm_output_capacity(&A, &B, &opt) < 0);

  /* struct layout, compared with the ctypes mirror by the Python test */
#define FIELD(T, f) printf("layout %s.%s %zu %zu\n", #T, #f, offsetof(T, f), sizeof(((T *)0)->f))
  printf("layout ttm_tt.sizeof 0 %zu\n", sizeof(ttm_tt));
  FIELD(ttm_tt, L); FIELD(ttm_tt, d); FIELD(ttm_tt, on_host); FIELD(ttm_tt, reserved);
  FIELD(ttm_tt, bonds); FIELD(ttm_tt, cores);
  printf("layout ttm_options.sizeof 0 %zu\n", sizeof(ttm_options));
  FIELD(ttm_options, prec); FIELD(ttm_options, eps); FIELD(ttm_options, chi_max);
  FIELD(ttm_options, chi_out); FIELD(ttm_options, max_sweeps); FIELD(ttm_options, use_graph);
  FIELD(ttm_options, check_finite); FIELD(ttm_options, profile_kernels);
  FIELD(ttm_options, f32_passes); FIELD(ttm_options, jacobi_kernel);
  FIELD(ttm_options, newton_steps); FIELD(ttm_options, split_digits);
  FIELD(ttm_options, reserved1); FIELD(ttm_options, env_budget_bytes);
  printf("layout ttm_report.sizeof 0 %zu\n", sizeof(ttm_report));
  FIELD(ttm_report, status); FIELD(ttm_report, jacobi_sweeps_max); FIELD(ttm_report, max_bond);
  FIELD(ttm_report, n_swaps); FIELD(ttm_report, n_contracts); FIELD(ttm_report, n_qr);
  FIELD(ttm_report, discarded_weight); FIELD(ttm_report, err_bound); FIELD(ttm_report, norm_out);
  FIELD(ttm_report, flops_counted); FIELD(ttm_report, seconds); FIELD(ttm_report, peak_workspace_bytes);
  FIELD(ttm_report, bond_trace); FIELD(ttm_report, bond_trace_len); FIELD(ttm_report, n_kernel_launches);
  FIELD(ttm_report, jacobi_launches); FIELD(ttm_report, gemm_ms); FIELD(ttm_report, newton_residual);
  FIELD(ttm_report, jacobi32_ms); FIELD(ttm_report, jacobi32_flops); FIELD(ttm_report, n_nonconverged);
  FIELD(ttm_report, n_frozen_pairs); FIELD(ttm_report, gemm_flops); FIELD(ttm_report, gemm_launches);
  FIELD(ttm_report, qr_ms); FIELD(ttm_report, n_fallback);
  FIELD(ttm_report, jacobi32_sweeps); FIELD(ttm_report, svd_trace); FIELD(ttm_report, svd_trace_len);
  FIELD(ttm_report, jacobi64_ms);
#undef FIELD

  if (failures == 0) printf("c abi check ok\n");
  return failures == 0 ? 0 : 1;
}

/* Host-only use of the C ABI from C: struct layouts (compared with the
 * Python binding's mirrors), a plan's matrix and program statistics, the
 * interpreter stream's self-check, and argument errors.  No GPU call. */
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "xorec.h"

#define SIZE(T) printf("sizeof %s %zu\n", #T, sizeof(T))
#define OFF(T, f) printf("offsetof %s.%s %zu\n", #T, #f, offsetof(T, f))

int main(void) {
  SIZE(ec_plan_opts);
  OFF(ec_plan_opts, stream_temps);
  SIZE(ec_slp_stats);
  SIZE(ec_program_info);
  OFF(ec_program_info, lop3);
  OFF(ec_program_info, window_temps);
  SIZE(ec_tune_result);
  SIZE(ec_job);
  SIZE(ec_batch_info);
  SIZE(ec_server_opts);
  SIZE(ec_server_stats);

  ec_plan *plan = NULL;
  if (ec_plan_create(10, 4, NULL, &plan) != EC_OK) {
    printf("error %s\n", ec_last_error());
    return 1;
  }
  uint8_t P[40];
  if (ec_plan_matrix(plan, P) != EC_OK) return 2;
  printf("matrix");
  for (int i = 0; i < 40; ++i) printf(" %d", P[i]);
  printf("\n");

  ec_program_info info;
  if (ec_plan_info(plan, NULL, 0, &info) != EC_OK) return 3;
  printf("encoder n_in %d n_out %d raw_xors %ld fused_xors %ld lop3 %d loads %d\n", info.n_in,
         info.n_out, info.raw.xors, info.fused.xors, info.lop3, info.loads);
  int er[4] = {11, 2, 5, 0};
  if (ec_plan_info(plan, er, 4, &info) != EC_OK) return 4;
  printf("decoder n_in %d n_out %d raw_xors %ld\n", info.n_in, info.n_out, info.raw.xors);

  size_t need = 0;
  if (ec_plan_program(plan, NULL, 0, NULL, 0, &need) != EC_OK || need == 0) return 5;
  uint16_t *code = (uint16_t *)malloc(need * sizeof(uint16_t));
  if (!code || ec_plan_program(plan, NULL, 0, code, need, NULL) != EC_OK) return 6;
  if (ec_plan_info(plan, NULL, 0, &info) != EC_OK) return 7;
  printf("program_check %d\n", (int)ec_program_check(code, need, info.n_in, info.n_out, info.slots));
  free(code);
  ec_plan_destroy(plan);

  /* argument errors are returned, with a message */
  ec_plan *bad = NULL;
  const ec_status s = ec_plan_create(0, 4, NULL, &bad);
  printf("bad_k %d %s\n", (int)s, bad == NULL && ec_last_error()[0] ? "message" : "none");
  int dup[2] = {3, 3};
  ec_plan_create(4, 2, NULL, &plan);
  printf("dup_erasure %d\n", (int)ec_plan_info(plan, dup, 2, &info));
  ec_plan_destroy(plan);
  return 0;
}

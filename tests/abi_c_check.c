/* Plain C99 consumer of the C ABI (include/hz.h): compiled with gcc and linked
 * against libhz.so by tests/test_abi_c.py.  It uses only calls that need no
 * device and checks their results and error behaviour; prints "ok" and
 * returns 0 when every check holds. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "hz.h"

#define CHECK(c)                                                         \
  do {                                                                   \
    if (!(c)) {                                                          \
      printf("failed: %s (line %d): %s\n", #c, __LINE__, hz_last_error()); \
      return 1;                                                          \
    }                                                                    \
  } while (0)

int main(void) {
  CHECK(hz_abi_version() == HZ_ABI_VERSION);
  CHECK(strlen(hz_status_string(HZ_ERR_INVALID_ARG)) > 0);

  hz_opts o;
  CHECK(hz_opts_default(2, &o) == HZ_OK);
  CHECK(o.levels == 4 && o.restart_m == 5 && o.cycle_visits == 1 && o.nrhs_max == 1);
  CHECK(hz_opts_default(4, &o) == HZ_ERR_INVALID_ARG);

  hz_grid g;
  memset(&g, 0, sizeof g);
  g.dim = 2;
  g.n[0] = 129;
  g.n[1] = 129;
  g.n[2] = 1;
  g.h = 1.0 / 128;
  hz_opts_default(2, &o);
  size_t bytes = 0;
  CHECK(hz_setup_bytes(&g, &o, &bytes) == HZ_OK && bytes > (size_t)129 * 129 * 16);
  o.restart_m = 129;
  CHECK(hz_setup_bytes(&g, &o, &bytes) == HZ_ERR_INVALID_ARG);
  o.restart_m = 40;
  o.nrhs_max = 4;
  CHECK(hz_setup_bytes(&g, &o, &bytes) == HZ_ERR_INVALID_ARG);   /* long restarts: one RHS only */

  /* Table relaxParam: 2D RB fine level */
  CHECK(fabs(hz_default_damping(2, HZ_PATCH_RB, 0) - 0.83) < 1e-12);
  CHECK(isnan(hz_default_damping(5, HZ_PATCH_RB, 0)));

  /* argument checks come before any device work */
  double st[9] = {0}, w = 0.8, mu, rho;
  CHECK(hz_lfa_factors(2, st, HZ_PATCH_PLUS, &w, 0, HZ_IG_CUBIC, HZ_IG_CUBIC, 1, 1, 16, &mu, &rho) ==
        HZ_ERR_INVALID_ARG);
  CHECK(hz_lfa_factors(2, st, HZ_PATCH_PLUS, &w, 1, HZ_IG_MIXED, HZ_IG_CUBIC, 1, 1, 16, &mu, &rho) ==
        HZ_ERR_INVALID_ARG);
  CHECK(hz_solve_history(NULL, 0, NULL, NULL, NULL, NULL) == HZ_ERR_INVALID_ARG);
  printf("ok\n");
  return 0;
}

/* Plain C99 client of libwave's C ABI (no C++, no torch): exercises the
 * host-side entry points that need no GPU.  Exit status 0 when every check
 * holds; each failing check prints its line. */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "wave.h"

static int failures = 0;
#define CHECK(c)                                          \
  do {                                                    \
    if (!(c)) {                                           \
      fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
      ++failures;                                         \
    }                                                     \
  } while (0)

int main(void) {
  /* status strings */
  CHECK(strcmp(wave_status_string(WAVE_OK), "ok") == 0);
  CHECK(strlen(wave_status_string(WAVE_EUNSTABLE)) > 0);
  /* stability bound: 2D, order 2, h = 10 m, vmax = 3000 m/s, half the limit */
  const double dt = wave_cfl_dt(2, 2, 10.0, 3000.0, 0.5);
  CHECK(fabs(dt - 0.5 * 10.0 / (3000.0 * sqrt(2.0))) < 1e-15);
  /* workspace size of a pitched 3D model (rows rounded up to 128 cells) */
  wave_grid_desc d;
  memset(&d, 0, sizeof(d));
  d.ndim = 3;
  d.order = 8;
  d.n[0] = 130;
  d.n[1] = 10;
  d.n[2] = 11;
  d.h = 10.0;
  d.dt = wave_cfl_dt(3, 8, 10.0, 4500.0, 0.5);
  d.physics = WAVE_VELOCITY;
  d.bc = WAVE_DIRICHLET;
  d.storage = WAVE_F32;
  size_t bytes = 0;
  CHECK(wave_model_workspace_size(&d, &bytes) == WAVE_OK);
  CHECK(bytes >= (size_t)256 * 10 * 11 * 4);
  /* invalid descriptors are rejected on the host */
  d.order = 3;
  CHECK(wave_model_workspace_size(&d, &bytes) == WAVE_EINVAL);
  d.order = 8;
  d.n[0] = 8; /* fewer than order + 1 cells */
  CHECK(wave_model_workspace_size(&d, &bytes) == WAVE_EINVAL);
  /* a null parameter grid is rejected before any device work */
  d.n[0] = 130;
  wave_model m = NULL;
  CHECK(wave_model_create(&d, NULL, NULL, 0, NULL, &m) == WAVE_EINVAL);
  /* the static-scratch misfit rejects sizes beyond its limit on the host */
  double out = 0.0;
  CHECK(wave_misfit_static(NULL, NULL, (int64_t)1 << 40, 1.0, 1.0, &out, NULL) != WAVE_OK);
  /* tuning setters reject a missing model */
  CHECK(wave_model_set_schedule(NULL, 1) == WAVE_EINVAL);
  CHECK(wave_model_set_tiling(NULL, 32, 16, 2, 4) == WAVE_EINVAL);
  if (failures == 0) printf("c abi host checks: ok\n");
  return failures == 0 ? 0 : 1;
}

/* A plain C99 caller of libpoba through include/poba.h alone: the paths that run on the host
 * before any CUDA call (defaults, status strings, argument validation).  Prints one line per
 * check and exits non-zero on the first failure. */
#include <stdio.h>
#include <string.h>

#include "poba.h"

static int fails = 0;

static void check(int ok, const char* what) {
  printf("%s %s\n", ok ? "ok  " : "FAIL", what);
  if (!ok) fails++;
}

int main(void) {
  ba_options o;
  check(ba_default_options(&o) == BA_OK, "ba_default_options");
  check(o.lambda0 == 1e-4 && o.func_tol == 1e-6 && o.eps == 0.01 && o.max_lm == 50 &&
            o.max_inner == 20 && o.damping_mode == 0 && o.series_exec == 2,
        "defaults of Sec. 5.1");
  check(ba_default_options(NULL) == BA_ERR_INVALID_ARG, "ba_default_options(NULL)");

  check(strcmp(ba_status_string(BA_OK), "BA_OK") == 0, "status string BA_OK");
  check(strcmp(ba_status_string(BA_ERR_TIMEOUT), "BA_ERR_TIMEOUT") == 0,
        "status string BA_ERR_TIMEOUT");

  /* a 2-camera, 2-landmark problem whose last observation names camera 2 (out of range) */
  double cams[2 * 9] = {0};
  double lms[2 * 3] = {0, 0, -5, 1, 0, -5};
  double obs[3 * 2] = {0};
  int32_t cam_idx[3] = {0, 1, 2};
  int32_t lm_idx[3] = {0, 1, 1};
  cams[6] = cams[15] = 500.0;
  ba_problem_desc d;
  memset(&d, 0, sizeof d);
  d.n_cams = 2;
  d.n_lms = 2;
  d.n_obs = 3;
  d.cams = cams;
  d.lms = lms;
  d.obs = obs;
  d.cam_idx = cam_idx;
  d.lm_idx = lm_idx;
  d.ptr_kind = 0;
  d.precision = BA_FP64;
  ba_handle* h = (ba_handle*)&d; /* must be overwritten with NULL on error */
  check(ba_create(&d, &o, &h) == BA_ERR_INVALID_ARG, "ba_create rejects an out-of-range index");
  check(h == NULL, "ba_create leaves *out NULL on error");
  check(strstr(ba_last_error(), "cam_idx[2]") != NULL, "ba_last_error names the index");
  check(ba_create(NULL, &o, &h) == BA_ERR_INVALID_ARG, "ba_create(NULL desc)");

  ba_options bad = o;
  bad.eps = -1.0;
  cam_idx[2] = 1;
  check(ba_create(&d, &bad, &h) == BA_ERR_INVALID_ARG, "ba_create rejects eps < 0");

  double cost = 0.0;
  check(ba_cost_noalloc(BA_NOALLOC_MAX_CAMS + 1, 1, 0, cams, lms, obs, cam_idx, lm_idx, NULL,
                        &cost, NULL) == BA_ERR_INVALID_ARG,
        "ba_cost_noalloc rejects more cameras than its scratch holds");
  check(ba_destroy(NULL) == BA_OK, "ba_destroy(NULL)");
  check(ba_linearize(NULL, NULL) == BA_ERR_INVALID_ARG, "ba_linearize(NULL handle)");

  printf("%d failure(s)\n", fails);
  return fails ? 1 : 0;
}

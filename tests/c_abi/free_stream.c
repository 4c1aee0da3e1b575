/* A plain C99 client of libaf (include/af.h only, no CUDA headers): a uniform
 * state on a ragged 37 x 29 outflow grid is stepped five times through host
 * buffers and must stay uniform (free-stream preservation) to 1e-13.
 * Exit codes: 0 pass, 1 failure, 77 no CUDA device (af_create reports AF_ECUDA). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "af.h"

int main(void) {
  const int nx = 37, ny = 29;
  const double prim[8] = {1.3, 0.4, -0.2, 0.1, 0.7, -0.5, 0.3, 2.0}; /* rho, v, B, p */
  const double gamma = 5.0 / 3.0;
  double cons[8];
  cons[0] = prim[0];
  for (int k = 1; k < 4; ++k) cons[k] = prim[0] * prim[k];
  for (int k = 4; k < 7; ++k) cons[k] = prim[k];
  cons[7] = prim[7] / (gamma - 1.0) +
            0.5 * prim[0] * (prim[1] * prim[1] + prim[2] * prim[2] + prim[3] * prim[3]) +
            0.5 * (prim[4] * prim[4] + prim[5] * prim[5] + prim[6] * prim[6]);
  af_ctx *ctx = NULL;
  int rc = af_create(nx, ny, gamma, AF_BC_OUTFLOW, &ctx);
  if (rc == AF_ECUDA) {
    printf("no CUDA device\n");
    return 77;
  }
  if (rc != AF_OK) return 1;
  if (af_set_domain(ctx, -1.0, 1.0, 0.0, 1.5) != AF_OK) return 1;
  double *U[4];
  size_t len[4];
  for (int c = 0; c < 4; ++c) {
    int nxp = 0, nyp = 0;
    if (af_sizes(ctx, c, &nxp, &nyp) != AF_OK) return 1;
    len[c] = (size_t)nxp * nyp;
    U[c] = (double *)malloc(sizeof(double) * 8 * len[c]);
    for (int k = 0; k < 8; ++k)
      for (size_t q = 0; q < len[c]; ++q) U[c][k * len[c] + q] = cons[k];
  }
  rc = af_set_state(ctx, (const double *const *)U, 0);
  double t = 0.0;
  for (int s = 0; s < 5 && rc == AF_OK; ++s) {
    double dt = 0.0;
    rc = af_step(ctx, &dt, 0);
    t += dt;
  }
  if (rc == AF_OK) rc = af_get_state(ctx, U, 0);
  long long cnt[AF_NSTAT];
  if (rc == AF_OK) rc = af_status(ctx, cnt, 0);
  if (rc != AF_OK) {
    printf("libaf error %d: %s\n", rc, af_last_error(ctx));
    return 1;
  }
  double worst = 0.0;
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < 8; ++k)
      for (size_t q = 0; q < len[c]; ++q) {
        const double e = fabs(U[c][k * len[c] + q] - cons[k]) / (fabs(cons[k]) + 1.0);
        if (e > worst) worst = e;
      }
  printf("t = %.6e, max relative deviation %.3e, points limited %lld\n", t, worst, cnt[AF_STAT_POINT_LIMITED]);
  af_destroy(ctx);
  for (int c = 0; c < 4; ++c) free(U[c]);
  return (worst <= 1e-13 && t > 0.0) ? 0 : 1;
}

/* A C program that uses the library through include/pat.h alone (no Python):
 * a plan whose library is generated on the device from a homogeneous medium
 * (Eq. 1-2), H (Eq. 7-8) and H* (Eq. 11) on host arrays, and the adjoint
 * identity <H x, y> = <x, H* y> (Eq. 9) checked in double precision; plus the
 * host-only queries of the folded layout. With the argument --layout only the
 * host-only queries run (no device needed). Exit status 0 = pass. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "pat.h"

/* splitmix64 (Steele, Lea and Flood, OOPSLA 2014): uniform doubles in [0, 1) */
static uint64_t state = 12345;
static double uniform01(void) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static int host_queries(void) {
  int64_t nrb = 0, nch = 0;
  if (pat_fold_blocks(256, 1, &nrb, &nch, NULL, NULL, NULL, NULL) != PAT_OK) {
    fprintf(stderr, "pat_fold_blocks: %s\n", pat_last_error());
    return 1;
  }
  if (nch != 189 || nrb != 277) {
    fprintf(stderr, "radial layout of 256 x 256: %lld chunks, %lld blocks\n", (long long)nch,
            (long long)nrb);
    return 1;
  }
  pat_geometry g = {128, 128, 64, 256, 256, 256, 1, 0};
  int64_t tb = 0, ws = 0;
  if (pat_plan_estimate(&g, 3, &tb, &ws) != PAT_OK || tb != 396361728 || ws <= 0) {
    fprintf(stderr, "pat_plan_estimate: %lld table bytes (%s)\n", (long long)tb,
            pat_last_error());
    return 1;
  }
  if (pat_fold_blocks(7, 1, &nrb, &nch, NULL, NULL, NULL, NULL) != PAT_ERR_ARG) {
    fprintf(stderr, "pat_fold_blocks accepted an odd length\n");
    return 1;
  }
  return 0;
}

int main(int argc, char** argv) {
  if (host_queries() != 0) return 1;
  if (argc > 1) {
    printf("host queries ok\n");
    return 0;
  }
  /* 32^2 -> 64^2, 16 depths, 64 samples, 100 um voxels, 20 ns sampling */
  pat_geometry g = {32, 32, 16, 64, 64, 64, 1, 0};
  pat_medium m = {1500.0, 1e-4, 1e-4, 1e-4, 2e-8, 64, 1};
  pat_plan* plan = NULL;
  if (pat_plan_create_kspace(&g, &m, NULL, &plan) != PAT_OK) {
    fprintf(stderr, "pat_plan_create_kspace: %s\n", pat_last_error());
    return 1;
  }
  pat_plan_info_t info;
  if (pat_plan_info(plan, &info) != PAT_OK || !info.folded || !info.radial || !info.real_table) {
    fprintf(stderr, "plan info: folded %d radial %d real %d\n", info.folded, info.radial,
            info.real_table);
    return 1;
  }
  const size_t nobj = (size_t)g.nz * g.ny * g.nx, ndat = (size_t)g.nt * g.ny * g.nx;
  float* x = malloc(nobj * sizeof(float));
  float* z = malloc(nobj * sizeof(float));
  float* y = malloc(ndat * sizeof(float));
  float* d = malloc(ndat * sizeof(float));
  if (!x || !z || !y || !d) return 1;
  for (size_t i = 0; i < nobj; ++i) x[i] = (float)uniform01();
  for (size_t i = 0; i < ndat; ++i) y[i] = (float)(2.0 * uniform01() - 1.0);
  /* host pointers: the library stages them and returns with the result on the host */
  if (pat_forward(plan, x, d, 1, NULL) != PAT_OK || pat_adjoint(plan, y, z, 1, NULL) != PAT_OK) {
    fprintf(stderr, "operator call: %s\n", pat_last_error());
    return 1;
  }
  double hxy = 0, xhy = 0, nd = 0, ny = 0;
  for (size_t i = 0; i < ndat; ++i) {
    hxy += (double)d[i] * y[i];
    nd += (double)d[i] * d[i];
    ny += (double)y[i] * y[i];
  }
  for (size_t i = 0; i < nobj; ++i) xhy += (double)x[i] * z[i];
  const double rel = fabs(hxy - xhy) / (sqrt(nd) * sqrt(ny));
  printf("<Hx, y> = %.9e  <x, H*y> = %.9e  relative gap %.2e\n", hxy, xhy, rel);
  pat_plan_destroy(plan);
  free(x);
  free(z);
  free(y);
  free(d);
  if (!(nd > 0) || rel > 1e-6) return 1;
  return 0;
}

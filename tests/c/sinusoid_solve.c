/* A plain C caller of the library: the 64^3 periodic sinusoid
 * rho = sin 2 pi x sin 2 pi y sin 2 pi z (Sec. 4.1), solved in mixed precision
 * from device arrays (mg_solve) and from host arrays (mg_solve_host).  The
 * discrete solution is exact: phi = rho h^2 / (-4 (3 sin^2(pi h))) for the
 * 7-point operator.  Exit status 0 when both agree with it to 1e-9. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "mg.h"

static int fail(const char *what, mg_status st, const mg_ctx *c) {
  fprintf(stderr, "%s: %s (%s)\n", what, mg_status_str(st), mg_last_error(c));
  return 1;
}

int main(void) {
  const int n = 64;
  const size_t N = (size_t)n * n * n;
  const double pi = 3.14159265358979323846, h = 1.0 / n;
  double *rho = malloc(N * sizeof(double)), *phi = malloc(N * sizeof(double));
  double *want = malloc(N * sizeof(double));
  if (!rho || !phi || !want) return 1;
  const double amp = h * h / (-12.0 * sin(pi * h) * sin(pi * h));
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const size_t t = ((size_t)k * n + j) * n + i;
        rho[t] = sin(2 * pi * (i + 0.5) * h) * sin(2 * pi * (j + 0.5) * h) *
                 sin(2 * pi * (k + 0.5) * h);
        want[t] = amp * rho[t];
      }
  mg_opts o;
  mg_opts_init(&o);
  o.prec = MG_MIXED;
  mg_ctx *c = NULL;
  mg_status st = mg_create(n, n, n, h, MG_BC_PERIODIC, &o, &c);
  if (st != MG_OK) return fail("mg_create", st, NULL);
  double *rho_d = NULL, *phi_d = NULL;
  if (cudaMalloc((void **)&rho_d, N * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&phi_d, N * sizeof(double)) != cudaSuccess)
    return 1;
  cudaMemcpy(rho_d, rho, N * sizeof(double), cudaMemcpyHostToDevice);
  double hist[64];
  int nh = 0;
  st = mg_solve(c, rho_d, 1.0, 1e-10, phi_d, hist, 64, &nh, NULL);
  if (st != MG_OK) return fail("mg_solve", st, c);
  cudaMemcpy(phi, phi_d, N * sizeof(double), cudaMemcpyDeviceToHost);
  double err = 0.0, mx = 0.0;
  for (size_t t = 0; t < N; ++t) {
    err = fmax(err, fabs(phi[t] - want[t]));
    mx = fmax(mx, fabs(want[t]));
  }
  printf("device: %d outer iterations, ||d||/||f|| = %.3e, error %.3e\n", nh, hist[nh - 1],
         err / mx);
  if (!(err / mx <= 1e-9)) return 1;
  for (size_t t = 0; t < N; ++t) phi[t] = 0.0;
  st = mg_solve_host(c, rho, 1.0, 1e-10, phi, hist, 64, &nh, NULL);
  if (st != MG_OK) return fail("mg_solve_host", st, c);
  err = 0.0;
  for (size_t t = 0; t < N; ++t) err = fmax(err, fabs(phi[t] - want[t]));
  printf("host: %d outer iterations, error %.3e\n", nh, err / mx);
  if (!(err / mx <= 1e-9)) return 1;
  mg_destroy(c);
  cudaFree(rho_d);
  cudaFree(phi_d);
  free(rho);
  free(phi);
  free(want);
  printf("C caller checks passed\n");
  return 0;
}

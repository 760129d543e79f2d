/* A static droplet through the C ABI alone (no Python, no PyTorch): 32^3 periodic box,
 * R = 8, D = 4, sigma = 0.01, rho 3:1, nu = 0.1, Mob = 0.1 (the droplet setup of
 * Sec. III).  Uses the library's own allocator (cudaMalloc) and the default stream.
 * Prints one line "steps=<n> sum_phi=<s0> -> <s1> max_phi=<m> mu_min=<x>" and exits 0
 * when sum phi is conserved to 1e-6 of sum |phi|, every field is finite and the state
 * read at a few listed cells (lbm_read_state_at) equals the whole state read there;
 * 1 if a check fails; 2 if a call fails (its status and message are printed). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "lbm.h"

#define N 32

static int check(lbm_ctx* ctx, lbm_status st, const char* what) {
  if (st == LBM_OK) return 0;
  fprintf(stderr, "%s failed: status %d: %s\n", what, (int)st, lbm_last_error(ctx));
  return 1;
}

int main(void) {
  const size_t n = (size_t)N * N * N;
  lbm_grid grid = {N, N, N, 0};
  lbm_params p = {0};
  p.rho_l = 3.0;
  p.rho_g = 1.0;
  p.nu_l = p.nu_g = 0.1;
  p.mobility = 0.1;
  p.D = 4.0;
  p.sigma = 0.01;
  p.A = 0.25;
  const double sf[7] = {1.0, 1.25, 1.25, 1.25, 1.2, 1.0, 1.0}; /* Eq. 45 */
  for (int i = 0; i < 7; ++i) p.sf[i] = sf[i];
  for (int i = 0; i < 15; ++i) p.sg[i] = 1.0;
  p.storage = LBM_STORAGE_FP32;
  p.pattern = LBM_PATTERN_AB;

  double* phi0 = malloc(n * sizeof(double));
  double* phi = malloc(n * sizeof(double));
  double* mu = malloc(n * sizeof(double));
  if (!phi0 || !phi || !mu) return 2;
  double sum0 = 0.0, abs0 = 0.0;
  for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        const double r = sqrt((x - N / 2.0) * (x - N / 2.0) + (y - N / 2.0) * (y - N / 2.0) +
                              (z - N / 2.0) * (z - N / 2.0));
        const double v = tanh(2.0 * (8.0 - r) / p.D);
        phi0[((size_t)z * N + y) * N + x] = v;
        sum0 += v;
        abs0 += fabs(v);
      }

  lbm_ctx* ctx = NULL;
  if (check(NULL, lbm_create(&grid, &p, NULL, NULL, &ctx), "lbm_create")) return 2;
  if (check(ctx, lbm_init_phi(ctx, phi0, NULL, NULL), "lbm_init_phi")) return 2;
  double s0, m0[3], s1, m1[3];
  if (check(ctx, lbm_reduce(ctx, &s0, m0), "lbm_reduce")) return 2;
  const int steps = 200;
  if (check(ctx, lbm_step(ctx, steps - 1), "lbm_step")) return 2;
  if (check(ctx, lbm_step_reduce(ctx, 1, &s1, m1), "lbm_step_reduce")) return 2;
  if (check(ctx, lbm_read_fields(ctx, LBM_FIELD_PHI | LBM_FIELD_MU, phi, NULL, NULL, NULL, mu),
            "lbm_read_fields"))
    return 2;
  long long t = -1;
  lbm_get_step(ctx, &t);
  /* the state at four listed cells against the whole state */
  float* fs = malloc(7 * n * sizeof(float));
  float* gs = malloc(15 * n * sizeof(float));
  if (!fs || !gs) return 2;
  const long long cells[4] = {0, (long long)n - 1, 12345, 12345};
  float fa[7 * 4], ga[15 * 4];
  long long ta = -1;
  if (check(ctx, lbm_read_state(ctx, fs, gs, NULL, NULL), "lbm_read_state")) return 2;
  if (check(ctx, lbm_read_state_at(ctx, cells, 4, fa, ga, NULL, &ta), "lbm_read_state_at"))
    return 2;
  int same = ta == t;
  for (int k = 0; k < 4; ++k) {
    for (int i = 0; i < 7; ++i) same = same && fa[i * 4 + k] == fs[(size_t)i * n + cells[k]];
    for (int i = 0; i < 15; ++i) same = same && ga[i * 4 + k] == gs[(size_t)i * n + cells[k]];
  }
  free(fs);
  free(gs);
  if (check(ctx, lbm_destroy(ctx), "lbm_destroy")) return 2;

  double maxphi = -1e30, minmu = 1e30;
  int finite = 1;
  for (size_t i = 0; i < n; ++i) {
    if (!isfinite(phi[i]) || !isfinite(mu[i])) finite = 0;
    if (phi[i] > maxphi) maxphi = phi[i];
    if (mu[i] < minmu) minmu = mu[i];
  }
  printf("steps=%lld sum_phi=%.9f -> %.9f max_phi=%.6f mu_min=%.6e\n", t, s0, s1, maxphi,
         minmu);
  free(phi0);
  free(phi);
  free(mu);
  const int ok = finite && same && t == steps && fabs(s1 - s0) <= 1e-6 * abs0 &&
                 fabs(s0 - sum0) <= 1e-5 * abs0 && maxphi > 0.9 && maxphi < 1.05;
  return ok ? 0 : 1;
}

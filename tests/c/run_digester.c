/* A plain C caller of the library: one digester without flow, read from a
   binary input file, integrated, written back.  Used by the tests to check
   that chad.h compiles as C99 and that a C program drives the library to the
   same result as the Python binding.

   Input (little-endian): int64 n, int64 n_intervals, double dt_s, double
   V_liq, double V_gas, double D_uniform, double rtol, double params[113],
   double atol[29], double y_in[29], double y[29][n], double T[n].
   Output: double y[29][n], double S_H[n], double h[n], int32 status[n]. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "chad.h"

static int rd(FILE* f, void* p, size_t size, size_t count) {
  return fread(p, size, count, f) == count;
}

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s input output\n", argv[0]);
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t n = 0, k = 0;
  double dt = 0, vl = 0, vg = 0, du = 0, rtol = 0;
  double params[CHAD_NPARAM], atol[29], y_in[29];
  int ok = rd(f, &n, 8, 1) && rd(f, &k, 8, 1) && rd(f, &dt, 8, 1) && rd(f, &vl, 8, 1) &&
           rd(f, &vg, 8, 1) && rd(f, &du, 8, 1) && rd(f, &rtol, 8, 1) &&
           rd(f, params, 8, CHAD_NPARAM) && rd(f, atol, 8, 29) && rd(f, y_in, 8, 29);
  if (!ok || n < 0) return 2;
  double* y = malloc(sizeof(double) * 29 * (size_t)n + 8);
  double* T = malloc(sizeof(double) * (size_t)n + 8);
  double* sh = malloc(sizeof(double) * (size_t)n + 8);
  double* h = malloc(sizeof(double) * (size_t)n + 8);
  int32_t* st = malloc(sizeof(int32_t) * (size_t)n + 8);
  if (!y || !T || !sh || !h || !st) return 2;
  ok = rd(f, y, 8, 29 * (size_t)n) && rd(f, T, 8, (size_t)n);
  fclose(f);
  if (!ok) return 2;

  chad_config cfg = {0};
  cfg.n_digesters = 1;
  cfg.n_particles = &n;
  cfg.V_liq = &vl;
  cfg.V_gas = &vg;
  cfg.params = params;
  cfg.D_uniform = &du;
  cfg.y_in = y_in;
  cfg.precision = CHAD_PREC_FP64;
  cfg.learned = 0;
  cfg.headspace = CHAD_HEADSPACE_PARTICLE;
  cfg.rtol = rtol;
  cfg.atol = atol;
  cfg.max_steps_per_interval = 100000;
  cfg.max_newton_iters = 50;
  cfg.fixed_substeps = 0;
  cfg.cuda_stream = NULL;
  cfg.h2_algebraic = 0;

  chad_ctx* ctx = NULL;
  chad_status s = chad_create(&cfg, &ctx);
  if (s != CHAD_OK) {
    fprintf(stderr, "chad_create: %d\n", (int)s);
    return 1;
  }
  s = chad_load_particles(ctx, 0, n, NULL, y, T, NULL, NULL, CHAD_MEM_HOST);
  if (s == CHAD_OK) s = chad_step(ctx, dt, (int)k);
  chad_stats stats;
  if (s == CHAD_OK) s = chad_read_states(ctx, 0, y, NULL, sh, h, st, &stats, CHAD_MEM_HOST);
  if (s != CHAD_OK && s != CHAD_E_PARTICLE) {
    fprintf(stderr, "chad: %d %s\n", (int)s, chad_last_error(ctx));
    chad_destroy(ctx);
    return 1;
  }
  chad_destroy(ctx);
  FILE* o = fopen(argv[2], "wb");
  if (!o) return 2;
  fwrite(y, 8, 29 * (size_t)n, o);
  fwrite(sh, 8, (size_t)n, o);
  fwrite(h, 8, (size_t)n, o);
  fwrite(st, 4, (size_t)n, o);
  fclose(o);
  printf("accepted %lld rejected %lld\n", (long long)stats.accepted_steps,
         (long long)stats.rejected_steps);
  return 0;
}

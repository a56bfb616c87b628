/* Sanitizer harness of the FP64 oracle (test infrastructure).  Built by
 * tests/test_oracle_sanitize.py with AddressSanitizer and
 * UndefinedBehaviorSanitizer (fatal on the first finding); it drives every
 * oracle routine on small inputs, including the edge cases the tests use
 * (both sample formats, half-bit sets, code-Doppler sums, several threads,
 * refinement with a Doppler pre-search, tracking), so that an out-of-bounds
 * access, a use after free, a signed overflow or a misaligned load anywhere in
 * them stops the run.  It checks a few results too (FFT round trip, FFT
 * correlation against the direct sum). */
#include "oracle.c"

#include <stdio.h>

#define FS 256000
#define N 256

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static double urand(void) { /* xorshift64*, uniform in [0, 1) */
  rng_state ^= rng_state >> 12;
  rng_state ^= rng_state << 25;
  rng_state ^= rng_state >> 27;
  return (double)((rng_state * 2685821657736338717ull) >> 11) * (1.0 / 9007199254740992.0);
}

int main(void) {
  const int coh = 2, nblocks = 3;
  const int64_t n = (int64_t)coh * N * nblocks + 37; /* a ragged tail */
  int8_t chips[32][ORC_CHIPS];
  for (int p = 1; p <= 32; ++p)
    if (orc_ca_code(p, chips[p - 1]) != 0) return 10;
  if (orc_ca_code(0, chips[0]) == 0 || orc_ca_code(33, chips[0]) == 0) return 11;

  /* recordings in both formats, unpacked */
  uint8_t *raw8 = malloc(2 * n), *raw2 = malloc((n + 1) / 2);
  for (int64_t k = 0; k < 2 * n; ++k) raw8[k] = (uint8_t)(urand() * 256.0);
  for (int64_t k = 0; k < (n + 1) / 2; ++k) raw2[k] = (uint8_t)(urand() * 256.0);
  double *xr = malloc(sizeof(double) * n), *xi = malloc(sizeof(double) * n);
  if (orc_unpack(raw2, n, 1, xr, xi) != 0) return 12;
  if (orc_unpack(raw8, n, 0, xr, xi) != 0) return 13;

  /* replica, fold, FFT / DFT round trip */
  double rep[N], yr[N], yi[N], dr[N], di[N];
  orc_replica(chips[4], N, rep);
  orc_wipe_fold(xr, xi, FS, N, coh, -1750, 1, yr, yi);
  orc_dft(yr, yi, N, 0, dr, di);
  double fr[N], fi[N];
  memcpy(fr, yr, sizeof fr);
  memcpy(fi, yi, sizeof fi);
  if (orc_fft(fr, fi, N, 0) != 0) return 14;
  double err = 0, mag = 0;
  for (int k = 0; k < N; ++k) {
    err = fmax(err, fabs(fr[k] - dr[k]) + fabs(fi[k] - di[k]));
    mag = fmax(mag, fabs(dr[k]) + fabs(di[k]));
  }
  if (err > 1e-9 * mag) return 15;
  if (orc_fft(fr, fi, N, 1) != 0) return 16;
  if (orc_fft(fr, fi, 3, 0) == 0) return 17; /* not a power of two */

  /* FFT correlation against the direct sum */
  double Rr[N], Ri[N], Qr[N], Qi[N];
  orc_corr_direct(xr, xi, FS, N, coh, 1250, 2, chips[9], Rr, Ri);
  orc_corr_fft(xr, xi, FS, N, coh, 1250, 2, chips[9], Qr, Qi);
  err = 0, mag = 0;
  for (int k = 0; k < N; ++k) {
    err = fmax(err, fabs(Rr[k] - Qr[k]) + fabs(Ri[k] - Qi[k]));
    mag = fmax(mag, fabs(Rr[k]) + fabs(Ri[k]));
  }
  if (err > 1e-9 * mag) return 18;

  /* surfaces (half-bit sets, code Doppler, threads) and detection */
  const int prns[3] = {3, 9, 30};
  const int64_t dopp[5] = {-10000, -4750, 0, 250, 9750};
  const int nsets = 2;
  double *surf = malloc(sizeof(double) * nsets * 3 * 5 * N);
  if (orc_surfaces(xr, xi, n, FS, coh, nblocks, 1, prns, 3, dopp, 5, 3, 1, surf) != 0) return 19;
  if (orc_surfaces(xr, xi, n, FS, coh, nblocks, 0, prns, 3, dopp, 5, 1, 0, surf) != 0) return 20;
  if (orc_surfaces(xr, xi, n, FS, coh, nblocks + 1, 0, prns, 3, dopp, 5, 1, 0, surf) == 0) return 21;
  orc_peak_result pk[3];
  orc_detect(surf, 1, 3, 5, N, 1, 0, 2.0, prns, pk);
  orc_detect(surf, 1, 3, 5, N, 1, 1, 2.0, prns, pk);

  /* fine acquisition: objective, gradient, ascent with a pre-search */
  double chipd[ORC_CHIPS], P, grad[2];
  for (int i = 0; i < ORC_CHIPS; ++i) chipd[i] = chips[9][i];
  orc_refine_eval(xr, xi, 2 * N, FS, chipd, 1250.5, 100.25, &P, grad);
  orc_refine_eval(xr, xi, 2 * N, FS, chipd, -300.0, -5.75, &P, grad); /* delay outside [0, 1023) */
  orc_refined rf;
  orc_refine(xr, xi, 2 * N, FS, chipd, 1250.0, 100.0, 12, 500.0, 1, &rf);
  orc_refine(xr, xi, 2 * N, FS, chipd, 1250.0, 100.0, 12, 500.0, 0, &rf);

  /* tracking channel: a 4 ms recording at 2.048 MHz (above the chip rate) */
  const int64_t fs2 = 2048000, n2 = 4 * 2048;
  double *tr_r = malloc(sizeof(double) * n2), *tr_i = malloc(sizeof(double) * n2);
  for (int64_t k = 0; k < n2; ++k) {
    tr_r[k] = urand() - 0.5;
    tr_i[k] = urand() - 0.5;
  }
  orc_track_rec tr[4];
  if (orc_track(tr_r, tr_i, n2, fs2, 1, 4, chips[9], 1250.0, 100.0, 1.0, 15.0, 2.0, tr) != 0) return 22;
  if (orc_track(tr_r, tr_i, n2, fs2, 2, 2, chips[9], -3000.0, 1022.9, 0.5, 10.0, 1.0, tr) != 0) return 23;
  if (orc_track(tr_r, tr_i, n2, fs2, 1, 5, chips[9], 1250.0, 100.0, 1.0, 15.0, 2.0, tr) == 0) return 24;
  if (orc_track(xr, xi, n, FS, 1, 4, chips[9], 1250.0, 100.0, 1.0, 15.0, 2.0, tr) == 0) return 25; /* fs < chip rate */
  free(tr_r);
  free(tr_i);

  free(raw8);
  free(raw2);
  free(xr);
  free(xi);
  free(surf);
  printf("oracle sanitize harness: ok\n");
  return 0;
}

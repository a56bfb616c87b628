/*
 * oracle.c -- plain FP64 CPU oracle for GPS L1 C/A acquisition by FFT parallel
 * code-phase search (the acquisition channel of Section 3, Fig. 2 of
 * "Accelerating a Cloud-Based Software GNSS Receiver", Karimi, Pamir, Afzal).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the timed CPU baseline of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Every quantity is computed in double precision with plain loops:
 *   - Gold codes from the G2-delay formulation (the CUDA path uses the
 *     two-tap phase-selector formulation instead),
 *   - exact integer carrier-phase reduction (f*n mod fs),
 *   - a textbook iterative radix-2 FFT with per-stage cos/sin twiddles,
 *   - a direct O(N^2) DFT and a brute-force time-domain correlation,
 *   - power surfaces (optionally code-Doppler compensated), peak /
 *     second-peak detection, and
 *   - the coherent-power objective of fine acquisition, its analytic
 *     gradient and a gradient-ascent refinement, and
 *   - a tracking channel: fixed-point carrier and code NCOs, early / prompt /
 *     late correlators, Costas PLL and carrier-aided DLL.
 *
 * The paper describes the acquisition channel only at block-diagram level:
 * code NCO -> replica, carrier NCO -> first mixing, FFT of the mixed signal
 * and of the replica, second (frequency-domain) mixing, IFFT, "signal
 * detection" (Section 3, Fig. 2).  The detailed readings (code definition,
 * replica sampling, Doppler sign, normalisation, detection statistic,
 * half-bit sets, refinement step rule) are stated next to each function.
 *
 * Parity pins: codes (ICD first-10-chip octals, balance, three-valued
 * auto/cross-correlation, a third phase-selector derivation in the tests);
 * FFT (numpy FFT, Parseval, impulse/tone, round trip); correlation (a
 * brute-force direct sum and a numpy brute force); surfaces (noise-free
 * closed form A^2 L^2 per block); detection (injected truth); refinement
 * objective (Dirichlet closed form with the code removed) and gradient
 * (central finite differences).  Parity unpinned (conventions, not results
 * of the paper): the half-bit set choice, the detection threshold, the
 * second-peak exclusion region and the refinement step rule.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CHIPS 1023
#define ORC_CHIP_RATE 1.023e6
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Gold codes (code NCO input, Section 3, Fig. 2)                            */
/* ------------------------------------------------------------------------ */

/* G2 delay in chips for PRN 1..32 (IS-GPS-200, Table 3-Ia). */
static const int orc_g2_delay[32] = {
    5,   6,   7,   8,   17,  18,  139, 140, 141, 251, 252,
    254, 255, 256, 257, 258, 469, 470, 471, 472, 473, 474,
    509, 512, 513, 514, 515, 516, 859, 860, 861, 862};

/* One full period of a 10-stage Fibonacci LFSR seeded with all ones.
 * taps[] lists the stages (1..10) XORed into the feedback; the output is
 * stage 10.  G1 = 1 + x^3 + x^10, G2 = 1 + x^2 + x^3 + x^6 + x^8 + x^9 + x^10. */
static void orc_lfsr_sequence(const int *taps, int ntaps, uint8_t *seq) {
  int reg[10];
  for (int s = 0; s < 10; ++s) reg[s] = 1;
  for (int i = 0; i < ORC_CHIPS; ++i) {
    seq[i] = (uint8_t)reg[9];
    int fb = 0;
    for (int t = 0; t < ntaps; ++t) fb ^= reg[taps[t] - 1];
    for (int s = 9; s > 0; --s) reg[s] = reg[s - 1];
    reg[0] = fb;
  }
}

/* C/A code of one PRN as +-1 chips: bit b maps to 1 - 2b.
 * chip[i] = G1[i] xor G2[(i - delay_p) mod 1023].  Returns 0, or -1 for a
 * PRN outside 1..32. */
int orc_ca_code(int prn, int8_t *chips) {
  static const int g1_taps[2] = {3, 10};
  static const int g2_taps[6] = {2, 3, 6, 8, 9, 10};
  if (prn < 1 || prn > 32) return -1;
  uint8_t g1[ORC_CHIPS], g2[ORC_CHIPS];
  orc_lfsr_sequence(g1_taps, 2, g1);
  orc_lfsr_sequence(g2_taps, 6, g2);
  int d = orc_g2_delay[prn - 1];
  for (int i = 0; i < ORC_CHIPS; ++i) {
    int bit = g1[i] ^ g2[(i - d + ORC_CHIPS) % ORC_CHIPS];
    chips[i] = (int8_t)(1 - 2 * bit);
  }
  return 0;
}

/* Replica sampled at fs over one code period of N samples (code NCO,
 * Fig. 2): c_s[m] = c[floor(m * 1023 / N)], chip 0 starting at sample 0. */
void orc_replica(const int8_t *chips, int N, double *rep) {
  for (int m = 0; m < N; ++m) rep[m] = chips[(int)(((int64_t)m * ORC_CHIPS) / N)];
}

/* ------------------------------------------------------------------------ */
/* Sample unpacking (the raw client recording, Section 1 / Section 4.2)      */
/* ------------------------------------------------------------------------ */

/* fmt 0: int8 I,Q interleaved (2 bytes per complex sample).
 * fmt 1: 2-bit I/Q, two complex samples per byte,
 *        byte = I0 | Q0<<2 | I1<<4 | Q1<<6, code c -> level 2c - 3. */
int orc_unpack(const uint8_t *raw, int64_t n, int fmt, double *re, double *im) {
  if (fmt == 0) {
    const int8_t *s = (const int8_t *)raw;
    for (int64_t k = 0; k < n; ++k) {
      re[k] = s[2 * k];
      im[k] = s[2 * k + 1];
    }
    return 0;
  }
  if (fmt == 1) {
    for (int64_t k = 0; k < n; ++k) {
      uint8_t byte = raw[k / 2];
      int shift = (int)(k % 2) * 4;
      int ci = (byte >> shift) & 3;
      int cq = (byte >> (shift + 2)) & 3;
      re[k] = 2 * ci - 3;
      im[k] = 2 * cq - 3;
    }
    return 0;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Carrier wipe-off and coherent fold (carrier NCO + first mixing, Fig. 2)   */
/* ------------------------------------------------------------------------ */

/* Phase of the local carrier at global sample n for Doppler f (integer Hz),
 * in cycles, reduced exactly: ((f * n) mod fs) / fs.  The recorded signal is
 * taken to carry exp(+j 2 pi f t), so bin f wipes it off with
 * exp(-j 2 pi f n / fs); the phase origin is the first recorded sample. */
static double orc_carrier_cycles(int64_t f, int64_t n, int64_t fs) {
  int64_t fr = ((f % fs) + fs) % fs;
  int64_t r = (fr * n) % fs;
  return (double)r / (double)fs;
}

/* y[m] = sum_{i < coh} x[b L + i N + m] exp(-j 2 pi ((f (bL+iN+m)) mod fs)/fs)
 * for m < N, with L = coh N.  The fold over the coherent milliseconds is
 * exact because the replica repeats every N samples. */
void orc_wipe_fold(const double *xr, const double *xi, int64_t fs, int N,
                   int coh, int64_t f, int b, double *yr, double *yi) {
  int64_t L = (int64_t)coh * N;
  for (int m = 0; m < N; ++m) {
    double ar = 0.0, ai = 0.0;
    for (int i = 0; i < coh; ++i) {
      int64_t n = (int64_t)b * L + (int64_t)i * N + m;
      double ph = -2.0 * ORC_PI * orc_carrier_cycles(f, n, fs);
      double c = cos(ph), s = sin(ph);
      ar += xr[n] * c - xi[n] * s;
      ai += xr[n] * s + xi[n] * c;
    }
    yr[m] = ar;
    yi[m] = ai;
  }
}

/* ------------------------------------------------------------------------ */
/* FFT (the FFT / IFFT blocks of Fig. 2)                                     */
/* ------------------------------------------------------------------------ */

/* Textbook iterative radix-2 decimation-in-time FFT, in place, N a power of
 * two.  Forward: X[k] = sum_n x[n] exp(-j 2 pi n k / N), unscaled.
 * Inverse (inverse != 0): x[n] = (1/N) sum_k X[k] exp(+j 2 pi n k / N).
 * Twiddles come from cos/sin once per (stage, offset). */
int orc_fft(double *re, double *im, int N, int inverse) {
  if (N < 1 || (N & (N - 1))) return -1;
  int bits = 0;
  while ((1 << bits) < N) ++bits;
  for (int k = 0; k < N; ++k) {
    int r = 0;
    for (int t = 0; t < bits; ++t) r |= ((k >> t) & 1) << (bits - 1 - t);
    if (r > k) {
      double tr = re[k], ti = im[k];
      re[k] = re[r];
      im[k] = im[r];
      re[r] = tr;
      im[r] = ti;
    }
  }
  double sign = inverse ? 1.0 : -1.0;
  for (int len = 2; len <= N; len <<= 1) {
    int half = len / 2;
    for (int j = 0; j < half; ++j) {
      double ang = sign * 2.0 * ORC_PI * (double)j / (double)len;
      double wr = cos(ang), wi = sin(ang);
      for (int s = 0; s < N; s += len) {
        int a = s + j, b = s + j + half;
        double br = re[b] * wr - im[b] * wi;
        double bi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - br;
        im[b] = im[a] - bi;
        re[a] += br;
        im[a] += bi;
      }
    }
  }
  if (inverse) {
    for (int k = 0; k < N; ++k) {
      re[k] /= N;
      im[k] /= N;
    }
  }
  return 0;
}

/* Direct O(N^2) DFT with the same sign and scaling conventions (any N). */
void orc_dft(const double *re, const double *im, int N, int inverse,
             double *outr, double *outi) {
  double sign = inverse ? 1.0 : -1.0;
  for (int k = 0; k < N; ++k) {
    double ar = 0.0, ai = 0.0;
    for (int n = 0; n < N; ++n) {
      double ang = sign * 2.0 * ORC_PI * (double)(((int64_t)n * k) % N) / N;
      double c = cos(ang), s = sin(ang);
      ar += re[n] * c - im[n] * s;
      ai += re[n] * s + im[n] * c;
    }
    outr[k] = inverse ? ar / N : ar;
    outi[k] = inverse ? ai / N : ai;
  }
}

/* ------------------------------------------------------------------------ */
/* Correlation (second mixing + IFFT, Fig. 2)                                */
/* ------------------------------------------------------------------------ */

/* Brute-force coherent correlation of block b, straight from the definition:
 * R[tau] = sum_{n < L} x[bL+n] exp(-j 2 pi ((f (bL+n)) mod fs)/fs)
 *          * c_s[(n - tau) mod N],   tau < N. */
void orc_corr_direct(const double *xr, const double *xi, int64_t fs, int N,
                     int coh, int64_t f, int b, const int8_t *chips,
                     double *Rr, double *Ri) {
  int64_t L = (int64_t)coh * N;
  double *rep = (double *)malloc(sizeof(double) * N);
  orc_replica(chips, N, rep);
  for (int tau = 0; tau < N; ++tau) {
    double ar = 0.0, ai = 0.0;
    for (int64_t n = 0; n < L; ++n) {
      int64_t g = (int64_t)b * L + n;
      double ph = -2.0 * ORC_PI * orc_carrier_cycles(f, g, fs);
      double c = cos(ph), s = sin(ph);
      double wr = xr[g] * c - xi[g] * s;
      double wi = xr[g] * s + xi[g] * c;
      double cv = rep[(int)((((n - tau) % N) + N) % N)];
      ar += wr * cv;
      ai += wi * cv;
    }
    Rr[tau] = ar;
    Ri[tau] = ai;
  }
  free(rep);
}

/* FFT form of the same correlation: R = IFFT( FFT(y) * conj(FFT(c_s)) ),
 * forward unscaled, inverse scaled by 1/N, y the folded wiped block. */
void orc_corr_fft(const double *xr, const double *xi, int64_t fs, int N,
                  int coh, int64_t f, int b, const int8_t *chips, double *Rr,
                  double *Ri) {
  double *cr = (double *)calloc(N, sizeof(double));
  double *ci = (double *)calloc(N, sizeof(double));
  orc_replica(chips, N, cr);
  orc_fft(cr, ci, N, 0);
  orc_wipe_fold(xr, xi, fs, N, coh, f, b, Rr, Ri);
  orc_fft(Rr, Ri, N, 0);
  for (int k = 0; k < N; ++k) {
    double a = Rr[k], bb = Ri[k];
    Rr[k] = a * cr[k] + bb * ci[k]; /* (a + jb) * (cr - j ci) */
    Ri[k] = bb * cr[k] - a * ci[k];
  }
  orc_fft(Rr, Ri, N, 1);
  free(cr);
  free(ci);
}

/* ------------------------------------------------------------------------ */
/* Power surfaces: |R|^2 summed non-coherently over blocks                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  const double *xr, *xi;
  int64_t fs;
  int N, coh, nblocks, half_bit, nprn, ndopp, code_doppler;
  const int64_t *dopp_hz;     /* [ndopp] */
  const double *code_re;      /* [nprn][N] FFT of the replica */
  const double *code_im;
  double *surf;               /* [sets][nprn][ndopp][N] */
  int next;                   /* next Doppler row to take */
  pthread_mutex_t lock;
} orc_surface_job;

/* Code Doppler.  The receiver's code NCO (Section 3, Fig. 2) runs at the
 * nominal chip rate R_c; a signal at Doppler f has its code compressed by the
 * same factor as its carrier, f / f_L1, so its delay falls by f t / f_L1 of a
 * second per second: f t fs / f_L1 samples after t seconds (f_L1 = 1540 R_c
 * = 1575.42 MHz).  At the start of block b (t = b L / fs) that is f b L / f_L1
 * samples; the shift used is the nearest integer, halves rounded up:
 * floor((2 f b L + f_L1) / (2 f_L1)), in exact integer arithmetic. */
static int64_t orc_code_doppler_shift(int64_t f, int64_t b, int64_t L) {
  const int64_t f_l1 = 1540LL * 1023000LL;
  const int64_t num = 2 * f * b * L + f_l1;
  const int64_t den = 2 * f_l1;
  int64_t q = num / den; /* C truncates toward zero */
  if (num % den != 0 && num < 0) q -= 1;
  return q;
}

/* S^{(s)}_{p,f}[tau] = sum over blocks b with set(b) = s of |R_{p,f,b}[tau]|^2,
 * set(b) = b mod 2 when half-bit sets are on, else 0 (one set).  With code
 * Doppler compensation, block b enters shifted by its code-Doppler shift
 * sigma_b: S[tau] += |R_b[(tau - sigma_b) mod N]|^2, so that a peak whose
 * delay falls by sigma_b samples at block b is summed at its block-0 delay.
 * Each Doppler row is independent, so worker threads take whole rows. */
static void *orc_surface_worker(void *arg) {
  orc_surface_job *job = (orc_surface_job *)arg;
  int N = job->N;
  double *yr = (double *)malloc(sizeof(double) * N);
  double *yi = (double *)malloc(sizeof(double) * N);
  double *zr = (double *)malloc(sizeof(double) * N);
  double *zi = (double *)malloc(sizeof(double) * N);
  int nsets = job->half_bit ? 2 : 1;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    int d = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (d >= job->ndopp) break;
    for (int b = 0; b < job->nblocks; ++b) {
      int s = job->half_bit ? (b % 2) : 0;
      orc_wipe_fold(job->xr, job->xi, job->fs, N, job->coh, job->dopp_hz[d], b,
                    yr, yi);
      orc_fft(yr, yi, N, 0);
      for (int p = 0; p < job->nprn; ++p) {
        const double *cr = job->code_re + (size_t)p * N;
        const double *ci = job->code_im + (size_t)p * N;
        for (int k = 0; k < N; ++k) {
          zr[k] = yr[k] * cr[k] + yi[k] * ci[k];
          zi[k] = yi[k] * cr[k] - yr[k] * ci[k];
        }
        orc_fft(zr, zi, N, 1);
        double *row = job->surf +
                      (((size_t)s * job->nprn + p) * job->ndopp + d) * (size_t)N;
        int64_t sigma = 0;
        if (job->code_doppler)
          sigma = orc_code_doppler_shift(job->dopp_hz[d], b, (int64_t)job->coh * N);
        for (int t = 0; t < N; ++t) {
          int64_t src = ((t - sigma) % N + N) % N;
          row[t] += zr[src] * zr[src] + zi[src] * zi[src];
        }
      }
    }
  }
  (void)nsets;
  free(yr);
  free(yi);
  free(zr);
  free(zi);
  return NULL;
}

/* Surfaces for every listed PRN and Doppler bin over nblocks whole blocks of
 * L = coh * N samples.  surf must hold sets*nprn*ndopp*N doubles and is
 * overwritten.  Returns 0, or -1 on bad arguments. */
int orc_surfaces(const double *xr, const double *xi, int64_t n_samples,
                 int64_t fs, int coh, int nblocks, int half_bit,
                 const int *prns, int nprn, const int64_t *dopp_hz, int ndopp,
                 int nthreads, int code_doppler, double *surf) {
  if (fs % 1000) return -1;
  int N = (int)(fs / 1000);
  if (N < 1 || (N & (N - 1))) return -1;
  if ((int64_t)nblocks * coh * N > n_samples || nblocks < 1) return -1;
  int nsets = half_bit ? 2 : 1;
  double *code_re = (double *)calloc((size_t)nprn * N, sizeof(double));
  double *code_im = (double *)calloc((size_t)nprn * N, sizeof(double));
  int8_t chips[ORC_CHIPS];
  for (int p = 0; p < nprn; ++p) {
    if (orc_ca_code(prns[p], chips)) {
      free(code_re);
      free(code_im);
      return -1;
    }
    orc_replica(chips, N, code_re + (size_t)p * N);
    orc_fft(code_re + (size_t)p * N, code_im + (size_t)p * N, N, 0);
  }
  memset(surf, 0, sizeof(double) * (size_t)nsets * nprn * ndopp * N);
  orc_surface_job job;
  job.xr = xr;
  job.xi = xi;
  job.fs = fs;
  job.N = N;
  job.coh = coh;
  job.nblocks = nblocks;
  job.half_bit = half_bit;
  job.code_doppler = code_doppler;
  job.nprn = nprn;
  job.ndopp = ndopp;
  job.dopp_hz = dopp_hz;
  job.code_re = code_re;
  job.code_im = code_im;
  job.surf = surf;
  job.next = 0;
  pthread_mutex_init(&job.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  for (int t = 0; t < nthreads; ++t)
    pthread_create(&th[t], NULL, orc_surface_worker, &job);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&job.lock);
  free(code_re);
  free(code_im);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Signal detection ("utilize the correlation results for signal detection", */
/* Section 3): peak against second peak                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int prn;
  int detected;
  int set;
  int dopp_bin;
  int code_phase;
  double peak;
  double second;
  double ratio;
} orc_peak_result;

/* One surface S[ndopp][N].  Peak = largest cell, ties to the smallest linear
 * index (Doppler-major, then code phase).  Second = largest cell of the
 * peak's Doppler row whose circular distance from the peak phase exceeds
 * excl samples (or of the whole surface outside that band when
 * whole_surface != 0).  ratio = peak / second (inf if second == 0). */
void orc_peak_one(const double *S, int ndopp, int N, int excl, int whole_surface,
                  orc_peak_result *out) {
  int bd = 0, bt = 0;
  double best = S[0];
  for (int d = 0; d < ndopp; ++d)
    for (int t = 0; t < N; ++t)
      if (S[(size_t)d * N + t] > best) {
        best = S[(size_t)d * N + t];
        bd = d;
        bt = t;
      }
  double second = 0.0;
  int have = 0;
  for (int d = 0; d < ndopp; ++d) {
    if (!whole_surface && d != bd) continue;
    for (int t = 0; t < N; ++t) {
      int dist = abs(t - bt);
      if (N - dist < dist) dist = N - dist;
      if (dist <= excl) continue;
      double v = S[(size_t)d * N + t];
      if (!have || v > second) {
        second = v;
        have = 1;
      }
    }
  }
  out->dopp_bin = bd;
  out->code_phase = bt;
  out->peak = best;
  out->second = second;
  out->ratio = second > 0.0 ? best / second : INFINITY;
}

/* Detection per PRN from the surfaces [sets][nprn][ndopp][N].  With two
 * half-bit sets the set with the larger ratio is kept (ties to set 0).
 * detected = ratio >= threshold. */
void orc_detect(const double *surf, int nsets, int nprn, int ndopp, int N,
                int excl, int whole_surface, double threshold, const int *prns,
                orc_peak_result *out) {
  for (int p = 0; p < nprn; ++p) {
    orc_peak_result best;
    for (int s = 0; s < nsets; ++s) {
      orc_peak_result r;
      orc_peak_one(surf + ((size_t)s * nprn + p) * ndopp * (size_t)N, ndopp, N,
                   excl, whole_surface, &r);
      r.set = s;
      if (s == 0 || r.ratio > best.ratio) best = r;
    }
    best.prn = prns[p];
    best.detected = best.ratio >= threshold;
    out[p] = best;
  }
}

/* ------------------------------------------------------------------------ */
/* Fine acquisition: coherent power P(f, tau) with a linearly interpolated   */
/* replica, its gradient, and gradient ascent from the coarse peak.          */
/* ------------------------------------------------------------------------ */

/* z = sum_{n<L} x[n] exp(-j 2 pi f n / fs) ctilde(t_n),
 * t_n = n R_c / fs - tau (chips since the code epoch delayed by tau),
 * ctilde(t) = (1 - a) c[k mod 1023] + a c[(k + 1) mod 1023] with
 * u = t - 1/2, k = floor(u), a = u - k: linear interpolation between chip
 * centres (chip k occupies [k, k+1) and its value sits at k + 1/2, so that
 * the power peak of a rectangular-chip signal lies at its true delay).
 * P = |z|^2.
 * dP/df   = 2 Re(conj(z) sum x[n] e^{-j theta_n} (-j 2 pi n / fs) ctilde(t_n))
 * dP/dtau = 2 Re(conj(z) sum x[n] e^{-j theta_n} (-(c[k+1] - c[k]))),
 *           k = floor(t_n - 1/2) (the slope of the segment t_n lies on).
 * chips is +-1 (or any real code, e.g. all ones for the pure-tone check).
 * grad may be NULL. */
void orc_refine_eval(const double *xr, const double *xi, int64_t L, double fs,
                     const double *chips, double f, double tau, double *P,
                     double *grad) {
  double zr = 0, zi = 0, dfr = 0, dfi = 0, dtr = 0, dti = 0;
  for (int64_t n = 0; n < L; ++n) {
    double th = 2.0 * ORC_PI * f * (double)n / fs;
    double c = cos(th), s = -sin(th); /* e^{-j theta} = c + j s */
    double wr = xr[n] * c - xi[n] * s;
    double wi = xr[n] * s + xi[n] * c;
    double u = (double)n * ORC_CHIP_RATE / fs - tau - 0.5;
    double fl = floor(u);
    double a = u - fl;
    int64_t k = (int64_t)fl;
    int i0 = (int)(((k % ORC_CHIPS) + ORC_CHIPS) % ORC_CHIPS);
    int i1 = (i0 + 1) % ORC_CHIPS;
    double ct = (1.0 - a) * chips[i0] + a * chips[i1];
    double slope = chips[i1] - chips[i0];
    zr += wr * ct;
    zi += wi * ct;
    /* (-j 2 pi n / fs) * (wr + j wi) = (2 pi n/fs) (wi - j wr) */
    double g = 2.0 * ORC_PI * (double)n / fs;
    dfr += g * wi * ct;
    dfi += -g * wr * ct;
    dtr += -wr * slope;
    dti += -wi * slope;
  }
  *P = zr * zr + zi * zi;
  if (grad) {
    grad[0] = 2.0 * (zr * dfr + zi * dfi);
    grad[1] = 2.0 * (zr * dtr + zi * dti);
  }
}

typedef struct {
  double f, tau, P;
  int iters;
  int status; /* 0 converged by step size, 1 no ascent step, 2 iteration cap */
} orc_refined;

/* Gradient ascent on P(f, tau) (coarse-to-fine hand-off of Section 3, Fig. 1;
 * the step rule is this library's reading, the paper gives none).
 * Doppler pre-search: with search_hz > 0, P(f0 + k d, tau0) is evaluated for
 * d = fs / (2 L) (half the main-lobe width 1/T) and k = +-1 .. +-K,
 * K = floor(search_hz / d), in the order -1, +1, -2, +2, ..., and the ascent
 * starts from the first largest value (f0 itself first).  Then each
 * iteration moves the two coordinates in turn:
 *   f:   Newton step d_f = g_f / (P (2 pi)^2 T^2 / 6) (closed-form peak
 *        curvature, T = L / fs); trials alpha = 1, 1/2, ... (at most
 *        max_halvings halvings); the first trial is taken when Armijo holds,
 *        P(new) >= P + c1 alpha g_f d_f, or (with flat_accept) when it
 *        reduces |dP/df| without losing more than 1e-5 of P.  The second
 *        clause is the rule of the FP32 kernel, where near the peak the
 *        change of P is below single-precision resolution while the
 *        gradient still resolves it; in FP64 Armijo alone resolves the peak,
 *        and the tests show both forms end at the same point (flat_accept is
 *        on by default so the oracle follows the kernel's rule);
 *   tau: sign step d_tau = s_tau sign(g_tau) (s_tau starts at step0 chip)
 *        with Armijo backtracking, then s_tau <- alpha s_tau.  The slope of
 *        the replica segment is one-sided where samples sit exactly on a
 *        kink, so when every trial fails the opposite direction is tried
 *        (taking the first trial that raises P).
 * When every tau trial on both sides, down to s_tau / 2^max_halvings, lowers
 * P, tau sits on the kink of the peak and s_tau is shrunk by that factor.
 * An iteration that ends with P no higher than it started (the flat_accept
 * clause can lower P while the tau step wins it back) halves s_tau: near the
 * peak the two steps can otherwise trade the last bits of P back and forth
 * with a tau step that is always accepted and never shrinks.  P and the
 * gradient are re-evaluated after every accepted step.  Stop as converged
 * (status 0) when the Newton step |d_f| is below tol_f Hz and s_tau below
 * tol_tau chip, as stuck (status 1) when neither coordinate moved, or after
 * max_iter iterations (status 2). */
void orc_refine(const double *xr, const double *xi, int64_t L, double fs,
                const double *chips, double f0, double tau0, int max_iter,
                double search_hz, int flat_accept, orc_refined *out) {
  const double c1 = 1e-4, step0 = 0.05, tol_tau = 1e-5, tol_f = 1e-3;
  const int max_halvings = 20;
  double T = (double)L / fs;
  double curv = (2.0 * ORC_PI) * (2.0 * ORC_PI) * T * T / 6.0;
  double f = f0, tau = tau0, P, g[2];
  double s_tau = step0;
  if (search_hz > 0.0) {
    double d = fs / (2.0 * (double)L);
    int K = (int)floor(search_hz / d);
    double best;
    orc_refine_eval(xr, xi, L, fs, chips, f0, tau0, &best, NULL);
    for (int k = 1; k <= K; ++k)
      for (int sg = -1; sg <= 1; sg += 2) {
        double fk = f0 + sg * k * d, Pk;
        orc_refine_eval(xr, xi, L, fs, chips, fk, tau0, &Pk, NULL);
        if (Pk > best) {
          best = Pk;
          f = fk;
        }
      }
  }
  orc_refine_eval(xr, xi, L, fs, chips, f, tau, &P, g);
  int it = 0, status = 2;
  for (; it < max_iter; ++it) {
    double move_f = 0.0, move_t = 0.0;
    const double P_start = P;
    double df = P > 0.0 ? g[0] / (P * curv) : 0.0;
    if (df != 0.0) {
      double alpha = 1.0;
      for (int h = 0; h <= max_halvings; ++h) {
        double Pn, gn[2];
        orc_refine_eval(xr, xi, L, fs, chips, f + alpha * df, tau, &Pn, gn);
        int armijo = Pn >= P + c1 * alpha * g[0] * df;
        int flatter = flat_accept && fabs(gn[0]) < fabs(g[0]) && Pn >= (1.0 - 1e-5) * P;
        if (armijo || flatter) {
          f += alpha * df;
          move_f = fabs(alpha * df);
          P = Pn;
          g[0] = gn[0];
          g[1] = gn[1];
          break;
        }
        alpha *= 0.5;
      }
    }
    double dt = g[1] > 0.0 ? s_tau : (g[1] < 0.0 ? -s_tau : 0.0);
    if (dt == 0.0) {
      s_tau = 0.0; /* exactly flat in tau */
    } else {
      double alpha = 1.0;
      int accepted = 0;
      for (int h = 0; h <= max_halvings; ++h) {
        double Pn;
        orc_refine_eval(xr, xi, L, fs, chips, f, tau + alpha * dt, &Pn, NULL);
        if (Pn >= P + c1 * alpha * g[1] * dt) {
          tau += alpha * dt;
          s_tau *= alpha;
          move_t = fabs(alpha * dt);
          orc_refine_eval(xr, xi, L, fs, chips, f, tau, &P, g);
          accepted = 1;
          break;
        }
        alpha *= 0.5;
      }
      /* At a kink the segment slope is one-sided: try the other direction
       * (strict increase of P), then treat tau as sitting on the kink. */
      if (!accepted) {
        alpha = 1.0;
        for (int h = 0; h <= max_halvings; ++h) {
          double Pn;
          orc_refine_eval(xr, xi, L, fs, chips, f, tau - alpha * dt, &Pn, NULL);
          if (Pn > P) {
            tau -= alpha * dt;
            s_tau *= alpha;
            move_t = fabs(alpha * dt);
            orc_refine_eval(xr, xi, L, fs, chips, f, tau, &P, g);
            accepted = 1;
            break;
          }
          alpha *= 0.5;
        }
      }
      /* every trial down to s_tau / 2^20 on both sides lowered P */
      if (!accepted) s_tau = ldexp(s_tau, -max_halvings);
    }
    if (P <= P_start) s_tau *= 0.5; /* no net gain this iteration */
    if (fabs(df) < tol_f && s_tau < tol_tau) {
      status = 0;
      ++it;
      break;
    }
    if (move_f == 0.0 && move_t == 0.0) {
      status = 1;
      break;
    }
  }
  out->f = f;
  out->tau = tau;
  out->P = P;
  out->iters = it;
  out->status = status;
}

/* ------------------------------------------------------------------------ */
/* Tracking channel (Section 3, Fig. 3): carrier and code NCOs, the first    */
/* mixing stage and time-domain early / prompt / late correlation, closed by */
/* a Costas phase-locked loop and a carrier-aided delay-locked loop.         */
/* ------------------------------------------------------------------------ */

/* The paper gives the tracking channel as a block diagram only; the loop
 * design below is this library's reading, written the way a hardware
 * receiver builds it.
 *
 * NCOs (fixed point, exact integer arithmetic):
 *   carrier phase  Phi (uint32, 2^32 = one cycle), word Wc = round(f 2^32 / fs)
 *                  as a two's-complement 32-bit increment per sample;
 *   code position  P (units of 2^-32 chip, kept in [0, 1023 2^32)), word
 *                  Wk = round(f_code 2^32 / fs) per sample (needs f_code < fs).
 * Interval k covers samples n = k L + i, i < L (L = coh_ms N):
 *   theta_i = Phi + i Wc (mod 2^32),   u_i = P + i Wk,
 *   s_i     = x[n] exp(-j 2 pi theta_i / 2^32),
 *   Z_E     = sum s_i c[floor((u_i + h) / 2^32) mod 1023],
 *   Z_P     = sum s_i c[floor(u_i / 2^32) mod 1023],
 *   Z_L     = sum s_i c[floor((u_i - h) / 2^32) mod 1023],
 * with h = round(spacing / 2 * 2^32) (early and late replicas half the
 * early-late spacing ahead of and behind the prompt one).  The replica delay
 * at the interval start is tau_k = (-P / 2^32) mod 1023 chips (k L samples
 * span a whole number of code periods).  Then Phi += L Wc, P += L Wk (mod).
 * Discriminators:
 *   e_phi = atan(Q_P / I_P) / (2 pi) cycles (Costas: blind to data bits;
 *           0 when Z_P = 0),
 *   e_tau = (1 - spacing / 2) (|Z_L| - |Z_E|) / (|Z_L| + |Z_E|) chips (the
 *           delay error of a triangular correlation peak within half the
 *           spacing; 0 when both are 0).
 * Loops (T = L / fs):
 *   PLL, second order, noise bandwidth B_pll, zeta = 1/sqrt(2),
 *       w_n = 8 zeta B_pll / (4 zeta^2 + 1):
 *       f_int += w_n^2 T e_phi,   f = f_int + 2 zeta w_n e_phi   (Hz);
 *   DLL, first order with carrier aiding, noise bandwidth B_dll:
 *       f_code = R_c (1 + f / f_L1) - 4 B_dll e_tau   (chip/s),
 *       f_L1 = 1540 R_c (the code Doppler is the carrier Doppler / 1540).
 * Start: f_int = f = f0, Phi = 0, P = round(-tau0 2^32) mod (1023 2^32). */
typedef struct {
  double f_hz;      /* carrier NCO frequency of the interval, Wc fs / 2^32 */
  double tau_chips; /* replica delay at the interval start */
  double ze[2], zp[2], zl[2];
  double e_phi, e_tau;
} orc_track_rec;

static uint32_t orc_round_word(double v) { /* round half away, to 32 bits */
  return (uint32_t)(int64_t)llround(v);
}

int orc_track(const double *xr, const double *xi, int64_t n_samples, int64_t fs, int coh_ms,
              int n_int, const int8_t *chips, double f0, double tau0, double spacing,
              double b_pll, double b_dll, orc_track_rec *out) {
  const int64_t N = fs / 1000, L = (int64_t)coh_ms * N;
  const double two32 = 4294967296.0;
  const int64_t period = (int64_t)ORC_CHIPS << 32;
  if (fs % 1000 || (int64_t)n_int * L > n_samples || spacing <= 0.0 || spacing > 1.0) return -1;
  const double T = (double)L / (double)fs;
  const double zeta = 1.0 / sqrt(2.0);
  const double wn = 8.0 * zeta * b_pll / (4.0 * zeta * zeta + 1.0);
  const double f_l1 = 1540.0 * ORC_CHIP_RATE;
  const uint32_t h = orc_round_word(spacing * 0.5 * two32);
  double f_int = f0, f = f0, e_tau = 0.0;
  uint32_t phi = 0;
  int64_t P = llround(-tau0 * two32) % period;
  if (P < 0) P += period;
  for (int k = 0; k < n_int; ++k) {
    const double f_code = ORC_CHIP_RATE * (1.0 + f / f_l1) - 4.0 * b_dll * e_tau;
    if (f_code <= 0.0 || f_code >= (double)fs || fabs(f) >= 0.5 * (double)fs) return -2;
    const uint32_t wc = orc_round_word(f * two32 / (double)fs);
    const uint32_t wk = orc_round_word(f_code * two32 / (double)fs);
    double z[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int64_t i = 0; i < L; ++i) {
      const int64_t n = (int64_t)k * L + i;
      const uint32_t theta = phi + (uint32_t)i * wc;
      const double ang = 2.0 * ORC_PI * (double)theta / two32;
      const double c = cos(ang), s = -sin(ang);
      const double sr = xr[n] * c - xi[n] * s, si = xr[n] * s + xi[n] * c;
      const int64_t u = P + i * (int64_t)wk; /* below (coh + 2) periods: no overflow */
      const int64_t pos[3] = {u + (int64_t)h, u, u - (int64_t)h};
      for (int r = 0; r < 3; ++r) {
        /* pos >= -2^31: one period added keeps it positive, so the division
         * by 2^32 is a floor */
        const int64_t chip = ((pos[r] + period) / ((int64_t)1 << 32)) % ORC_CHIPS;
        z[r][0] += sr * chips[chip];
        z[r][1] += si * chips[chip];
      }
    }
    orc_track_rec *o = out + k;
    o->f_hz = (double)(int32_t)wc * (double)fs / two32;
    o->tau_chips = (double)((period - P) % period) / two32;
    for (int r = 0; r < 2; ++r) {
      o->ze[r] = z[0][r];
      o->zp[r] = z[1][r];
      o->zl[r] = z[2][r];
    }
    const double ip = z[1][0], qp = z[1][1];
    const double e_phi = (ip == 0.0 && qp == 0.0) ? 0.0 : atan(qp / ip) / (2.0 * ORC_PI);
    const double me = hypot(z[0][0], z[0][1]), ml = hypot(z[2][0], z[2][1]);
    e_tau = (me + ml > 0.0) ? (1.0 - spacing / 2.0) * (ml - me) / (ml + me) : 0.0;
    o->e_phi = e_phi;
    o->e_tau = e_tau;
    phi += (uint32_t)L * wc;
    P = (P + L * (int64_t)wk) % period;
    f_int += wn * wn * T * e_phi;
    f = f_int + 2.0 * zeta * wn * e_phi;
  }
  return 0;
}

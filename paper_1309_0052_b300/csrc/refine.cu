// refine.cu -- fine acquisition: coherent power P(f, tau) with a linearly
// interpolated replica, its analytic gradient, and gradient ascent from the
// coarse peak, for many candidates at once (sm_103a).
//
// The paper hands the coarse Doppler / code phase of acquisition to the
// tracking channels for fine tuning (Section 3, Fig. 1); this is that
// hand-off written as a continuous optimisation:
//   z(f, tau)  = sum_{n<L} x[n] exp(-j 2 pi f n / fs) ctilde(u_n),
//   u_n        = n R_c / fs - tau - 1/2     (R_c / fs = 1023 / N chips/sample)
//   ctilde(u)  = (1 - a) c[k mod 1023] + a c[(k + 1) mod 1023],  k = floor(u), a = u - k
//   P          = |z|^2
//   dP/df      = 2 Re(conj(z) sum x e^{-j theta_n} (-j 2 pi n / fs) ctilde(u_n))
//   dP/dtau    = 2 Re(conj(z) sum x e^{-j theta_n} (-(c[k+1] - c[k])))
// Chip k's value sits at the chip centre k + 1/2 (nodes between chip centres).
//
// Arithmetic: per-sample sums in FP32.  The code position is exact: with
// n * 1023 = q N + rem, u_n = (q - tau_int) + (rem / N - tau_frac - 1/2).
// The code sits in shared memory as a sign-bit table; each group of 8
// samples reads one 64-bit window of it, so neighbouring threads (whose
// chips are far apart) make no bank conflicts and no sample needs a modulo.
// The carrier starts from a double-precision phase per thread chunk and
// advances by a per-sample rotation.  Only the optimiser state (f, tau) is
// kept in double.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fft.cuh"
#include "internal.h"

namespace gnss {

struct EvalOut {
  float P, gf, gt;
};

// Sums of K per-thread values over the CTA, all in one pass: a warp shuffle
// tree per value, one shared-memory exchange (red holds 32 K floats) and the
// warps' partial sums added in warp order -- per value the same order as K
// separate reductions, with two CTA barriers instead of 2 K.
template <int T, int K>
__device__ __forceinline__ void block_sums(float (&v)[K], float* red) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  constexpr int W = T / 32;
  if constexpr (W > 1) {
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) red[k * 32 + (threadIdx.x >> 5)] = v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = 0.f;
#pragma unroll
      for (int w = 0; w < W; ++w) v[k] += red[k * 32 + w];
    }
  }
}

// Samples [n0, n0 + 8) as floats.
template <int FMT>
__device__ __forceinline__ void load8(const uint8_t* __restrict__ base, int n0, float (&xi)[8], float (&xq)[8]) {
  if constexpr (FMT == GNSS_FMT_2BIT_IQ) {
    const uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(base + n0 / 2));
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      xi[e] = (float)(int)(2u * ((w >> (4 * e)) & 3u)) - 3.f;
      xq[e] = (float)(int)(2u * ((w >> (4 * e + 2)) & 3u)) - 3.f;
    }
  } else {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(base + 2 * n0));
    const uint32_t wv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xi[2 * k] = (float)(int8_t)(wv[k] & 0xFF);
      xq[2 * k] = (float)(int8_t)((wv[k] >> 8) & 0xFF);
      xi[2 * k + 1] = (float)(int8_t)((wv[k] >> 16) & 0xFF);
      xq[2 * k + 1] = (float)(int8_t)((wv[k] >> 24) & 0xFF);
    }
  }
}

// One evaluation of P (and, with GRAD, the gradient) by the whole CTA.  The
// window is cut into groups of 8 samples (L is a multiple of 8); thread t
// sums the contiguous groups [t * gpt, (t + 1) * gpt) that exist.
// Code of the candidate's PRN as a sign-bit table in shared memory: bit j is
// set when chip j mod 1023 is -1, for j < 1023 + 65, so that a 64-bit window
// read at any chip k < 1023 covers chips k .. k + 63 without a wrap.
static constexpr int kRefBitWords = 34;

struct CodeBits {
  uint32_t w[kRefBitWords];
  float scale;  // 1, or 0 when the PRN is not in the plan (P and gradient 0)
};

// This thread's share of the window (fixed for the CTA): samples
// [n0, n0 + chunk), and the code position of n0, n0 * 1023 = q0 N + rem0.
struct Span {
  int n0, chunk, q0, rem0;
  __device__ __forceinline__ Span(const RefineJob& J, int T) {
    const int groups = J.L / 8;
    const int gpt = (groups + T - 1) / T;
    const int g_end = min(groups, ((int)threadIdx.x + 1) * gpt);
    chunk = max(0, g_end - (int)threadIdx.x * gpt) * 8;
    n0 = min((int)threadIdx.x * gpt, groups) * 8;
    const long long prod = (long long)n0 * 1023;
    q0 = (int)(prod / J.N);
    rem0 = (int)(prod - (long long)q0 * J.N);
  }
};

// Quantities of one evaluation that are the same for every thread, formed by
// thread 0 in FP64 (which runs at a small fraction of the FP32 rate) and
// read by all after a CTA barrier.
struct EvalPoint {
  uint64_t s_fx;  // cycles per sample s = frac(f / fs), times 2^64
  float2 rot;     // e^{-j 2 pi s}
  int ti;         // code delay: integer part (tau modulo 1023)
  float tf;       // and its fraction + 1/2, in [0.5, 1.5)
};

template <int T, int FMT, bool GRAD, bool W32>
__device__ EvalOut evaluate(const RefineJob& J, const CodeBits& cb, const Span& sp, double f, double tau, float* red,
                            EvalPoint* pt) {
  if (threadIdx.x == 0) {
    // carrier e^{-j 2 pi f n / fs}: the phase of sample n0 is frac(n0 s), an
    // exact integer product modulo one cycle in 64-bit fixed point
    const double step_cyc = f * J.inv_fs;
    const double s_frac = step_cyc - floor(step_cyc);  // [0, 1)
    pt->s_fx = (uint64_t)(s_frac * 18446744073709551616.0);
    float ss, sc;
    sincospif((float)(-2.0 * s_frac), &ss, &sc);
    pt->rot = make_float2(sc, ss);
    // P has period 1023 chips in tau: wrap it so the integer part stays small
    const double tw = tau - 1023.0 * floor(tau * (1.0 / 1023.0));
    const double tfl = floor(tw);
    pt->ti = (int)tfl;
    pt->tf = (float)(tw - tfl) + 0.5f;
  }
  __syncthreads();  // the previous evaluation's readers passed its reduction barrier
  const int n0 = sp.n0, chunk = sp.chunk;
  const uint64_t ph_fx = (uint64_t)n0 * pt->s_fx;  // n0 s modulo 1, times 2^64
  const float ph0 = (float)(uint32_t)(ph_fx >> 40) * 0x1p-24f;
  float s0, c0;
  sincospif(-2.f * ph0, &s0, &c0);
  float2 car = make_float2(c0, s0);
  const float2 rot = pt->rot;
  // code position: n * 1023 = q N + rem; u = (q - ti) + (rem / N - tf - 1/2).
  // The thread's first sample takes it from the exact integers; each next
  // sample advances it by 1023 / N chips: k by the integer part, the weight a
  // by the fraction (a multiple of 1 / N, N a power of two), carrying into k.
  const int ti = pt->ti;
  const float tf = pt->tf;
  const float invN = 1.f / (float)J.N;
  const int istep = 1023 / J.N;                              // whole chips per sample
  const float fstep = (float)(1023 - istep * J.N) * invN;  // and the fraction, exact
  const float u0 = fmaf((float)sp.rem0, invN, -tf);          // in (-1.5, 0.5)
  const float fl0 = floorf(u0);
  int k = sp.q0 - ti + (int)fl0;  // chip of the sample (before reduction modulo 1023)
  float a = u0 - fl0;             // its interpolation weight, in [0, 1)
  float nn = (float)n0 - 0.5f * (float)J.L;  // n - L/2, exact in FP32 (|n| < 2^24)
  float zr = 0.f, zi = 0.f, fr = 0.f, fi = 0.f, tr = 0.f, tii = 0.f;
  for (int base = 0; base < chunk; base += 8) {
    float xi[8], xq[8];
    load8<FMT>(J.samples, n0 + base, xi, xq);
    // chips of the group: the position only grows, by at most 8 (istep + 1)
    // chips over 8 samples, so one window from the group's first chip serves
    // all of them and each next chip: 32 bits for N >= 512 (under 18 chips),
    // 64 for N = 256 (under 33)
    const int kf = k;
    int km = kf % 1023;
    km += (km < 0) ? 1023 : 0;
    const uint32_t lo = __funnelshift_r(cb.w[km >> 5], cb.w[(km >> 5) + 1], km & 31);
    uint32_t hi = 0;
    if constexpr (!W32) hi = __funnelshift_r(cb.w[(km >> 5) + 1], cb.w[(km >> 5) + 2], km & 31);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      // wiped sample w = x e^{-j theta}
      const float wr = fmaf(xi[e], car.x, -xq[e] * car.y);
      const float wi = fmaf(xi[e], car.y, xq[e] * car.x);
      // interpolated chip: the sign bits of chips k and k + 1 as +-1
      const uint32_t rel = (uint32_t)(k - kf);
      uint32_t s0, s1;
      if constexpr (W32) {
        s0 = (lo << (31u - rel)) & 0x80000000u;
        s1 = (lo << (30u - rel)) & 0x80000000u;
      } else {
        const uint64_t win = ((uint64_t)hi << 32) | lo;
        s0 = (uint32_t)((win >> rel) & 1u) << 31;
        s1 = (uint32_t)((win >> (rel + 1u)) & 1u) << 31;
      }
      const float c0v = __int_as_float(0x3f800000 | (int)s0);  // +-1
      const float c1v = __int_as_float(0x3f800000 | (int)s1);
      const float sl = c1v - c0v;
      const float ct = fmaf(a, sl, c0v);
      zr = fmaf(wr, ct, zr);
      zi = fmaf(wi, ct, zi);
      if constexpr (GRAD) {
        // sum (n - L/2) w ctilde: the L/2 z part of sum n w ctilde adds
        // 2 Re(conj(z) (-j 2 pi L/2 / fs) z) = 0 to dP/df, and centring n
        // keeps the FP32 sum free of that cancellation
        fr = fmaf(nn * wr, ct, fr);
        fi = fmaf(nn * wi, ct, fi);
        tr = fmaf(-wr, sl, tr);      // sum -w slope
        tii = fmaf(-wi, sl, tii);
        nn += 1.f;
      }
      car = c_mul(car, rot);
      a += fstep;
      k += istep;
      if (a >= 1.f) {
        a -= 1.f;
        ++k;
      }
    }
  }
  EvalOut o;
  if constexpr (GRAD) {
    float sums[6] = {zr * cb.scale, zi * cb.scale, fr * cb.scale, fi * cb.scale, tr * cb.scale, tii * cb.scale};
    block_sums<T, 6>(sums, red);
    zr = sums[0];
    zi = sums[1];
    fr = sums[2];
    fi = sums[3];
    tr = sums[4];
    tii = sums[5];
  } else {
    float sums[2] = {zr * cb.scale, zi * cb.scale};
    block_sums<T, 2>(sums, red);
    zr = sums[0];
    zi = sums[1];
  }
  o.P = zr * zr + zi * zi;
  o.gf = o.gt = 0.f;
  if constexpr (GRAD) {
    // dz/df -> (-j 2 pi / fs) sum (n - L/2) w ctilde = (2 pi / fs) (fi - j fr)
    const float g = (float)(2.0 * 3.14159265358979323846 * J.inv_fs);
    const float dfr = g * fi, dfi = -g * fr;
    o.gf = 2.f * (zr * dfr + zi * dfi);
    o.gt = 2.f * (zr * tr + zi * tii);
  }
  return o;
}

template <int T>
__device__ __forceinline__ void load_chips(const RefineJob& J, int prn, CodeBits& cb) {
  const int idx = (prn >= 1 && prn <= 32) ? J.prn_index[prn] : -1;
  for (int w = threadIdx.x; w < kRefBitWords; w += T) {
    uint32_t v = 0;
    if (idx >= 0)
      for (int b = 0; b < 32; ++b)
        if (J.codes[idx * 1023 + (32 * w + b) % 1023] < 0) v |= 1u << b;
    cb.w[w] = v;
  }
  if (threadIdx.x == 0) cb.scale = idx >= 0 ? 1.f : 0.f;
  __syncthreads();
}

// K6/K7: P and gradient for candidate blockIdx.x.
template <int T, int FMT, bool W32>
__global__ void __launch_bounds__(T) k_refine_eval(RefineJob J, const int* __restrict__ prn, const double* __restrict__ f,
                                                  const double* __restrict__ tau, float* __restrict__ P,
                                                  float* __restrict__ dPdf, float* __restrict__ dPdtau) {
  __shared__ CodeBits chips;
  __shared__ float red[32 * 6];
  load_chips<T>(J, prn[blockIdx.x], chips);
  __shared__ EvalPoint pt;
  const Span sp(J, T);
  const EvalOut o = evaluate<T, FMT, true, W32>(J, chips, sp, f[blockIdx.x], tau[blockIdx.x], red, &pt);
  if (threadIdx.x == 0) {
    P[blockIdx.x] = o.P;
    if (dPdf) dPdf[blockIdx.x] = o.gf;
    if (dPdtau) dPdtau[blockIdx.x] = o.gt;
  }
}

// Gradient ascent, one CTA per candidate (the rule of the FP64 oracle).
// Doppler pre-search over f0 + k d, d = fs / (2 L), k = -1, +1, ..., +-K,
// K = floor(search_hz / d) (first largest P wins, f0 first).  Then each
// iteration takes
//   an f step: Newton d_f = g_f / (P (2 pi)^2 T^2 / 6); trials alpha = 1,
//     1/2, ... (<= 20 halvings), the first taken when Armijo holds
//     (P_new >= P + 1e-4 alpha g_f d_f) or when it reduces |dP/df| without
//     losing more than 1e-5 of P (near the peak the change of P is below
//     single-precision resolution while the gradient still resolves it);
//   a tau step: d_tau = s_tau sign(g_tau), s_tau from 0.05 chip, Armijo,
//     s_tau <- alpha s_tau; when every trial fails, the opposite direction is
//     tried (first trial that raises P), because the segment slope is
//     one-sided where samples sit exactly on a kink;
// re-evaluating P and the gradient after each accepted step; when every tau
// trial on both sides lowers P, tau sits on the kink of the peak and s_tau
// shrinks by 2^20; an iteration that ends with P no higher than it started
// halves s_tau (near the peak the f step's flat acceptance and the tau step
// can otherwise trade the last bit of P back and forth forever).
// Stop: converged (status 0) when the Newton step |d_f| < 1e-3 Hz and
// s_tau < 1e-5 chip, stuck (status 1) when neither coordinate moved, or
// max_iter (status 2).  Control flow is uniform over the CTA because every
// decision uses block-reduced values.
template <int T, int FMT, bool W32>
__global__ void __launch_bounds__(T) k_refine(RefineJob J, const gnss_candidate* __restrict__ cands, int max_iter,
                                             double search_hz, gnss_refined* __restrict__ out) {
  __shared__ CodeBits chips;
  __shared__ float red[32 * 6];
  const gnss_candidate c = cands[blockIdx.x];
  load_chips<T>(J, c.prn, chips);
  __shared__ EvalPoint pt;
  const Span sp(J, T);
  const double c1 = 1e-4, tol_tau = 1e-5, tol_f = 1e-3;
  const double Tw = (double)J.L / J.fs;
  const double curv = (2.0 * 3.14159265358979323846) * (2.0 * 3.14159265358979323846) * Tw * Tw / 6.0;
  double f = c.f_hz, tau = c.tau_chips, s_tau = 0.05;
  // evaluations run (P alone, P and gradient): the work of this candidate
  unsigned n_p = 0, n_pg = 0;
  auto eval_p = [&](double ff, double tt, float* rd, EvalPoint* p) {
    ++n_p;
    return evaluate<T, FMT, false, W32>(J, chips, sp, ff, tt, rd, p);
  };
  auto eval_pg = [&](double ff, double tt, float* rd, EvalPoint* p) {
    ++n_pg;
    return evaluate<T, FMT, true, W32>(J, chips, sp, ff, tt, rd, p);
  };
  if (search_hz > 0.0) {
    const double d = J.fs / (2.0 * (double)J.L);
    const int K = (int)floor(search_hz / d);
    float best = eval_p(c.f_hz, tau, red, &pt).P;
    for (int k = 1; k <= K; ++k)
      for (int sg = -1; sg <= 1; sg += 2) {
        const double fk = c.f_hz + sg * k * d;
        const float Pk = eval_p(fk, tau, red, &pt).P;
        if (Pk > best) {
          best = Pk;
          f = fk;
        }
      }
  }
  EvalOut e = eval_pg(f, tau, red, &pt);
  int it = 0, status = 2;
  for (; it < max_iter; ++it) {
    double move_f = 0.0, move_t = 0.0;
    const float P_start = e.P;
    const double df = e.P > 0.f ? (double)e.gf / ((double)e.P * curv) : 0.0;
    if (df != 0.0) {
      double alpha = 1.0;
      for (int h = 0; h <= 20; ++h) {
        const EvalOut en = eval_pg(f + alpha * df, tau, red, &pt);
        const bool armijo = (double)en.P >= (double)e.P + c1 * alpha * (double)e.gf * df;
        const bool flatter = fabsf(en.gf) < fabsf(e.gf) && (double)en.P >= (1.0 - 1e-5) * (double)e.P;
        if (armijo || flatter) {
          f += alpha * df;
          move_f = fabs(alpha * df);
          e = en;
          break;
        }
        alpha *= 0.5;
      }
    }
    const double dt = e.gt > 0.f ? s_tau : (e.gt < 0.f ? -s_tau : 0.0);
    if (dt == 0.0) {
      s_tau = 0.0;  // exactly flat in tau
    } else {
      double alpha = 1.0;
      bool accepted = false;
      for (int h = 0; h <= 20; ++h) {
        const EvalOut en = eval_p(f, tau + alpha * dt, red, &pt);
        if ((double)en.P >= (double)e.P + c1 * alpha * (double)e.gt * dt) {
          tau += alpha * dt;
          s_tau *= alpha;
          move_t = fabs(alpha * dt);
          e = eval_pg(f, tau, red, &pt);
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      if (!accepted) {  // a segment slope is one-sided at an exact kink: try the other direction
        alpha = 1.0;
        for (int h = 0; h <= 20; ++h) {
          const EvalOut en = eval_p(f, tau - alpha * dt, red, &pt);
          if (en.P > e.P) {
            tau -= alpha * dt;
            s_tau *= alpha;
            move_t = fabs(alpha * dt);
            e = eval_pg(f, tau, red, &pt);
            accepted = true;
            break;
          }
          alpha *= 0.5;
        }
      }
      if (!accepted) s_tau = ldexp(s_tau, -20);  // every trial on both sides lowered P: on the kink
    }
    if (e.P <= P_start) s_tau *= 0.5;  // no net gain this iteration
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
  if (threadIdx.x == 0) {
    gnss_refined r;
    r.f_hz = f;
    r.tau_chips = tau;
    r.power = e.P;
    r.iters = (uint32_t)it;
    r.status = status;
    r.n_eval = (uint16_t)min(n_p, 65535u);
    r.n_eval_grad = (uint16_t)min(n_pg, 65535u);
    out[blockIdx.x] = r;
  }
}

static constexpr int kRefineThreads = 256;

template <int FMT>
static cudaError_t refine_eval_fmt(const RefineJob& J, int n, const int* prn, const double* f, const double* tau,
                                   float* P, float* dPdf, float* dPdtau, cudaStream_t s) {
  // 32-bit chip windows when N >= 512 (under 18 chips per group of 8 samples)
  if (J.N >= 512)
    k_refine_eval<kRefineThreads, FMT, true><<<n, kRefineThreads, 0, s>>>(J, prn, f, tau, P, dPdf, dPdtau);
  else
    k_refine_eval<kRefineThreads, FMT, false><<<n, kRefineThreads, 0, s>>>(J, prn, f, tau, P, dPdf, dPdtau);
  return cudaGetLastError();
}

template <int FMT>
static cudaError_t refine_fmt(const RefineJob& J, int n, const gnss_candidate* cands, int max_iter,
                              double search_hz, gnss_refined* out, cudaStream_t s) {
  // 32-bit chip windows when N >= 512 (under 18 chips per group of 8 samples)
  if (J.N >= 512)
    k_refine<kRefineThreads, FMT, true><<<n, kRefineThreads, 0, s>>>(J, cands, max_iter, search_hz, out);
  else
    k_refine<kRefineThreads, FMT, false><<<n, kRefineThreads, 0, s>>>(J, cands, max_iter, search_hz, out);
  return cudaGetLastError();
}

int refine_threads() { return kRefineThreads; }

cudaError_t launch_refine_eval(const RefineJob& J, int n, const int* prn, const double* f, const double* tau,
                               float* P, float* dPdf, float* dPdtau, cudaStream_t s) {
  return J.format == GNSS_FMT_2BIT_IQ ? refine_eval_fmt<GNSS_FMT_2BIT_IQ>(J, n, prn, f, tau, P, dPdf, dPdtau, s)
                                      : refine_eval_fmt<GNSS_FMT_I8_IQ>(J, n, prn, f, tau, P, dPdf, dPdtau, s);
}

cudaError_t launch_refine(const RefineJob& J, int n, const gnss_candidate* cands, int max_iter, double search_hz,
                          gnss_refined* out, cudaStream_t s) {
  return J.format == GNSS_FMT_2BIT_IQ ? refine_fmt<GNSS_FMT_2BIT_IQ>(J, n, cands, max_iter, search_hz, out, s)
                                      : refine_fmt<GNSS_FMT_I8_IQ>(J, n, cands, max_iter, search_hz, out, s);
}

}  // namespace gnss

using namespace gnss;

static gnss_status refine_job(const gnss_plan* plan, const void* samples_dev, size_t n_samples, uint32_t coh_ms,
                              RefineJob* J) {
  if (coh_ms < 1) return fail_status(GNSS_EINVAL, "coh_ms must be >= 1");
  const size_t L = (size_t)coh_ms * plan->N;
  if (n_samples < L) return fail_status(GNSS_EINVAL, "n_samples is shorter than the coherent window");
  if (L > (size_t)INT32_MAX / 1023) return fail_status(GNSS_EINVAL, "coherent window too long");
  if ((uintptr_t)samples_dev & 15u) return fail_status(GNSS_EINVAL, "device samples must be 16-byte aligned");
  J->samples = (const uint8_t*)samples_dev;
  J->format = (int)plan->desc.format;
  J->N = plan->N;
  J->L = (int)L;
  J->fs = (double)plan->desc.fs_hz;
  J->inv_fs = 1.0 / J->fs;
  J->codes = plan->d_codes;
  J->prn_index = plan->d_prn_index;
  return GNSS_OK;
}

extern "C" {

gnss_status gnss_refine_eval(gnss_plan* plan, const void* samples_dev, size_t n_samples, uint32_t coh_ms,
                             const int32_t* prn_dev, const double* f_dev, const double* tau_dev, size_t n,
                             float* P_dev, float* dPdf_dev, float* dPdtau_dev, void* stream) {
  if (!plan || !samples_dev || !prn_dev || !f_dev || !tau_dev || !P_dev) return fail_status(GNSS_EINVAL, "NULL argument");
  if (n == 0) return GNSS_OK;
  if (n > (size_t)INT32_MAX) return fail_status(GNSS_EINVAL, "too many candidates");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  RefineJob J;
  st = refine_job(plan, samples_dev, n_samples, coh_ms, &J);
  if (st != GNSS_OK) return st;
  cudaError_t e = launch_refine_eval(J, (int)n, prn_dev, f_dev, tau_dev, P_dev, dPdf_dev, dPdtau_dev,
                                     (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e, "gnss_refine_eval");
  return GNSS_OK;
}

gnss_status gnss_refine_device(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                               const gnss_candidate* cands_dev, size_t n_cand, uint32_t coh_ms, uint32_t max_iter,
                               double search_hz, gnss_refined* out_dev, void* stream) {
  if (!plan || !samples_dev || !cands_dev || !out_dev) return fail_status(GNSS_EINVAL, "NULL argument");
  if (n_cand == 0) return GNSS_OK;
  if (n_cand > (size_t)INT32_MAX) return fail_status(GNSS_EINVAL, "too many candidates");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  RefineJob J;
  st = refine_job(plan, samples_dev, n_samples, coh_ms, &J);
  if (st != GNSS_OK) return st;
  if (!(search_hz >= 0.0) || search_hz > 1e6) return fail_status(GNSS_EINVAL, "search_hz must be in [0, 1e6]");
  cudaError_t e = launch_refine(J, (int)n_cand, cands_dev, (int)max_iter, search_hz, out_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e, "gnss_refine_device");
  return GNSS_OK;
}

gnss_status gnss_refine(gnss_plan* plan, const void* samples, size_t n_samples, int samples_on_device,
                        const gnss_candidate* cands, size_t n_cand, uint32_t coh_ms, uint32_t max_iter,
                        double search_hz, gnss_refined* out, void* stream) {
  if (!plan || !samples || !cands || !out) return fail_status(GNSS_EINVAL, "NULL argument");
  if (!(search_hz >= 0.0) || search_hz > 1e6) return fail_status(GNSS_EINVAL, "search_hz must be in [0, 1e6]");
  if (n_cand == 0) return GNSS_OK;
  if (n_cand > (size_t)INT32_MAX) return fail_status(GNSS_EINVAL, "too many candidates");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  if (coh_ms < 1 || n_samples < (size_t)coh_ms * plan->N) return fail_status(GNSS_EINVAL, "n_samples is shorter than the coherent window");
  if (samples_on_device && ((uintptr_t)samples & 15u)) return fail_status(GNSS_EINVAL, "device samples must be 16-byte aligned");
  cudaStream_t cs = (cudaStream_t)stream;
  const size_t L = (size_t)coh_ms * plan->N;
  const size_t c_bytes = (n_cand * sizeof(gnss_candidate) + 255) & ~(size_t)255;
  const size_t o_bytes = (n_cand * sizeof(gnss_refined) + 255) & ~(size_t)255;
  const size_t rb = plan->desc.format == GNSS_FMT_I8_IQ ? 2 * L : (L + 1) / 2;
  const size_t s_bytes = samples_on_device ? 0 : (rb + 255) & ~(size_t)255;
  char* ws = nullptr;
  st = scratch_alloc(plan->device, c_bytes + o_bytes + s_bytes, cs, (void**)&ws);
  if (st != GNSS_OK) return st;
  gnss_candidate* d_c = reinterpret_cast<gnss_candidate*>(ws);
  gnss_refined* d_o = reinterpret_cast<gnss_refined*>(ws + c_bytes);
  const void* d_s = samples;
  cudaError_t e = cudaMemcpyAsync(d_c, cands, n_cand * sizeof(gnss_candidate), cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && !samples_on_device) {
    e = cudaMemcpyAsync(ws + c_bytes + o_bytes, samples, rb, cudaMemcpyHostToDevice, cs);
    d_s = ws + c_bytes + o_bytes;
  }
  RefineJob J;
  if (e == cudaSuccess) {
    st = refine_job(plan, d_s, n_samples, coh_ms, &J);
    if (st != GNSS_OK) {
      cudaFreeAsync(ws, cs);
      return st;
    }
    e = launch_refine(J, (int)n_cand, d_c, (int)max_iter, search_hz, d_o, cs);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_o, n_cand * sizeof(gnss_refined), cudaMemcpyDeviceToHost, cs);
  cudaError_t ef = cudaFreeAsync(ws, cs);
  if (e != cudaSuccess) return cuda_status(e, "gnss_refine");
  if (ef != cudaSuccess) return cuda_status(ef, "cudaFreeAsync");
  if (cs == nullptr) {
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamSynchronize");
  }
  return GNSS_OK;
}

}  // extern "C"

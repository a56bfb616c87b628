// track.cu -- tracking channels (Section 3, Fig. 3) for many satellites or
// hypotheses at once (sm_103a).
//
// A tracking channel shares the front of the acquisition channel -- carrier
// and code NCOs and the first mixing stage -- but correlates in the time
// domain at three code offsets (early, prompt, late) and closes two loops
// around them.  The paper draws the channel as a block diagram; the loop
// design is this library's reading, built the way a hardware receiver builds
// it:
//   NCOs in fixed point: carrier phase Phi (uint32, 2^32 = one cycle) with
//     word Wc = round(f 2^32 / fs); code position P (2^-32 chip, kept in
//     [0, 1023 2^32)) with word Wk = round(f_code 2^32 / fs).
//   Interval k (L = coh_ms N samples): theta_i = Phi + i Wc, u_i = P + i Wk,
//     s_i = x[kL + i] exp(-j 2 pi theta_i / 2^32), and
//     Z_E/P/L = sum s_i c[floor((u_i + h, u_i, u_i - h) / 2^32) mod 1023],
//     h = spacing / 2 chips; replica delay tau_k = (-P / 2^32) mod 1023.
//   Costas PLL: e_phi = atan(Q_P / I_P) / 2 pi; second order, zeta = 1/sqrt 2,
//     w_n = 8 zeta B_pll / (4 zeta^2 + 1): f_int += w_n^2 T e_phi,
//     f = f_int + 2 zeta w_n e_phi.
//   DLL, carrier aided: e_tau = (1 - spacing/2) (|Z_L| - |Z_E|) / (|Z_L| + |Z_E|),
//     f_code = R_c (1 + f / f_L1) - 4 B_dll e_tau, f_L1 = 1540 R_c.
//
// A group of threads per channel -- the whole CTA when there are few
// channels, down to one warp when there are enough to fill the GPU -- runs
// the intervals in order.  Each thread takes a contiguous run of the interval's
// samples in groups of 8: the carrier is started
// from its exact NCO phase for every group (sincospif of the 32-bit phase)
// and rotated by one sample's phase inside it; the code NCO runs in 64-bit
// integers and the three replica chips are read from a 32-chip window of a
// bit table of the PRN's code in shared memory (bit = 1 for chip -1), so the
// +-1 multiplies are sign flips.  Sums are FP32, reduced over the group; the
// group's first thread forms the discriminators (FP32), runs the loop filters
// in double and hands the next interval's NCO words to the group through
// shared memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.h"

namespace gnss {

static constexpr int kTrackThreads = 256;
// Bit table: bit b holds the sign of chip (b - 1) mod 1023, b < 1023 + 64,
// so that a 32-bit window starting at bit k covers chips k - 1 .. k + 30.
static constexpr int kCodeBits = 1023 + 64;
static constexpr int kCodeWords = (kCodeBits + 31) / 32 + 1;

struct TrackJob {
  const uint8_t* samples;  // device recording, 16-byte aligned
  int L;                   // samples per interval (coh_ms N), a multiple of 8 * 256
  int n_int;               // intervals
  double fs;
  const int8_t* codes;     // [P][1023] +-1
  const int* prn_index;    // [33] plan index of PRN 1..32 (-1 = not in the plan)
  uint32_t half;           // early / late offset, 2^-32 chip
  double spacing;          // early-late spacing (chips)
  double wn, zeta, T;      // PLL natural frequency (rad/s), damping, interval (s)
  double b_dll;            // DLL noise bandwidth (Hz)
};

// NCO words of the next interval from the loop outputs; status -2 when the
// carrier or code frequency leaves the range a 32-bit NCO can hold.
__device__ __forceinline__ int track_words(const TrackJob& J, double f, double e_tau, uint32_t* wc, uint32_t* wk) {
  const double rc = 1.023e6;
  const double f_code = rc * (1.0 + f / (1540.0 * rc)) - 4.0 * J.b_dll * e_tau;
  if (!(f_code > 0.0 && f_code < J.fs) || !(fabs(f) < 0.5 * J.fs)) return -2;
  *wc = (uint32_t)llround(f * 4294967296.0 / J.fs);
  *wk = (uint32_t)llround(f_code * 4294967296.0 / J.fs);
  return 0;
}

struct TrackNco {
  int64_t P;      // code position of the interval's first sample (2^-32 chip)
  uint32_t phi;   // carrier phase of the interval's first sample
  uint32_t wc;    // carrier word
  uint32_t wk;    // code word
  int status;     // 0 running; < 0 stopped (record status)
};

// Samples [n0, n0 + 8) as floats (2-bit I/Q: one aligned 4-byte word; int8
// I/Q: one aligned 16-byte load).
template <int FMT>
__device__ __forceinline__ void track_load8(const uint8_t* __restrict__ base, int64_t n0, float (&xi)[8],
                                            float (&xq)[8]) {
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

// exp(-j 2 pi theta / 2^32) for a 32-bit phase: the phase read as a signed
// fraction of half a turn is exact in its top 24 bits.
__device__ __forceinline__ float2 nco_carrier(uint32_t theta) {
  float s, c;
  sincospif((float)(int32_t)theta * (1.f / 2147483648.f), &s, &c);
  return make_float2(c, -s);
}

__device__ __forceinline__ float flip(float v, uint32_t sign_bit) {
  return __int_as_float(__float_as_int(v) ^ (int)sign_bit);
}

// Barrier of one channel's thread group (group lc of the CTA): a warp, a
// named barrier of TPC threads (IDs 1 .. 256 / TPC), or the whole CTA.
template <int TPC>
__device__ __forceinline__ void group_sync(int lc) {
  if constexpr (TPC == 32) __syncwarp();
  else if constexpr (TPC == kTrackThreads) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(1 + lc), "r"(TPC) : "memory");
}

// TPC threads per channel (32: one warp per channel, 8 channels per CTA; 64
// or 128: 4 or 2 channels per CTA; 256: one CTA per channel).
template <int FMT, int TPC>
__global__ void __launch_bounds__(kTrackThreads) k_track(const TrackJob J, const gnss_candidate* __restrict__ chans,
                                                         int n_chan, gnss_track_rec* __restrict__ out) {
  constexpr int CPC = kTrackThreads / TPC;  // channels per CTA
  constexpr int W = TPC / 32;               // warps per channel
  __shared__ uint32_t s_code[CPC][kCodeWords];
  __shared__ float s_red[CPC][6][W];
  __shared__ TrackNco s_nco[CPC];
  const int lc = threadIdx.x / TPC;
  const int t = threadIdx.x % TPC;
  const int c = blockIdx.x * CPC + lc;
  if (c >= n_chan) return;  // whole warps only (TPC = 32 when CPC > 1)
  const gnss_candidate ch = chans[c];
  const int row = (ch.prn >= 1 && ch.prn <= 32) ? __ldg(J.prn_index + ch.prn) : -1;
  gnss_track_rec* rec = out + (size_t)c * J.n_int;
  if (row < 0) {  // PRN not in the plan: every record says so
    for (int k = t; k < J.n_int; k += TPC) {
      gnss_track_rec r = {};
      r.status = -1;
      rec[k] = r;
    }
    return;
  }
  const int8_t* code = J.codes + (size_t)row * 1023;
  uint32_t* tab = s_code[lc];
  for (int w = t; w < kCodeWords; w += TPC) {
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
      const int bit = 32 * w + b;
      if (bit < kCodeBits) {
        const int chip = (bit - 1 + 1023) % 1023;
        if (code[chip] < 0) v |= 1u << b;
      }
    }
    tab[w] = v;
  }
  // the group's first thread owns the loop state
  const double two32 = 4294967296.0;
  const int64_t period = (int64_t)1023 << 32;
  double f_int = ch.f_hz, f = ch.f_hz;
  TrackNco& nco_s = s_nco[lc];
  if (t == 0) {
    int64_t P = llround(-ch.tau_chips * two32) % period;
    if (P < 0) P += period;
    nco_s.P = P;
    nco_s.phi = 0;
    nco_s.status = track_words(J, f, 0.0, &nco_s.wc, &nco_s.wk);
  }
  group_sync<TPC>(lc);
  const int S = J.L / TPC;  // samples per thread, a multiple of 8
  const int i0 = t * S;
  for (int k = 0; k < J.n_int; ++k) {
    const TrackNco nco = nco_s;
    if (nco.status != 0) {  // uniform over the group: every thread read the same word
      if (t == 0)
        for (int kk = k; kk < J.n_int; ++kk) {
          gnss_track_rec r = {};
          r.status = nco.status;
          rec[kk] = r;
        }
      return;
    }
    const float2 rot = nco_carrier(nco.wc);  // one sample's carrier step
    float ze_r = 0.f, ze_i = 0.f, zp_r = 0.f, zp_i = 0.f, zl_r = 0.f, zl_i = 0.f;
    const int64_t nk = (int64_t)k * J.L;
    for (int g = 0; g < S; g += 8) {
      const int i = i0 + g;
      float xi[8], xq[8];
      track_load8<FMT>(J.samples, nk + i, xi, xq);
      float2 car = nco_carrier(nco.phi + (uint32_t)i * nco.wc);
      const int64_t u0 = nco.P + (int64_t)i * nco.wk;
      const uint32_t chip0 = (uint32_t)(u0 >> 32);  // < 1023 (coh + 2)
      const int kc = (int)(chip0 % 1023u);           // chip of the group's first sample
      const uint32_t win = __funnelshift_r(tab[kc >> 5], tab[(kc >> 5) + 1], kc & 31);  // chips kc - 1 ..
      uint64_t acc = (uint32_t)u0;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float sr = xi[e] * car.x - xq[e] * car.y;
        const float si = fmaf(xi[e], car.y, xq[e] * car.x);
        const uint32_t rp = 1u + (uint32_t)(acc >> 32);
        const uint32_t re = 1u + (uint32_t)((acc + J.half) >> 32);
        const uint32_t rl = (uint32_t)((acc + 0x100000000ull - J.half) >> 32);
        const uint32_t mp = (win << (31u - rp)) & 0x80000000u;
        const uint32_t me = (win << (31u - re)) & 0x80000000u;
        const uint32_t ml = (win << (31u - rl)) & 0x80000000u;
        zp_r += flip(sr, mp);
        zp_i += flip(si, mp);
        ze_r += flip(sr, me);
        ze_i += flip(si, me);
        zl_r += flip(sr, ml);
        zl_i += flip(si, ml);
        car = make_float2(car.x * rot.x - car.y * rot.y, fmaf(car.x, rot.y, car.y * rot.x));
        acc += nco.wk;
      }
    }
    // group sums of the six correlator components
    float v[6] = {ze_r, ze_i, zp_r, zp_i, zl_r, zl_i};
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    if constexpr (W > 1) {
      if ((t & 31) == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q) s_red[lc][q][t >> 5] = v[q];
      group_sync<TPC>(lc);
      if (t == 0)
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          float a = 0.f;
          for (int w = 0; w < W; ++w) a += s_red[lc][q][w];
          v[q] = a;
        }
    }
    if (t == 0) {
      // discriminators in FP32, loop state and NCO words in double / integers
      const float ip = v[2], qp = v[3];
      const float e_phi = (ip == 0.f && qp == 0.f) ? 0.f : atanf(qp / ip) * 0.15915494309189535f;
      const float me = hypotf(v[0], v[1]), ml = hypotf(v[4], v[5]);
      const float e_tau = (me + ml > 0.f) ? (float)(1.0 - J.spacing / 2.0) * (ml - me) / (ml + me) : 0.f;
      gnss_track_rec r;
      r.f_hz = (double)(int32_t)nco.wc * J.fs / two32;
      r.tau_chips = (double)(nco.P == 0 ? 0 : period - nco.P) / two32;
      r.ze[0] = v[0];
      r.ze[1] = v[1];
      r.zp[0] = v[2];
      r.zp[1] = v[3];
      r.zl[0] = v[4];
      r.zl[1] = v[5];
      r.e_phi = e_phi;
      r.e_tau = e_tau;
      r.status = 0;
      r.reserved = 0;
      rec[k] = r;
      f_int += J.wn * J.wn * J.T * (double)e_phi;
      f = f_int + 2.0 * J.zeta * J.wn * (double)e_phi;
      int64_t P = nco.P + (int64_t)J.L * nco.wk;
      while (P >= period) P -= period;
      nco_s.P = P;
      nco_s.phi = nco.phi + (uint32_t)J.L * nco.wc;
      nco_s.status = track_words(J, f, (double)e_tau, &nco_s.wc, &nco_s.wk);
    }
    group_sync<TPC>(lc);
  }
}

}  // namespace gnss

using namespace gnss;

extern "C" gnss_status gnss_track(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                  const gnss_candidate* chans_dev, size_t n_chan, const gnss_track_config* cfg,
                                  gnss_track_rec* out_dev, void* stream) {
  if (!plan || !samples_dev || !chans_dev || !cfg || !out_dev) return fail_status(GNSS_EINVAL, "NULL argument");
  if (plan->N < 2048) return fail_status(GNSS_EINVAL, "tracking needs fs >= 2.048 MHz (under one chip per sample)");
  if (cfg->coh_ms < 1 || cfg->coh_ms > 1000) return fail_status(GNSS_EINVAL, "coh_ms must be in [1, 1000]");
  if (cfg->n_int < 1) return fail_status(GNSS_EINVAL, "n_int must be >= 1");
  const size_t L = (size_t)cfg->coh_ms * plan->N;
  if ((size_t)cfg->n_int > n_samples / L) return fail_status(GNSS_EINVAL, "n_int intervals exceed the recording");
  if (L * cfg->n_int > (size_t)INT64_MAX / 4 || L > (size_t)INT32_MAX) return fail_status(GNSS_EINVAL, "recording too long");
  if (!(cfg->spacing_chips > 0.f && cfg->spacing_chips <= 1.f))
    return fail_status(GNSS_EINVAL, "spacing_chips must be in (0, 1]");
  if (!(cfg->pll_bw_hz >= 0.f && cfg->pll_bw_hz <= 1000.f) || !(cfg->dll_bw_hz >= 0.f && cfg->dll_bw_hz <= 1000.f))
    return fail_status(GNSS_EINVAL, "loop bandwidths must be in [0, 1000] Hz");
  if ((uintptr_t)samples_dev & 15u) return fail_status(GNSS_EINVAL, "device samples must be 16-byte aligned");
  if (n_chan == 0) return GNSS_OK;
  if (n_chan > (size_t)INT32_MAX) return fail_status(GNSS_EINVAL, "too many channels");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  TrackJob J;
  J.samples = (const uint8_t*)samples_dev;
  J.L = (int)L;
  J.n_int = (int)cfg->n_int;
  J.fs = (double)plan->desc.fs_hz;
  J.codes = plan->d_codes;
  J.prn_index = plan->d_prn_index;
  J.spacing = (double)cfg->spacing_chips;
  J.half = (uint32_t)llround(J.spacing * 0.5 * 4294967296.0);
  J.zeta = 1.0 / sqrt(2.0);
  J.wn = 8.0 * J.zeta * (double)cfg->pll_bw_hz / (4.0 * J.zeta * J.zeta + 1.0);
  J.T = (double)L / J.fs;
  J.b_dll = (double)cfg->dll_bw_hz;
  cudaStream_t cs = (cudaStream_t)stream;
  // Threads per channel: the smallest power of two (32 .. 256) that gives the
  // channels together the GPU's resident threads (1024 per SM at 64
  // registers), since a channel's intervals run in order and only more
  // threads per channel shorten them.  1280 channels on 148 SMs: 128 (13.1
  // ms per launch against 18.2 ms with one warp per channel and 13.5 ms
  // with one CTA per channel).
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device);
  const int n = (int)n_chan;
  int tpc = 32;
  while (tpc < kTrackThreads && (size_t)tpc * n_chan < (size_t)sms * 1024) tpc *= 2;
  const unsigned grid = (unsigned)((n_chan + (kTrackThreads / tpc) - 1) / (kTrackThreads / tpc));
  if (plan->desc.format == GNSS_FMT_2BIT_IQ) {
    if (tpc == 32) k_track<GNSS_FMT_2BIT_IQ, 32><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
    else if (tpc == 64) k_track<GNSS_FMT_2BIT_IQ, 64><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
    else if (tpc == 128) k_track<GNSS_FMT_2BIT_IQ, 128><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
    else k_track<GNSS_FMT_2BIT_IQ, kTrackThreads><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
  } else {
    if (tpc == 32) k_track<GNSS_FMT_I8_IQ, 32><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
    else if (tpc == 64) k_track<GNSS_FMT_I8_IQ, 64><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
    else if (tpc == 128) k_track<GNSS_FMT_I8_IQ, 128><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
    else k_track<GNSS_FMT_I8_IQ, kTrackThreads><<<grid, kTrackThreads, 0, cs>>>(J, chans_dev, n, out_dev);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "gnss_track");
  return GNSS_OK;
}

// acq.cu -- acquisition kernels (Section 3, Fig. 2) for sm_103a.
//
//   k_gold         G1/G2 LFSR Gold codes (code NCO input), bit-exact
//   k_code_spectra replica sampling at fs + forward FFT -> resident C_p
//   k_fold         2-bit / int8 I/Q unpack and coherent fold of T_coh ms with
//                  the per-millisecond carrier factor, once per group of
//                  Doppler bins sharing f mod 1000          (first mixing)
//   k_carrier_fft  per-bin carrier wipe-off + forward FFT: Y_{f,b}
//   k_xcorr        Y * conj(C_p), IFFT, |.|^2, non-coherent accumulation over
//                  blocks in registers, per-row peak statistics, and in the
//                  last CTA of each PRN the peak / second peak / ratio
//                  detection                  (second mixing + IFFT + detection)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cooperative_groups.h>
#include <mutex>

#include "fft.cuh"
#include "internal.h"
#include "xcorr.cuh"

namespace gnss {

// ---------------------------------------------------------------------------
// K1: Gold codes.  Two-tap G2 phase selector per PRN (IS-GPS-200 Table 3-Ia).
// Register bit s-1 holds stage s; the output is stage 10.
// ---------------------------------------------------------------------------
__constant__ uint8_t c_phase_sel[32][2] = {
    {2, 6}, {3, 7}, {4, 8}, {5, 9}, {1, 9}, {2, 10}, {1, 8}, {2, 9}, {3, 10}, {2, 3}, {3, 4},
    {5, 6}, {6, 7}, {7, 8}, {8, 9}, {9, 10}, {1, 4}, {2, 5}, {3, 6}, {4, 7}, {5, 8}, {6, 9},
    {1, 3}, {4, 6}, {5, 7}, {6, 8}, {7, 9}, {8, 10}, {1, 6}, {2, 7}, {3, 8}, {4, 9}};

__global__ void k_gold(const int* __restrict__ prns, int8_t* __restrict__ codes) {
  __shared__ uint8_t bits[1023];
  const int p = blockIdx.x;
  if (threadIdx.x == 0) {
    const int prn = prns[p];
    const int a = c_phase_sel[prn - 1][0] - 1, b = c_phase_sel[prn - 1][1] - 1;
    uint32_t g1 = 0x3FFu, g2 = 0x3FFu;
    for (int i = 0; i < 1023; ++i) {
      const uint32_t out1 = (g1 >> 9) & 1u;
      const uint32_t out2 = ((g2 >> a) ^ (g2 >> b)) & 1u;
      bits[i] = (uint8_t)(out1 ^ out2);
      const uint32_t fb1 = ((g1 >> 2) ^ (g1 >> 9)) & 1u;                                       // x^3, x^10
      const uint32_t fb2 = ((g2 >> 1) ^ (g2 >> 2) ^ (g2 >> 5) ^ (g2 >> 7) ^ (g2 >> 8) ^ (g2 >> 9)) & 1u;  // x^2,3,6,8,9,10
      g1 = ((g1 << 1) | fb1) & 0x3FFu;
      g2 = ((g2 << 1) | fb2) & 0x3FFu;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 1023; i += blockDim.x) codes[p * 1023 + i] = (int8_t)(1 - 2 * (int)bits[i]);
}


// ---------------------------------------------------------------------------
// K1b: code spectra.  Thread j builds the replica samples j + T r directly
// (c_s[m] = c[floor(m * 1023 / N)]) and transforms them in place.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Cfg<N>::T) k_code_spectra(const int8_t* __restrict__ codes,
                                                           float2* __restrict__ cspec) {
  constexpr int E = Cfg<N>::E, T = Cfg<N>::T;
  extern __shared__ __align__(16) float2 sm[];
  float2* buf0 = sm;
  float2* buf1 = Cfg<N>::DB ? sm + FftShape<N>::smem_elems : sm;
  const int p = blockIdx.x, j = threadIdx.x;
  float2 v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int m = j + T * r;
    v[r] = make_float2((float)codes[p * 1023 + (int)(((int64_t)m * 1023) / N)], 0.f);
  }
  int phase = 0;
  fft_block<N, E, false, Cfg<N>::DB>(v, j, buf0, buf1, phase);
#pragma unroll
  for (int r = 0; r < E; ++r) cspec[(size_t)p * N + j + T * r] = v[r];
}

// ---------------------------------------------------------------------------
// K2+K3: unpack, carrier wipe-off, coherent fold, forward FFT.
//
// With n = bL + iN + m the wipe-off phase splits exactly as
//   f n / fs = f (bL + m) / fs + f i / 1000        (N / fs = 1 ms),
// so y[m] = exp(-j 2 pi ((f (bL+m)) mod fs)/fs) * sum_i x[n] w_i with the
// per-millisecond constant w_i = exp(-j 2 pi ((f i) mod 1000) / 1000), which
// depends on f only through f mod 1000.  The fold sum is therefore computed
// once per group of bins with the same f mod 1000 (k_fold; vector loads of
// 8 or 16 bytes of 2-bit data, 32 or 64 bytes of int8 per thread and
// millisecond), and each bin applies only its own carrier before the FFT
// (k_carrier_fft).
// ---------------------------------------------------------------------------
template <int E, int FMT>
__device__ __forceinline__ void load_ms(const uint8_t* __restrict__ base, int64_t n0, float (&xi)[E],
                                        float (&xq)[E]) {
  if constexpr (FMT == GNSS_FMT_2BIT_IQ) {
    // E samples = E/2 bytes; sample e: bits [4e, 4e+4) of the little-endian words
    const uint32_t* w = reinterpret_cast<const uint32_t*>(base + n0 / 2);
    uint32_t words[E >= 8 ? E / 8 : 1];
    if constexpr (E == 4) {
      words[0] = __ldg(reinterpret_cast<const uint16_t*>(w));
    } else if constexpr (E == 8) {
      words[0] = __ldg(w);
    } else if constexpr (E == 16) {
      const uint2 t = __ldg(reinterpret_cast<const uint2*>(w));
      words[0] = t.x;
      words[1] = t.y;
    } else {
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(w));
      words[0] = t.x;
      words[1] = t.y;
      words[2] = t.z;
      words[3] = t.w;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t word = words[e / 8];
      const int sh = 4 * (e % 8);
      // code c in 0..3 -> float c exactly via the 2^23 mantissa trick
      xi[e] = __int_as_float(0x4B000000 | ((word >> sh) & 3u)) - 8388608.f;
      xq[e] = __int_as_float(0x4B000000 | ((word >> (sh + 2)) & 3u)) - 8388608.f;
    }
  } else if constexpr (E == 4) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(reinterpret_cast<const int8_t*>(base) + 2 * n0));
    const uint32_t wv[2] = {t.x, t.y};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      xi[2 * k] = (float)(int8_t)(wv[k] & 0xFF);
      xq[2 * k] = (float)(int8_t)((wv[k] >> 8) & 0xFF);
      xi[2 * k + 1] = (float)(int8_t)((wv[k] >> 16) & 0xFF);
      xq[2 * k + 1] = (float)(int8_t)((wv[k] >> 24) & 0xFF);
    }
  } else {
    const int8_t* s = reinterpret_cast<const int8_t*>(base) + 2 * n0;
#pragma unroll
    for (int c = 0; c < E / 8; ++c) {
      const uint4 t = __ldg(reinterpret_cast<const uint4*>(s) + c);
      const uint32_t wv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = 8 * c + 2 * k;
        xi[e] = (float)(int8_t)(wv[k] & 0xFF);
        xq[e] = (float)(int8_t)((wv[k] >> 8) & 0xFF);
        xi[e + 1] = (float)(int8_t)((wv[k] >> 16) & 0xFF);
        xq[e + 1] = (float)(int8_t)((wv[k] >> 24) & 0xFF);
      }
    }
  }
}

// k_fold: z_g[m] = sum_i x[bL + iN + m] w_i for every fold group g and block b,
// with w_i = exp(-j 2 pi ((rho_g i) mod 1000) / 1000), rho_g = f mod 1000 of
// the Doppler bins of the group (all bins share one group when T_coh = 1).
// Each thread folds 4 consecutive samples (one 2-byte load of 2-bit data or
// one 8-byte load of int8 per millisecond: short per-thread chains, many
// warps, since the fold is latency-bound); FoldCfg<N>::CPB CTAs of
// FoldCfg<N>::T threads cover one (g, b).  Output in natural order.  CTA 0
// also clears the per-PRN completion counters of k_xcorr.
template <int N>
struct FoldCfg {
  static constexpr int E = 4;
  static constexpr int T = N / E < 128 ? N / E : 128;
  static constexpr int CPB = N / (E * T);  // CTAs per (group, block)
};

// exp(-j 2 pi k / 1000), k < 1000: the per-millisecond wipe-off factors
// w_i = c_root1000[(rho i) mod 1000], computed in double on the host and
// rounded once; every lane of a CTA reads the same entry (a broadcast).
__constant__ float2 c_root1000[1000];

cudaError_t ensure_fold_roots() {
  static std::mutex mu;
  static bool done[128];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  float2 h[1000];
  for (int k = 0; k < 1000; ++k) {
    const double ang = 2.0 * M_PI * (double)k / 1000.0;
    h[k] = make_float2((float)cos(ang), (float)-sin(ang));
  }
  e = cudaMemcpyToSymbol(c_root1000, h, sizeof(h));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// Fold of E consecutive samples starting at n_first (ms 0 of the block) over
// coh milliseconds: z[e] = sum_i x[n_first + i N + e] w_i.  For 2-bit data
// x = 2c - 3(1 + j): fold 2c w, then subtract 3(1 + j) sum(w).
template <int N, int E, int FMT>
__device__ __forceinline__ void fold_samples(const uint8_t* __restrict__ samples, int64_t n_first, int coh, int rho,
                                             float (&ar)[E], float (&ai)[E]) {
#pragma unroll
  for (int e = 0; e < E; ++e) ar[e] = ai[e] = 0.f;
  float wsum_r = 0.f, wsum_i = 0.f;
#pragma unroll 10
  for (int i = 0; i < coh; ++i) {
    const float2 w = c_root1000[(int)(((int64_t)rho * i) % 1000)];
    const float ws = w.y, wc = w.x;
    float xi[E], xq[E];
    load_ms<E, FMT>(samples, n_first + (int64_t)i * N, xi, xq);
    float wr = wc, wi = ws;
    if constexpr (FMT == GNSS_FMT_2BIT_IQ) {
      wr *= 2.f;
      wi *= 2.f;
      wsum_r += wc;
      wsum_i += ws;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      ar[e] = fmaf(xi[e], wr, ar[e]);
      ar[e] = fmaf(-xq[e], wi, ar[e]);
      ai[e] = fmaf(xi[e], wi, ai[e]);
      ai[e] = fmaf(xq[e], wr, ai[e]);
    }
  }
  if constexpr (FMT == GNSS_FMT_2BIT_IQ) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      ar[e] = fmaf(-3.f, wsum_r - wsum_i, ar[e]);  // (1 + j)(wr + j wi) = (wr - wi) + j (wr + wi)
      ai[e] = fmaf(-3.f, wsum_r + wsum_i, ai[e]);
    }
  }
}

template <int N, int FMT>
__device__ __forceinline__ void fold_tile(const FoldArgs& a, int tile) {
  constexpr int E = FoldCfg<N>::E, T = FoldCfg<N>::T, CPB = FoldCfg<N>::CPB;
  griddep_release();
  const int B = a.B;
  const int gb = tile / CPB;             // g * B + b
  const int m0 = E * ((tile % CPB) * T + threadIdx.x);
  const int g = gb / B, b = gb % B;
  if (a.counters != nullptr && tile == 0)
    for (int p = threadIdx.x; p <= a.P; p += T) a.counters[p] = 0u;  // and the status word
  float ar[E], ai[E];
  fold_samples<N, E, FMT>(a.samples, (int64_t)b * a.coh * N + m0, a.coh, a.gkey[g], ar, ai);
  float4* out = reinterpret_cast<float4*>(a.Z + ((size_t)gb * N + m0));
#pragma unroll
  for (int e = 0; e < E; e += 2) out[e / 2] = make_float4(ar[e], ai[e], ar[e + 1], ai[e + 1]);
}


template <int N, int FMT>
__global__ void __launch_bounds__(FoldCfg<N>::T) k_fold(const FoldArgs a) {
  fold_tile<N, FMT>(a, blockIdx.x);
}

template <int N, int FMT>
__global__ void __launch_bounds__(FoldCfg<N>::T) k_fold_batch(const BatchReq* __restrict__ reqs,
                                                             const uint32_t* __restrict__ base, int n) {
  const int r = find_request(base, n);
  fold_tile<N, FMT>(reqs[r].fold, (int)(blockIdx.x - __ldg(base + r)));
}

// Code-Doppler shift of block b of bin f (GNSS_CODE_DOPPLER), in samples:
// sigma = floor(f b L / f_L1 + 1/2), f_L1 = 1540 x 1.023 MHz, as the floor of
// (2 f b L + f_L1) / (2 f_L1) in exact 64-bit integer arithmetic.
__device__ __forceinline__ int64_t code_doppler_sigma(int f, int b, int64_t L) {
  constexpr int64_t kL1 = 1540LL * 1023000LL;
  const int64_t num = 2 * (int64_t)f * b * L + kL1, den = 2 * kL1;
  int64_t q = num / den;
  if (num % den != 0 && num < 0) --q;
  return q;
}

// k_carrier_fft: one CTA per (Doppler d, block b), tile = d * B + b -- or per
// (spectrum class, block) when bins a whole number of kHz apart share one
// spectrum (the correlate kernel reads it shifted).  Loads the
// folded block of its group in the FFT's register layout, multiplies by the
// carrier exp(-j 2 pi ((f (bL + m)) mod fs) / fs) -- exact integer phase for
// r = 0, then a rotation by T samples per r -- and runs the forward FFT:
// Y_{f,b} = FFT_N(y_{f,b}).  Element n = j + T r holds sample m = (n + sh)
// mod N of the block: sh = 0, or (-sigma_b) mod N with GNSS_CODE_DOPPLER
// (the rotation y'[n] = y[(n - sigma_b) mod N]).  The carrier chain runs over
// the unwrapped m' = n + sh < 2N; a wrapped sample m = m' - N sits N samples
// earlier, so its carrier is the chain's value times exp(+j 2 pi f N / fs).
template <int N>
__device__ __forceinline__ void carrier_tile(const CarrierArgs& a, int tile, float2* sm) {
  constexpr int E = Cfg<N>::E, T = Cfg<N>::T;
  griddep_release();
  float2* buf0 = sm;
  float2* buf1 = Cfg<N>::DB ? sm + FftShape<N>::smem_elems : sm;
  const int fs = a.fs, coh = a.coh, B = a.B;
  const int j = threadIdx.x;
  const int d = tile / B, b = tile % B;  // d: a bin, or a spectrum class
  const int f = a.cls_fgroup ? a.cls_base[d] : a.dopp_min + d * a.dopp_step;
  const float2* z = a.Z + ((size_t)(a.cls_fgroup ? a.cls_fgroup[d] : a.group[d]) * B + b) * N;
  int sh = 0;
  if (a.code_dopp) sh = (int)(((-code_doppler_sigma(f, b, (int64_t)coh * N)) % N + N) % N);
  const int64_t fr = (((int64_t)f % fs) + fs) % fs;
  const int64_t r0 = (fr * ((int64_t)b * coh * N + j + sh)) % fs;
  const int64_t rs = (fr * T) % fs;
  const float inv_fs = 1.f / (float)fs;
  float s0, c0, ss, sc;
  sincospif(-2.f * (float)r0 * inv_fs, &s0, &c0);
  sincospif(-2.f * (float)rs * inv_fs, &ss, &sc);
  float2 car = make_float2(c0, s0);
  const float2 step = make_float2(sc, ss);
  griddep_wait();  // the fold kernel's blocks are complete and visible
  float2 v[E];
  if (sh == 0) {  // uniform over the CTA
#pragma unroll
    for (int r = 0; r < E; ++r) {
      v[r] = c_mul(__ldg(z + j + T * r), car);
      car = c_mul(car, step);
    }
  } else {
    const int64_t rw = (fr * N) % fs;
    float sw, cw;
    sincospif(2.f * (float)rw * inv_fs, &sw, &cw);
    const float2 unwrap = make_float2(cw, sw);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int m = j + sh + T * r;
      const bool wrapped = m >= N;
      v[r] = c_mul(__ldg(z + (wrapped ? m - N : m)), wrapped ? c_mul(car, unwrap) : car);
      car = c_mul(car, step);
    }
  }
  int phase = 0;
  fft_block<N, E, false, Cfg<N>::DB>(v, j, buf0, buf1, phase);
  float2* out = a.Y + (size_t)tile * N;
#pragma unroll
  for (int r = 0; r < E; ++r) out[j + T * r] = v[r];
}

template <int N>
__global__ void __launch_bounds__(Cfg<N>::T) k_carrier_fft(const CarrierArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  carrier_tile<N>(a, blockIdx.x, sm);
}

template <int N>
__global__ void __launch_bounds__(Cfg<N>::T) k_carrier_fft_batch(const BatchReq* __restrict__ reqs,
                                                                const uint32_t* __restrict__ base, int n) {
  extern __shared__ __align__(16) float2 sm[];
  const int r = find_request(base, n);
  carrier_tile<N>(reqs[r].car, (int)(blockIdx.x - __ldg(base + r)), sm);
}


// ---------------------------------------------------------------------------
// TMA staging of the next block's spectrum (the staged correlate variant):
// one thread issues a bulk copy (cp.async.bulk) of the N-point row into a
// shared-memory stage, completing on an mbarrier, while the CTA transforms
// the current block; the CTA waits on the barrier's phase before it reads
// the stage.  Every wait is bounded.  The CTA agrees on each wait's outcome;
// once one has given up it issues no further copy, reads the rest of its
// spectra from global memory (the results stay complete), sets the call's
// status word (the records' GNSS_DET_STAGE_TIMEOUT flag) and, before it
// leaves, waits once more, with the full bound, for the one copy in flight.
// ---------------------------------------------------------------------------
// try_wait polls of one wait before it gives up (lowered only by the testing
// entry point, which makes every wait give up at once)
__device__ unsigned g_stage_wait_limit = 1u << 22;
constexpr unsigned kStageDrainLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void stage_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One thread: the stage's previous contents were read by every thread before
// a CTA barrier that this thread has passed; order those generic-proxy reads
// before the async-proxy writes, then arm the barrier and copy.
__device__ __forceinline__ void stage_issue(float2* stg, const float2* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(stg)),
               "l"(src), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ bool stage_wait(uint64_t* mbar, uint32_t parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

struct StageIssue {
  float2* stg;
  const float2* src;  // nullptr: no next block
  uint64_t* mbar;
  uint32_t bytes;
  int j;
  __device__ __forceinline__ void operator()() const {
    if (j == 0 && src != nullptr) stage_issue(stg, src, bytes, mbar);
  }
};

// ---------------------------------------------------------------------------
// K4: correlate.  One CTA per (PRN p, Doppler d), tile = d * P + p; CTAs that
// share d are adjacent, so the spectra of one Doppler bin are read from L2
// while they are hot.  The CTA runs its sets one after the other (with
// half-bit sets: the even blocks, then the odd blocks), accumulating |R|^2
// of the set in registers, so one accumulator serves both sets.
// ---------------------------------------------------------------------------
// One block: Y * conj(C_p) -> IFFT -> |.|^2 added to acc.  Without staging
// Y is read from L2; with staging it is read from the shared-memory stage
// (once the stage's barrier phase has completed) and the copy of the next
// block is issued after the IFFT's first barrier.
template <int N, int E, bool DB, bool TWC, bool ST, bool CL>
__device__ __forceinline__ void corr_block(const float2* __restrict__ y, int ksh, const float2* __restrict__ cp,
                                           int j, float2* buf0, float2* buf1, int& phase, FftTw<N, E, true>& tw,
                                           float (&acc)[E], const StageIssue& next, uint32_t& parity,
                                           bool& stage_ok) {
  constexpr int T = N / E;
  constexpr bool SHACC = XCfg<N, E, ST, CL>::SHACC;
  const int js = j + ksh;  // element k of the bin's spectrum is element k + ksh of the row
  if constexpr (TWC) tw.launder();
  // Re-read the code spectrum from L1 every block: hoisting these 16 loads
  // out of the block loop would pin 32 registers and force spills.
  asm volatile("" : "+l"(cp));
  float2 v[E];
  if constexpr (ST) {
    // this block's copy: waited for while the copies are in step; the CTA
    // agrees on the outcome, so every thread reads the same source and the
    // issuing thread stops with the others
    bool landed = false;
    if (stage_ok) {
      landed = __syncthreads_and(stage_wait(next.mbar, parity, g_stage_wait_limit)) != 0;
      if (landed) parity ^= 1u;  // else the copy in flight still owes phase 'parity'
      else stage_ok = false;
    }
    const float2* src = landed ? next.stg : y;  // the stage, or the row itself from L2
    // ksh < 16 <= T (spectrum classes are cut so): only the last element can wrap
    const float2* ys = src + js;
#pragma unroll
    for (int r = 0; r < E - 1; ++r) v[r] = c_mulconj(ys[T * r], __ldg(cp + j + T * r));
    const int last = js + T * (E - 1);
    v[E - 1] = c_mulconj(src[last >= N ? last - N : last], __ldg(cp + j + T * (E - 1)));
    StageIssue issue = next;
    if (!stage_ok) issue.src = nullptr;  // no copy after a wait gave up
    fft_block_tw<N, E, true, DB>(v, j, buf0, buf1, phase, tw, issue);
  } else {
    // Y streams from L2 (not kept in L1); the code spectrum goes through the
    // non-coherent path (measured: it too is served from L2, and loads that
    // allocate in L1 ran slower, their hits using the data path the exchanges load).
    // ksh < 16 <= T (spectrum classes are cut so): only the last element can wrap
    const float2* ys = y + js;
#pragma unroll
    for (int r = 0; r < E - 1; ++r) v[r] = c_mulconj(__ldcg(ys + T * r), __ldg(cp + j + T * r));
    const int last = js + T * (E - 1);
    v[E - 1] = c_mulconj(__ldcg(y + (last >= N ? last - N : last)), __ldg(cp + j + T * (E - 1)));
    if constexpr (CL) {
      // one buffer per block, alternating: the next block's first-pass stores
      // go to the other buffer, so no barrier guards this block's last reads
      fft_class_local<N, true>(v, j, phase ? buf1 : buf0, tw);
      phase ^= 1;
    } else if constexpr (TWC) {
      fft_block_tw<N, E, true, DB>(v, j, buf0, buf1, phase, tw);
    } else {
      fft_block<N, E, true, DB>(v, j, buf0, buf1, phase);
    }
  }
  if constexpr (SHACC) {
    float* sacc = reinterpret_cast<float*>(reinterpret_cast<char*>(buf0) + XCfg<N, E, ST, CL>::sacc_off) + j;
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, acc[r]));
#pragma unroll
    for (int r = 8; r < E; ++r) sacc[(r - 8) * T] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, sacc[(r - 8) * T]));
  } else {
#pragma unroll
    for (int r = 0; r < E; ++r) acc[r] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, acc[r]));
  }
}


template <int N, int E, bool HALF, bool ST, bool CL>
__device__ __forceinline__ void xcorr_tile(const XcorrArgs& a, int tile, float2* sm) {
  using X = XCfg<N, E, ST, CL>;
  constexpr int T = X::T;
  constexpr bool DB = X::DB, TWC = X::TWC;
  constexpr int S = HALF ? 2 : 1;
  static_assert(!ST || TWC, "staging is built with cached twiddles");
  float2* buf0 = sm;
  float2* buf1 = (DB || CL) ? sm + X::buf_bytes / sizeof(float2) : sm;
  __shared__ float s_val[32];
  __shared__ uint32_t s_idx[32];
  __shared__ unsigned s_last;
  __shared__ __align__(8) uint64_t s_mbar;
  const int j = threadIdx.x;
  // thread j ends each transform holding |R|^2 of phases PhaseMap::at(jo, r)
  const int jo = CL ? ClassLocal<(CL ? N : 4096)>::perm(j) : j;
  const int p = tile % a.P, d = a.bin_order ? __ldg(a.bin_order + tile / a.P) : tile / a.P;
  const float2* cp = a.cspec + (size_t)p * N;
  // bin d's spectrum: its own row, or its class's row read K bins further
  // (Y_{f + 1000 K}[k] = Y_f[k + K]: a whole kHz is one bin of a 1 ms FFT)
  const float2* yd = a.Y + (size_t)(a.bin_cls ? __ldg(a.bin_cls + d) : d) * a.B * N;
  const int ksh = a.bin_shift ? __ldg(a.bin_shift + d) : 0;
  StageIssue next{reinterpret_cast<float2*>(reinterpret_cast<char*>(sm) + X::stage_off), nullptr, &s_mbar,
                  (uint32_t)(sizeof(float2) * N), j};
  uint32_t parity = 0;
  bool stage_ok = true;
  FftTw<N, E, true> tw;
  // the first pass has no twiddles; later passes run butterfly jo
  if constexpr (CL) ClassLocal<(CL ? N : 4096)>::init_twiddles(tw, jo);
  else if constexpr (TWC) tw.init(jo);
  griddep_wait();  // the spectra and the cleared counters are complete and visible
  if constexpr (ST) {
    if (j == 0) stage_init(&s_mbar);
    __syncthreads();
    if (j == 0) stage_issue(next.stg, yd, next.bytes, &s_mbar);  // block 0 of set 0
  }
  int phase = 0;
#pragma unroll 1
  for (int set = 0; set < S; ++set) {
    float acc[E];
#pragma unroll
    for (int r = 0; r < E; ++r) acc[r] = 0.f;
    float* const sacc = reinterpret_cast<float*>(reinterpret_cast<char*>(sm) + X::sacc_off) + j;
    if constexpr (X::SHACC) {
#pragma unroll
      for (int r = 8; r < E; ++r) sacc[(r - 8) * T] = 0.f;  // this thread's own slots
    }
    for (int b = set; b < a.B; b += S) {
      if constexpr (ST) {
        // the block after b: the next of this set, else the first of the next set
        int nb = b + S;
        if (nb >= a.B) nb = set + 1 < S ? set + 1 : a.B;
        next.src = nb < a.B ? yd + (size_t)nb * N : nullptr;
      }
      corr_block<N, E, DB, TWC, ST, CL>(yd + (size_t)b * N, ksh, cp, j, buf0, buf1, phase, tw, acc, next,
                                        parity, stage_ok);
    }
    if constexpr (X::SHACC) {
#pragma unroll
      for (int r = 8; r < E; ++r) acc[r] = sacc[(r - 8) * T];
    }
    // R = IFFT / N, so |R|^2 = |.|^2 / N^2 (an exact power of two)
    constexpr float sc = 1.f / ((float)N * (float)N);
#pragma unroll
    for (int r = 0; r < E; ++r) acc[r] *= sc;
    if (a.surface != nullptr) {
      float* row = a.surface + (((size_t)set * a.P + p) * a.D + d) * (size_t)N;
#pragma unroll
      for (int r = 0; r < E; ++r) row[PhaseMap<N, E, CL>::at(jo, r)] = acc[r];
    }
    row_stats<N, E, CL>(acc, jo, a.excl, s_val, s_idx, a.rows + ((size_t)set * a.P + p) * a.D + d);
  }
  if constexpr (ST) {
    // stage_ok is uniform.  After a wait that gave up, one copy may still be
    // in flight (the one that owes phase 'parity'; none was issued after it):
    // report the call and wait for that copy with the full bound before the
    // CTA's shared memory is released.  The status word is ordered before
    // this CTA's count below by thread 0's fence.
    if (!stage_ok && j == 0) {
      atomicOr(a.counters + a.P, (unsigned)GNSS_DET_STAGE_TIMEOUT);
      stage_wait(&s_mbar, parity, kStageDrainLimit);
    }
  }
  // The last CTA of PRN p (of its D Doppler rows) runs the detection.  The
  // CTA barrier orders every row and surface write of this CTA before thread
  // 0's fence and count (release); the CTA that counts last fences before
  // reading the other CTAs' rows (acquire).
  __syncthreads();
  if (a.second_whole) {
    // the whole-surface second peak scans D N cells per set: all threads
    if (j == 0) {
      __threadfence();
      s_last = (atomicAdd(a.counters + p, 1u) == (unsigned)(a.D - 1)) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finalize_prn<N, T>(a, p, S, s_val, s_idx);
    }
    return;
  }
  // otherwise warp 0 alone counts and detects; the other warps leave now
  if (j >= 32) return;
  unsigned last = 0;
  if (j == 0) {
    __threadfence();
    last = (atomicAdd(a.counters + p, 1u) == (unsigned)(a.D - 1)) ? 1u : 0u;
  }
  if (__shfl_sync(0xffffffffu, last, 0)) {
    __threadfence();
    finalize_prn<N, 32>(a, p, S, s_val, s_idx);
  }
}

template <int N, int E, bool HALF, bool ST, bool CL>
__global__ void __launch_bounds__(XCfg<N, E, ST, CL>::T, XCfg<N, E, ST, CL>::MINB) k_xcorr(const XcorrArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  xcorr_tile<N, E, HALF, ST, CL>(a, blockIdx.x, sm);
}

template <int N, int E, bool HALF, bool ST, bool CL>
__global__ void __launch_bounds__(XCfg<N, E, ST, CL>::T, XCfg<N, E, ST, CL>::MINB)
    k_xcorr_batch(const BatchReq* __restrict__ reqs, const uint32_t* __restrict__ base, int n) {
  extern __shared__ __align__(16) float2 sm[];
  const int r = find_request(base, n);
  xcorr_tile<N, E, HALF, ST, CL>(reqs[r].xc, (int)(blockIdx.x - __ldg(base + r)), sm);
}

// ---------------------------------------------------------------------------
// N = 16384 over a cluster of two CTAs (the split correlate variant).  The
// inverse FFT of Section 3 is split once by decimation in time: with
// x = Y conj(C) and M = N / 2,
//   X[2q + h] = sum_{k < M} z_h[k] e^{2 pi i k q / M},
//   z_0[k] = x[k] + x[k + M],   z_1[k] = (x[k] - x[k + M]) e^{2 pi i k / N},
// so CTA h of the pair (its rank in the cluster) sums |X[2q + h]|^2 with the
// 8192-point class-local transform: 16 accumulators per thread and no spills,
// where one 16384-point CTA holds 32 elements and 32 sums per thread.  Each
// CTA reads both halves of Y, and C's lower half (the upper one through its
// Hermitian symmetry), and forms the products it needs (handing the halves
// over through distributed shared memory instead took two cluster barriers
// per block and ran 40% slower).  Offered to the autotuner; the default at
// 16384 is the 32-per-thread form.  The pair merges its row
// statistics through distributed shared memory: the row's peak and the
// smallest phase holding it, then each half's maximum outside the band
// around that phase.
// ---------------------------------------------------------------------------
// cos(pi m / 16), 0 <= m <= 8 (mathematical constants)
__device__ __forceinline__ float cos_pi16(int m) {
  return m == 0 ? 1.f
       : m == 1 ? 0.98078528040323044913f
       : m == 2 ? 0.92387953251128675613f
       : m == 3 ? 0.83146961230254523708f
       : m == 4 ? 0.70710678118654752440f
       : m == 5 ? 0.55557023301960222474f
       : m == 6 ? 0.38268343236508977173f
       : m == 7 ? 0.19509032201612826785f
                : 0.f;
}
// e^{i pi r / 16}, 0 <= r < 16
__device__ __forceinline__ float2 rot32(int r) {
  return r <= 8 ? make_float2(cos_pi16(r), cos_pi16(8 - r)) : make_float2(-cos_pi16(16 - r), cos_pi16(r - 8));
}

struct SplitCfg {
  static constexpr int N = 16384, M = 8192, T = 512;
  static constexpr size_t smem = 2 * sizeof(float2) * ClassLocal<M>::smem_elems;  // ping-pong exchange buffers
};

// One block: thread j forms z_h at k = j + 512 r (the 8192-point input
// layout; e^{2 pi i k / N} = wj e^{i pi r / 16}, wj = e^{2 pi i j / N}),
// transforms it and adds |.|^2.  Only the last element of the upper half can
// wrap around the row (ksh < 16).  The replica is real, so its spectrum is
// Hermitian: conj(C[k + M]) = C[M - k], and a CTA reads only C[0 .. M]
// (64 KB, resident in L1 beside the exchange buffers) instead of all of C.
template <int H>
__device__ __forceinline__ void split_block(const float2* __restrict__ y, int ksh, const float2* __restrict__ cp,
                                            int j, float2* buf, FftTw<8192, 16, true>& tw, float2 wj,
                                            float (&acc)[16]) {
  constexpr int N = SplitCfg::N, M = SplitCfg::M, T = SplitCfg::T;
  tw.launder();
  asm volatile("" : "+l"(cp));
  const float2* ys = y + j + ksh;
  const float2* cs = cp + j;
  float2 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const float2 lo = c_mulconj(__ldcg(ys + T * r), __ldg(cs + T * r));
    const int kb = j + ksh + T * r + M;
    const float2 hi = c_mul(__ldcg(y + (r < 15 || kb < N ? kb : kb - N)), __ldg(cp + M - j - T * r));
    if constexpr (H == 0) v[r] = c_add(lo, hi);
    else v[r] = c_mul(c_sub(lo, hi), c_mul(wj, rot32(r)));
  }
  fft_class_local<M, true>(v, j, buf, tw);
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, acc[r]));
}

template <bool HALF>
__device__ __forceinline__ void xcorr_tile_split(const XcorrArgs& a, int tile, float2* sm) {
  namespace cg = cooperative_groups;
  constexpr int N = SplitCfg::N, M = SplitCfg::M, T = SplitCfg::T;
  constexpr int S = HALF ? 2 : 1;
  cg::cluster_group cluster = cg::this_cluster();
  const int h = (int)cluster.block_rank();  // the parity of the phases this CTA sums
  float2* buf0 = sm;
  float2* buf1 = sm + ClassLocal<M>::smem_elems;
  __shared__ float s_val[32];
  __shared__ uint32_t s_idx[32];
  __shared__ float s_peak, s_sec;  // read by the other CTA of the pair
  __shared__ uint32_t s_tau;
  const int j = threadIdx.x;
  const int jo = ClassLocal<M>::perm(j);  // thread j ends holding X_h[out_index(jo, r)]
  const int p = tile % a.P, d = a.bin_order ? __ldg(a.bin_order + tile / a.P) : tile / a.P;
  const float2* cp = a.cspec + (size_t)p * N;
  const float2* yd = a.Y + (size_t)(a.bin_cls ? __ldg(a.bin_cls + d) : d) * a.B * N;
  const int ksh = a.bin_shift ? __ldg(a.bin_shift + d) : 0;
  FftTw<M, 16, true> tw;
  ClassLocal<M>::init_twiddles(tw, jo);
  float2 wj;
  sincospif(2.f * (float)j / (float)N, &wj.y, &wj.x);
  griddep_wait();  // the spectra and the cleared counters are complete and visible
  int phase = 0;
#pragma unroll 1
  for (int set = 0; set < S; ++set) {
    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0.f;
    for (int b = set; b < a.B; b += S) {
      // one buffer per transform, alternating (no barrier guards the last reads)
      float2* buf = phase ? buf1 : buf0;
      if (h == 0) split_block<0>(yd + (size_t)b * N, ksh, cp, j, buf, tw, wj, acc);
      else split_block<1>(yd + (size_t)b * N, ksh, cp, j, buf, tw, wj, acc);
      phase ^= 1;
    }
    constexpr float sc = 1.f / ((float)N * (float)N);
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] *= sc;
    if (a.surface != nullptr) {
      float* row = a.surface + (((size_t)set * a.P + p) * a.D + d) * (size_t)N;
#pragma unroll
      for (int r = 0; r < 16; ++r) row[2 * ClassLocal<M>::out_index(jo, r) + h] = acc[r];
    }
    // this half's peak and the smallest phase holding it
    float tmax = acc[0];
#pragma unroll
    for (int r = 1; r < 16; ++r) tmax = fmaxf(tmax, acc[r]);
    float best = block_max<T>(tmax, s_val);
    uint32_t bt = 0xffffffffu;
    if (tmax == best) {
#pragma unroll
      for (int r = 15; r >= 0; --r)
        if (acc[r] == best) bt = (uint32_t)(2 * ClassLocal<M>::out_index(jo, r) + h);
    }
    bt = block_min_u32<T>(bt, s_idx);
    if (j == 0) {
      s_peak = best;
      s_tau = bt;
    }
    cluster.sync();
    {
      const float ob = *cluster.map_shared_rank(&s_peak, h ^ 1);
      const uint32_t ot = *cluster.map_shared_rank(&s_tau, h ^ 1);
      if (ob > best || (ob == best && ot < bt)) {
        best = ob;
        bt = ot;
      }
    }
    // this half's maximum outside the band around the row's peak phase: the
    // phases of thread j are all 2 jo + h modulo 512 (> 2 excl + 1)
    float sec = tmax;
    if (2 * a.excl + 1 > 512 || ((2 * jo + h - (int)bt + a.excl) & 511) <= 2 * a.excl) {
      sec = 0.f;  // every cell is >= 0
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        int dist = abs(2 * ClassLocal<M>::out_index(jo, r) + h - (int)bt);
        dist = min(dist, N - dist);
        if (dist > a.excl) sec = fmaxf(sec, acc[r]);
      }
    }
    sec = block_max<T>(sec, s_val);
    if (j == 0) s_sec = sec;
    cluster.sync();
    sec = fmaxf(sec, *cluster.map_shared_rank(&s_sec, h ^ 1));
    if (h == 0 && j == 0) {
      RowStat rs;
      rs.peak = best;
      rs.tau = bt;
      rs.second = sec;
      rs.pad = 0;
      a.rows[((size_t)set * a.P + p) * a.D + d] = rs;
    }
  }
  // neither CTA leaves while the other may still read its shared memory
  cluster.sync();
  if (h != 0) return;
  // CTA 0 of the pair counts the row for its PRN; the last one detects (as
  // in xcorr_tile).  The cluster barrier ordered CTA 1's surface writes
  // before this CTA's fence.
  __shared__ unsigned s_last;
  __syncthreads();
  if (a.second_whole) {
    if (j == 0) {
      __threadfence();
      s_last = (atomicAdd(a.counters + p, 1u) == (unsigned)(a.D - 1)) ? 1u : 0u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      finalize_prn<N, T>(a, p, S, s_val, s_idx);
    }
    return;
  }
  if (j >= 32) return;
  unsigned last = 0;
  if (j == 0) {
    __threadfence();
    last = (atomicAdd(a.counters + p, 1u) == (unsigned)(a.D - 1)) ? 1u : 0u;
  }
  if (__shfl_sync(0xffffffffu, last, 0)) {
    __threadfence();
    finalize_prn<N, 32>(a, p, S, s_val, s_idx);
  }
}

// Grid: two CTAs per (PRN, Doppler) tile, CTA 2 t + h in cluster t.
template <bool HALF>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(SplitCfg::T, 1) k_xcorr_split(const XcorrArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  xcorr_tile_split<HALF>(a, (int)(blockIdx.x >> 1), sm);
}

template <bool HALF>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(SplitCfg::T, 1)
    k_xcorr_split_batch(const BatchReq* __restrict__ reqs, const uint32_t* __restrict__ base, int n) {
  extern __shared__ __align__(16) float2 sm[];
  const unsigned tile = blockIdx.x >> 1;
  const int r = find_request(base, n, tile);
  xcorr_tile_split<HALF>(reqs[r].xc, (int)(tile - __ldg(base + r)), sm);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
bool supported_fft_size(int N) {
  return N == 256 || N == 512 || N == 1024 || N == 2048 || N == 4096 || N == 8192 || N == 16384;
}

cudaError_t launch_gold(const int* d_prns, int P, int8_t* d_codes, cudaStream_t stream) {
  k_gold<<<P, 128, 0, stream>>>(d_prns, d_codes);
  return cudaGetLastError();
}

template <int N>
static cudaError_t code_spectra_n(const int8_t* d_codes, int P, float2* d_cspec, cudaStream_t stream) {
  cudaError_t e = set_smem(k_code_spectra<N>, Cfg<N>::smem);
  if (e != cudaSuccess) return e;
  k_code_spectra<N><<<P, Cfg<N>::T, Cfg<N>::smem, stream>>>(d_codes, d_cspec);
  return cudaGetLastError();
}

#define GNSS_DISPATCH_N(N, CALL)          \
  switch (N) {                            \
    case 256: { constexpr int NN = 256; CALL; } \
    case 512: { constexpr int NN = 512; CALL; } \
    case 1024: { constexpr int NN = 1024; CALL; } \
    case 2048: { constexpr int NN = 2048; CALL; } \
    case 4096: { constexpr int NN = 4096; CALL; } \
    case 8192: { constexpr int NN = 8192; CALL; } \
    case 16384: { constexpr int NN = 16384; CALL; } \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_code_spectra(const int8_t* d_codes, int P, int N, float2* d_cspec, cudaStream_t stream) {
  GNSS_DISPATCH_N(N, return code_spectra_n<NN>(d_codes, P, d_cspec, stream));
}

template <int N>
static cudaError_t wipe_fft_n(const AcqShape& s, const uint8_t* d_samples, const int* d_group, const int* d_gkey,
                              float2* d_Z, float2* d_Y, unsigned* d_counters, cudaStream_t stream,
                              cudaEvent_t between) {
  const int fgrid = s.G * s.B * FoldCfg<N>::CPB;
  const FoldArgs fa = fold_args(s, d_samples, d_gkey, d_Z, d_counters);
  if (s.format == GNSS_FMT_2BIT_IQ)
    k_fold<N, GNSS_FMT_2BIT_IQ><<<fgrid, FoldCfg<N>::T, 0, stream>>>(fa);
  else
    k_fold<N, GNSS_FMT_I8_IQ><<<fgrid, FoldCfg<N>::T, 0, stream>>>(fa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (between && (e = cudaEventRecord(between, stream)) != cudaSuccess) return e;
  e = set_smem(k_carrier_fft<N>, Cfg<N>::smem);
  if (e != cudaSuccess) return e;
  return launch_dependent(k_carrier_fft<N>, (s.C ? s.C : s.D) * s.B, Cfg<N>::T, Cfg<N>::smem, stream,
                          carrier_args(s, d_group, d_Z, d_Y));
}

cudaError_t launch_wipe_fft(const AcqShape& s, const uint8_t* d_samples, const int* d_group, const int* d_gkey,
                            float2* d_Z, float2* d_Y, unsigned* d_counters, cudaStream_t stream,
                            cudaEvent_t between) {
  GNSS_DISPATCH_N(s.N, return wipe_fft_n<NN>(s, d_samples, d_group, d_gkey, d_Z, d_Y, d_counters, stream,
                                             between));
}

// Correlate-kernel variant per device and FFT size: elements per thread E,
// plus GNSS_TUNE_STAGED for the TMA-staged form or GNSS_TUNE_CLASS_LOCAL for
// the class-local schedule (at 16384: the two-CTA cluster split).
static int g_xcorr_e[128][15];

int xcorr_default_e(int N) {
  // At 4096, 8192 and 16384 the tensor-memory occupancy form (the code
  // spectra, sums and twiddle bases in TMEM, 64 registers, one exchange
  // buffer per CTA, 32 warps per SM: four CTAs at 4096, 0.211 vs 0.230 ms for
  // the class-local register form on the 100 ms, 10 ms-block request and
  // 1.84 vs 2.08 ms with 1 ms blocks; two at 8192, 4.24 vs 4.57 ms for 100 ms
  // at 8.192 MHz, 1 ms blocks; one of 1024 threads at 16384, 9.59 vs 11.81 ms
  // for the 32-per-thread form with two bins per CTA, 100 ms at 16.384 MHz),
  // else at 16384 that two-bin form, each where the GPU can hold its columns.
  const int occ = 16 | (int)GNSS_TUNE_TMEM | (int)GNSS_TUNE_OCC;
  const int tm16384 = 32 | (int)GNSS_TUNE_TMEM | (int)GNSS_TUNE_BINS(2);
  if ((N == 4096 || N == 8192 || N == 16384) && xcorr_tm_valid(N, occ)) return occ;
  if (N == 16384 && xcorr_tm_valid(N, tm16384)) return tm16384;
  if (N == 4096 || N == 8192) return 16 | (int)GNSS_TUNE_CLASS_LOCAL;
  // at 16384 otherwise the 32-per-thread form: faster than the two-CTA split
  // alone (13.27 vs 13.54 ms for 100 ms at 16.384 MHz, 1 ms blocks) and beside
  // concurrent requests (each cluster needs two SMs of one GPC free at once)
  return N >= 16384 ? 32 : 16;
}

static bool stage_fits(int N) {
  switch (N) {
    case 256: return StageFits<256>::value;
    case 512: return StageFits<512>::value;
    case 1024: return StageFits<1024>::value;
    case 2048: return StageFits<2048>::value;
    case 4096: return StageFits<4096>::value;
    case 8192: return StageFits<8192>::value;
    case 16384: return StageFits<16384>::value;
    default: return false;
  }
}

bool xcorr_valid_e(int N, int code) {
  if (code & (int)GNSS_TUNE_TMEM) return xcorr_tm_valid(N, code);
  if (code == (16 | (int)GNSS_TUNE_STAGED)) return N / 16 <= 1024 && stage_fits(N);
  if (code == (16 | (int)GNSS_TUNE_CLASS_LOCAL)) return N == 4096 || N == 8192;
  if (code == (32 | (int)GNSS_TUNE_CLASS_LOCAL)) return N == 16384;
  return (code == 16 && N / 16 <= 1024) || (code == 32 && N >= 1024) || (code == 8 && N / 8 <= 1024);
}

int xcorr_variant(int N) {
  int dev = 0;
  cudaGetDevice(&dev);
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  if (dev < 0 || dev >= 128 || lg >= 15) return xcorr_default_e(N);
  int e = __atomic_load_n(&g_xcorr_e[dev][lg], __ATOMIC_RELAXED);
  if (e == 0) {
    // the default is settled once per device and size (it asks the runtime
    // whether the tensor-memory form fits); a concurrent tuner store wins
    int expect = 0;
    e = xcorr_default_e(N);
    if (!__atomic_compare_exchange_n(&g_xcorr_e[dev][lg], &expect, e, false, __ATOMIC_RELAXED, __ATOMIC_RELAXED))
      e = expect;
  }
  return e;
}

void set_xcorr_variant(int N, int E) {
  int dev = 0;
  cudaGetDevice(&dev);
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  if (dev >= 0 && dev < 128 && lg < 15) __atomic_store_n(&g_xcorr_e[dev][lg], E, __ATOMIC_RELAXED);
}

template <int N, int E, bool ST, bool CL = false>
static cudaError_t xcorr_ne(const AcqShape& s, const XcorrArgs& a, cudaStream_t stream) {
  using X = XCfg<N, E, ST, CL>;
  const int grid = s.P * s.D;
  if (s.sets == 2) {
    cudaError_t e = set_smem(k_xcorr<N, E, true, ST, CL>, X::smem);
    if (e != cudaSuccess) return e;
    return launch_dependent(k_xcorr<N, E, true, ST, CL>, grid, X::T, X::smem, stream, a);
  } else {
    cudaError_t e = set_smem(k_xcorr<N, E, false, ST, CL>, X::smem);
    if (e != cudaSuccess) return e;
    return launch_dependent(k_xcorr<N, E, false, ST, CL>, grid, X::T, X::smem, stream, a);
  }
}

template <int N>
static cudaError_t xcorr_n(const AcqShape& s, const XcorrArgs& a, cudaStream_t stream) {
  const int v = xcorr_variant(N);
  if (v & (int)GNSS_TUNE_TMEM) return launch_xcorr_tm(v, s, a, stream);
  if constexpr (N >= 1024) {
    if (v == 32) return xcorr_ne<N, 32, false>(s, a, stream);
  }
  if constexpr (N / 8 <= 1024) {
    if (v == 8) return xcorr_ne<N, 8, false>(s, a, stream);
  }
  if constexpr (StageFits<N>::value) {
    if (v == (16 | (int)GNSS_TUNE_STAGED)) return xcorr_ne<N, 16, true>(s, a, stream);
  }
  if constexpr (N == 4096 || N == 8192) {
    if (v == (16 | (int)GNSS_TUNE_CLASS_LOCAL)) return xcorr_ne<N, 16, false, true>(s, a, stream);
  }
  if constexpr (N == 16384) {
    if (v == (32 | (int)GNSS_TUNE_CLASS_LOCAL)) {
      const unsigned grid = 2u * (unsigned)(s.P * s.D);
      cudaError_t e;
      if (s.sets == 2) {
        if ((e = set_smem(k_xcorr_split<true>, SplitCfg::smem)) != cudaSuccess) return e;
        return launch_dependent(k_xcorr_split<true>, grid, SplitCfg::T, SplitCfg::smem, stream, a);
      }
      if ((e = set_smem(k_xcorr_split<false>, SplitCfg::smem)) != cudaSuccess) return e;
      return launch_dependent(k_xcorr_split<false>, grid, SplitCfg::T, SplitCfg::smem, stream, a);
    }
  }
  return xcorr_ne<N, 16, false>(s, a, stream);
}

FoldArgs fold_args(const AcqShape& s, const uint8_t* d_samples, const int* d_gkey, float2* d_Z,
                   unsigned* d_counters) {
  FoldArgs a;
  a.samples = d_samples;
  a.gkey = d_gkey;
  a.Z = d_Z;
  a.counters = d_counters;
  a.coh = s.coh;
  a.B = s.B;
  a.P = s.P;
  return a;
}

CarrierArgs carrier_args(const AcqShape& s, const int* d_group, const float2* d_Z, float2* d_Y) {
  CarrierArgs a;
  a.Z = d_Z;
  a.group = d_group;
  a.Y = d_Y;
  a.fs = s.fs;
  a.coh = s.coh;
  a.B = s.B;
  a.dopp_min = s.dopp_min;
  a.dopp_step = s.dopp_step;
  a.code_dopp = s.code_dopp;
  a.cls_fgroup = s.C ? s.cls_fgroup : nullptr;
  a.cls_base = s.C ? s.cls_base : nullptr;
  return a;
}

// spectra above this size (a fifth of the B300's 126 MB L2) run class by class
static constexpr size_t kClassOrderBytes = 24u << 20;

XcorrArgs xcorr_args(const AcqShape& s, const float2* d_Y, const float2* d_cspec, const int* d_prns,
                     float* d_surface, RowStat* d_rows, unsigned* d_counters, gnss_detection* d_out) {
  XcorrArgs a;
  a.Y = d_Y;
  a.bin_cls = s.C ? s.bin_cls : nullptr;
  a.bin_shift = s.C ? s.bin_shift : nullptr;
  // Tiles run class by class only when the spectra outgrow L2: then CTAs
  // resident together re-read few rows (a 359 ms request at 16.384 MHz:
  // 92 MB of spectra, DRAM reads 1.7 -> 0.9 GB with the two-CTA split).
  // Spectra that stay resident are read faster spread over many rows
  // (1.3% at 100 ms and 4.096 MHz, 2.6 MB).
  a.bin_order = (s.C && (size_t)s.C * s.B * s.N * sizeof(float2) > kClassOrderBytes) ? s.bin_order : nullptr;
  a.cspec = d_cspec;
  a.B = s.B;
  a.D = s.D;
  a.P = s.P;
  a.excl = s.excl;
  a.surface = d_surface;
  a.rows = d_rows;
  a.counters = d_counters;
  a.prns = d_prns;
  a.out = d_out;
  a.dopp_min = s.dopp_min;
  a.dopp_step = s.dopp_step;
  a.threshold = s.threshold;
  a.second_whole = s.second_whole;
  return a;
}

cudaError_t launch_xcorr(const AcqShape& s, const float2* d_Y, const float2* d_cspec, const int* d_prns,
                         float* d_surface, RowStat* d_rows, unsigned* d_counters, gnss_detection* d_out,
                         cudaStream_t stream) {
  const XcorrArgs a = xcorr_args(s, d_Y, d_cspec, d_prns, d_surface, d_rows, d_counters, d_out);
  GNSS_DISPATCH_N(s.N, return xcorr_n<NN>(s, a, stream));
}

template <int N, int E, bool ST, bool CL = false>
static cudaError_t xcorr_batch_ne(const BatchGroup& g, cudaStream_t stream) {
  using X = XCfg<N, E, ST, CL>;
  cudaError_t e;
  if (g.sets == 2) {
    if ((e = set_smem(k_xcorr_batch<N, E, true, ST, CL>, X::smem)) != cudaSuccess) return e;
    return launch_dependent(k_xcorr_batch<N, E, true, ST, CL>, g.xc_ctas, X::T, X::smem, stream, g.reqs, g.xc_base,
                            g.n);
  } else {
    if ((e = set_smem(k_xcorr_batch<N, E, false, ST, CL>, X::smem)) != cudaSuccess) return e;
    return launch_dependent(k_xcorr_batch<N, E, false, ST, CL>, g.xc_ctas, X::T, X::smem, stream, g.reqs,
                            g.xc_base, g.n);
  }
}

// Batched launches: every request of the group shares N, format and sets.
template <int N>
static cudaError_t batch_n(const BatchGroup& g, cudaStream_t stream) {
  cudaError_t e;
  if (g.format == GNSS_FMT_2BIT_IQ)
    k_fold_batch<N, GNSS_FMT_2BIT_IQ><<<g.fold_ctas, FoldCfg<N>::T, 0, stream>>>(g.reqs, g.fold_base, g.n);
  else
    k_fold_batch<N, GNSS_FMT_I8_IQ><<<g.fold_ctas, FoldCfg<N>::T, 0, stream>>>(g.reqs, g.fold_base, g.n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = set_smem(k_carrier_fft_batch<N>, Cfg<N>::smem)) != cudaSuccess) return e;
  if ((e = launch_dependent(k_carrier_fft_batch<N>, g.car_ctas, Cfg<N>::T, Cfg<N>::smem, stream, g.reqs, g.car_base,
                            g.n)) != cudaSuccess)
    return e;
  // the variant the wave's CTA offsets were counted for
  const int v = g.variant;
  if (v & (int)GNSS_TUNE_TMEM) return launch_xcorr_tm_batch(v, g, stream);
  if constexpr (N >= 1024) {
    if (v == 32) return xcorr_batch_ne<N, 32, false>(g, stream);
  }
  if constexpr (N / 8 <= 1024) {
    if (v == 8) return xcorr_batch_ne<N, 8, false>(g, stream);
  }
  if constexpr (StageFits<N>::value) {
    if (v == (16 | (int)GNSS_TUNE_STAGED)) return xcorr_batch_ne<N, 16, true>(g, stream);
  }
  if constexpr (N == 4096 || N == 8192) {
    if (v == (16 | (int)GNSS_TUNE_CLASS_LOCAL)) return xcorr_batch_ne<N, 16, false, true>(g, stream);
  }
  if constexpr (N == 16384) {
    if (v == (32 | (int)GNSS_TUNE_CLASS_LOCAL)) {
      const unsigned grid = 2u * g.xc_ctas;
      if (g.sets == 2) {
        if ((e = set_smem(k_xcorr_split_batch<true>, SplitCfg::smem)) != cudaSuccess) return e;
        return launch_dependent(k_xcorr_split_batch<true>, grid, SplitCfg::T, SplitCfg::smem, stream, g.reqs,
                                g.xc_base, g.n);
      }
      if ((e = set_smem(k_xcorr_split_batch<false>, SplitCfg::smem)) != cudaSuccess) return e;
      return launch_dependent(k_xcorr_split_batch<false>, grid, SplitCfg::T, SplitCfg::smem, stream, g.reqs,
                              g.xc_base, g.n);
    }
  }
  return xcorr_batch_ne<N, 16, false>(g, stream);
}

// Polls of each staged-correlate wait before it gives up (testing).
cudaError_t set_stage_wait_limit(unsigned iters, cudaStream_t stream) {
  cudaError_t e = cudaMemcpyToSymbolAsync(g_stage_wait_limit, &iters, sizeof(unsigned), 0, cudaMemcpyHostToDevice,
                                          stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  return e;
}

cudaError_t launch_batch(const BatchGroup& g, cudaStream_t stream) {
  GNSS_DISPATCH_N(g.N, return batch_n<NN>(g, stream));
}

uint32_t fold_ctas_per_block(int N) {
  switch (N) {
    case 256: return FoldCfg<256>::CPB;
    case 512: return FoldCfg<512>::CPB;
    case 1024: return FoldCfg<1024>::CPB;
    case 2048: return FoldCfg<2048>::CPB;
    case 4096: return FoldCfg<4096>::CPB;
    case 8192: return FoldCfg<8192>::CPB;
    default: return FoldCfg<16384>::CPB;
  }
}

AcqScratch scratch_layout(const AcqShape& s) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  AcqScratch L;
  L.z = 0;
  L.y = L.z + al((size_t)s.G * s.B * s.N * sizeof(float2));
  L.rows = L.y + al((size_t)(s.C ? s.C : s.D) * s.B * s.N * sizeof(float2));
  L.counters = L.rows + al((size_t)s.sets * s.P * s.D * sizeof(RowStat));
  L.total = L.counters + al((size_t)(s.P + 1) * sizeof(unsigned));
  return L;
}

}  // namespace gnss

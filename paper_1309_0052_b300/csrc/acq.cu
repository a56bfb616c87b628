// acq.cu -- acquisition kernels (Section 3, Fig. 2) for sm_103a.
//
//   k_gold         G1/G2 LFSR Gold codes (code NCO input), bit-exact
//   k_code_spectra replica sampling at fs + forward FFT -> resident C_p
//   k_wipe_fft     2-bit / int8 I/Q unpack, carrier wipe-off, coherent fold
//                  of T_coh ms, forward FFT: Y_{f,b}     (first mixing + FFT)
//   k_xcorr        Y * conj(C_p), IFFT, |.|^2, non-coherent accumulation over
//                  blocks in registers, per-row peak statistics
//                                                   (second mixing + IFFT)
//   k_peak         per-PRN peak / second peak / ratio (signal detection)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fft.cuh"
#include "internal.h"

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
// Per-N launch configuration.  E = elements per thread, T = N / E threads.
// ---------------------------------------------------------------------------
template <int N>
struct Cfg {
  static constexpr int E = N >= 16384 ? 32 : 16;
  static constexpr int T = N / E;
  static constexpr bool TWC = (E == 16);                        // twiddle bases cached in registers
  static constexpr size_t buf_bytes = sizeof(float2) * FftShape<N>::smem_elems;
  static constexpr bool DB = 2 * buf_bytes <= 160 * 1024;     // ping-pong exchange buffers
  static constexpr size_t smem = (DB ? 2 : 1) * buf_bytes;
  static constexpr int MINB = T <= 256 ? 2 : 1;
};

// ---------------------------------------------------------------------------
// K1b: code spectra.  Thread j builds the replica samples j + T r directly
// (c_s[m] = c[floor(m * 1023 / N)]) and transforms them in place.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Cfg<N>::T) k_code_spectra(const int8_t* __restrict__ codes,
                                                           float2* __restrict__ cspec) {
  constexpr int E = Cfg<N>::E, T = Cfg<N>::T;
  extern __shared__ float2 sm[];
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
// per-millisecond constant w_i = exp(-j 2 pi ((f i) mod 1000) / 1000).  Each
// thread folds E consecutive samples m = E j + e (vector loads: 8 or 16 bytes
// of 2-bit data, 32 or 64 bytes of int8 per millisecond), computes the
// carrier of its first sample from the exact integer phase and steps it by
// the per-sample rotation, then the block is transposed through shared
// memory into the FFT's register layout.
// Grid: one CTA per (Doppler d, block b), tile = d * B + b.
// ---------------------------------------------------------------------------
template <int E, int FMT>
__device__ __forceinline__ void load_ms(const uint8_t* __restrict__ base, int64_t n0, float (&xi)[E],
                                        float (&xq)[E]) {
  if constexpr (FMT == GNSS_FMT_2BIT_IQ) {
    // E samples = E/2 bytes; sample e: bits [4e, 4e+4) of the little-endian words
    const uint32_t* w = reinterpret_cast<const uint32_t*>(base + n0 / 2);
    uint32_t words[E / 8];
    if constexpr (E == 16) {
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

template <int N, int FMT>
__global__ void __launch_bounds__(Cfg<N>::T) k_wipe_fft(const uint8_t* __restrict__ samples, int fs, int coh,
                                                       int B, int dopp_min, int dopp_step,
                                                       float2* __restrict__ Y) {
  constexpr int E = Cfg<N>::E, T = Cfg<N>::T;
  extern __shared__ float2 sm[];
  float2* buf0 = sm;
  float2* buf1 = Cfg<N>::DB ? sm + FftShape<N>::smem_elems : sm;
  const int j = threadIdx.x;
  const int d = blockIdx.x / B, b = blockIdx.x % B;
  const int f = dopp_min + d * dopp_step;
  const int64_t L = (int64_t)coh * N;
  const int64_t n_first = (int64_t)b * L + (int64_t)E * j;  // first sample of this thread, ms 0

  // fold: acc[e] = sum_i x[n_first + iN + e] w_i
  float ar[E], ai[E];
#pragma unroll
  for (int e = 0; e < E; ++e) ar[e] = ai[e] = 0.f;
  float wsum_r = 0.f, wsum_i = 0.f;
  const int f1000 = ((f % 1000) + 1000) % 1000;
  for (int i = 0; i < coh; ++i) {
    const int ri = (int)(((int64_t)f1000 * i) % 1000);
    float ws, wc;
    sincospif(-2.f * (float)ri / 1000.f, &ws, &wc);
    float xi[E], xq[E];
    load_ms<E, FMT>(samples, n_first + (int64_t)i * N, xi, xq);
    float wr = wc, wi = ws;
    if constexpr (FMT == GNSS_FMT_2BIT_IQ) {  // x = 2c - 3(1 + j): fold 2c w here, -3(1 + j) sum(w) after
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
  // carrier of sample bL + E j + e: exact integer phase for e = 0, then steps
  const int64_t fr = (((int64_t)f % fs) + fs) % fs;
  const int64_t r0 = (fr * (int64_t)((int64_t)b * L + (int64_t)E * j)) % fs;
  float cs0, cc0, ss, sc;
  const float inv_fs = 1.f / (float)fs;
  sincospif(-2.f * (float)r0 * inv_fs, &cs0, &cc0);
  sincospif(-2.f * (float)fr * inv_fs, &ss, &sc);
  float2 car = make_float2(cc0, cs0);
  const float2 step = make_float2(sc, ss);
  float2 v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    v[e] = c_mul(make_float2(ar[e], ai[e]), car);
    car = c_mul(car, step);
  }
  // transpose m = E j + e  ->  register layout j + T r
  {
    float2* b = buf0 + pad16(E * j);  // E j is a multiple of 16
#pragma unroll
    for (int e = 0; e < E; ++e) b[e + (e >> 4)] = v[e];
  }
  __syncthreads();
  gather_regs<N, E>(v, j, buf0);
  int phase = 1;  // next exchange uses buf1 (buf0 may still be read by a slower thread)
  if constexpr (!Cfg<N>::DB) phase = 0;
  fft_block<N, E, false, Cfg<N>::DB>(v, j, buf0, buf1, phase);
  float2* out = Y + (size_t)blockIdx.x * N;
#pragma unroll
  for (int r = 0; r < E; ++r) out[j + T * r] = v[r];
}

// ---------------------------------------------------------------------------
// Block-wide (max, argmax) with the smallest index on ties, then max over
// the cells outside the circular exclusion band around the argmax.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void better(float& v, uint32_t& t, float ov, uint32_t ot) {
  if (ov > v || (ov == v && ot < t)) {
    v = ov;
    t = ot;
  }
}

// Lanes that exist in a CTA of T threads (T is a power of two >= 16).
template <int T>
struct WarpShape {
  static constexpr unsigned mask = T >= 32 ? 0xffffffffu : ((1u << T) - 1u);
  static constexpr int first = T >= 32 ? 16 : T / 2;
};

template <int T>
__device__ __forceinline__ void block_argmax(float& v, uint32_t& t, float* s_val, uint32_t* s_idx) {
  constexpr int W = (T + 31) / 32;
#pragma unroll
  for (int o = WarpShape<T>::first; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(WarpShape<T>::mask, v, o);
    const uint32_t ot = __shfl_xor_sync(WarpShape<T>::mask, t, o);
    better(v, t, ov, ot);
  }
  if constexpr (W > 1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
      s_val[warp] = v;
      s_idx[warp] = t;
    }
    __syncthreads();
    v = s_val[0];
    t = s_idx[0];
#pragma unroll
    for (int w = 1; w < W; ++w) better(v, t, s_val[w], s_idx[w]);
  }
}

template <int T>
__device__ __forceinline__ float block_max(float v, float* s_val) {
  constexpr int W = (T + 31) / 32;
#pragma unroll
  for (int o = WarpShape<T>::first; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(WarpShape<T>::mask, v, o));
  if constexpr (W > 1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_val[warp] = v;
    __syncthreads();
    v = s_val[0];
#pragma unroll
    for (int w = 1; w < W; ++w) v = fmaxf(v, s_val[w]);
  }
  return v;
}

template <int N, int E>
__device__ __forceinline__ void row_stats(const float (&a)[E], int j, int excl, float* s_val, uint32_t* s_idx,
                                          RowStat* out) {
  constexpr int T = N / E;
  float best = -1.f;
  uint32_t bt = 0;
#pragma unroll
  for (int r = 0; r < E; ++r) {  // ascending r = ascending code phase for this thread
    if (a[r] > best) {
      best = a[r];
      bt = (uint32_t)(j + T * r);
    }
  }
  block_argmax<T>(best, bt, s_val, s_idx);
  float sec = 0.f;  // every cell is >= 0
#pragma unroll
  for (int r = 0; r < E; ++r) {
    int dist = abs(j + T * r - (int)bt);
    dist = min(dist, N - dist);
    if (dist > excl) sec = fmaxf(sec, a[r]);
  }
  sec = block_max<T>(sec, s_val);
  if (threadIdx.x == 0) {
    RowStat rs;
    rs.peak = best;
    rs.tau = bt;
    rs.second = sec;
    rs.pad = 0;
    *out = rs;
  }
}

// ---------------------------------------------------------------------------
// K4: correlate.  One CTA per (PRN p, Doppler d), tile = d * P + p; loops
// over the B blocks of Y[d], accumulating |R|^2 per set in registers.
// ---------------------------------------------------------------------------
// One block: Y * conj(C_p) -> IFFT -> |.|^2 added to acc0 (even blocks) or,
// with half-bit sets, to acc1 (odd blocks); one loop body serves both sets.
template <int N, int E, bool DB, bool TWC, bool HALF>
__device__ __forceinline__ void corr_block(const float2* __restrict__ y, const float2* __restrict__ cp, int j,
                                           float2* buf0, float2* buf1, int& phase, FftTw<N, E, true>& tw,
                                           float (&acc0)[E], float (&acc1)[E], bool odd) {
  constexpr int T = N / E;
  if constexpr (TWC) tw.launder();
  // Re-read the code spectrum from L1 every block: hoisting these 16 loads
  // out of the block loop would pin 32 registers and force spills.
  asm volatile("" : "+l"(cp));
  float2 v[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    // Y streams from L2 (not kept in L1); the code spectrum stays L1-resident
    v[r] = c_mulconj(__ldcg(y + j + T * r), __ldg(cp + j + T * r));
  }
  if constexpr (TWC) fft_block_tw<N, E, true, DB>(v, j, buf0, buf1, phase, tw);
  else fft_block<N, E, true, DB>(v, j, buf0, buf1, phase);
  if (HALF && odd) {  // uniform across the CTA
#pragma unroll
    for (int r = 0; r < E; ++r) acc1[r] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, acc1[r]));
  } else {
#pragma unroll
    for (int r = 0; r < E; ++r) acc0[r] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, acc0[r]));
  }
}

template <int N, bool HALF>
__global__ void __launch_bounds__(Cfg<N>::T, Cfg<N>::MINB)
    k_xcorr(const float2* __restrict__ Y, const float2* __restrict__ cspec, int B, int D, int P, int excl,
            float* __restrict__ surface, RowStat* __restrict__ rows) {
  constexpr int E = Cfg<N>::E, T = Cfg<N>::T;
  constexpr bool DB = Cfg<N>::DB, TWC = Cfg<N>::TWC;
  extern __shared__ float2 sm[];
  float2* buf0 = sm;
  float2* buf1 = DB ? sm + FftShape<N>::smem_elems : sm;
  __shared__ float s_val[32];
  __shared__ uint32_t s_idx[32];
  const int j = threadIdx.x;
  const int p = blockIdx.x % P, d = blockIdx.x / P;
  const float2* cp = cspec + (size_t)p * N;
  FftTw<N, E, true> tw;
  if constexpr (TWC) tw.init(j);
  float acc0[E], acc1[E];
#pragma unroll
  for (int r = 0; r < E; ++r) acc0[r] = acc1[r] = 0.f;
  const float2* yd = Y + (size_t)d * B * N;
  int phase = 0;
  for (int b = 0; b < B; ++b)
    corr_block<N, E, DB, TWC, HALF>(yd + (size_t)b * N, cp, j, buf0, buf1, phase, tw, acc0, acc1, (b & 1) != 0);
  // R = IFFT / N, so |R|^2 = |.|^2 / N^2 (an exact power of two)
  constexpr float sc = 1.f / ((float)N * (float)N);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    acc0[r] *= sc;
    acc1[r] *= sc;
  }
  constexpr int sets = HALF ? 2 : 1;
#pragma unroll
  for (int s = 0; s < sets; ++s) {
    const float(&a)[E] = (s == 0) ? acc0 : acc1;
    if (surface != nullptr) {
      float* row = surface + (((size_t)s * P + p) * D + d) * (size_t)N;
#pragma unroll
      for (int r = 0; r < E; ++r) row[j + T * r] = a[r];
    }
    row_stats<N, E>(a, j, excl, s_val, s_idx, rows + ((size_t)s * P + p) * D + d);
  }
}

// ---------------------------------------------------------------------------
// K5: per-PRN detection.  One warp per PRN: best row (ties to the smallest
// Doppler index), ratio = peak / second, set with the larger ratio.
// With GNSS_SECOND_WHOLE the second peak is searched over the whole stored
// surface outside the exclusion band around the peak phase.
// ---------------------------------------------------------------------------
__global__ void k_peak(const RowStat* __restrict__ rows, const int* __restrict__ prns, const float* __restrict__ surface,
                       int P, int D, int N, int sets, int excl, int dopp_min, int dopp_step, float threshold,
                       int second_whole, gnss_detection* __restrict__ out) {
  const int p = blockIdx.x, lane = threadIdx.x;
  float best_ratio = -1.f;
  gnss_detection rec;
  for (int s = 0; s < sets; ++s) {
    const RowStat* rs = rows + ((size_t)s * P + p) * D;
    float v = -1.f;
    uint32_t dbest = 0;
    for (int d = lane; d < D; d += 32) {
      const float pk = rs[d].peak;
      if (pk > v) {
        v = pk;
        dbest = (uint32_t)d;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, o);
      const uint32_t od = __shfl_xor_sync(0xffffffffu, dbest, o);
      better(v, dbest, ov, od);
    }
    const RowStat r = rs[dbest];
    float second = r.second;
    if (second_whole) {
      const float* S = surface + ((size_t)s * P + p) * D * (size_t)N;
      float m = 0.f;
      for (size_t idx = lane; idx < (size_t)D * N; idx += 32) {
        int t = (int)(idx % N);
        int dist = abs(t - (int)r.tau);
        dist = min(dist, N - dist);
        if (dist > excl) m = fmaxf(m, S[idx]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      second = m;
    }
    const float ratio = second > 0.f ? r.peak / second : INFINITY;
    if (s == 0 || ratio > best_ratio) {
      best_ratio = ratio;
      rec.prn = (uint8_t)prns[p];
      rec.set = (uint8_t)s;
      rec.reserved = 0;
      rec.dopp_bin = (int32_t)dbest;
      rec.dopp_hz = dopp_min + (int32_t)dbest * dopp_step;
      rec.code_phase = r.tau;
      rec.peak = r.peak;
      rec.second = second;
      rec.ratio = ratio;
    }
  }
  rec.detected = (uint8_t)(best_ratio >= threshold);
  if (lane == 0) out[p] = rec;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
bool supported_fft_size(int N) {
  return N == 256 || N == 512 || N == 1024 || N == 2048 || N == 4096 || N == 8192 || N == 16384;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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
static cudaError_t wipe_fft_n(const AcqShape& s, const uint8_t* d_samples, float2* d_Y, cudaStream_t stream) {
  const int grid = s.D * s.B;
  if (s.format == GNSS_FMT_2BIT_IQ) {
    cudaError_t e = set_smem(k_wipe_fft<N, GNSS_FMT_2BIT_IQ>, Cfg<N>::smem);
    if (e != cudaSuccess) return e;
    k_wipe_fft<N, GNSS_FMT_2BIT_IQ><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(d_samples, s.fs, s.coh, s.B,
                                                                             s.dopp_min, s.dopp_step, d_Y);
  } else {
    cudaError_t e = set_smem(k_wipe_fft<N, GNSS_FMT_I8_IQ>, Cfg<N>::smem);
    if (e != cudaSuccess) return e;
    k_wipe_fft<N, GNSS_FMT_I8_IQ><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(d_samples, s.fs, s.coh, s.B,
                                                                           s.dopp_min, s.dopp_step, d_Y);
  }
  return cudaGetLastError();
}

cudaError_t launch_wipe_fft(const AcqShape& s, const uint8_t* d_samples, float2* d_Y, cudaStream_t stream) {
  GNSS_DISPATCH_N(s.N, return wipe_fft_n<NN>(s, d_samples, d_Y, stream));
}

template <int N>
static cudaError_t xcorr_n(const AcqShape& s, const float2* d_Y, const float2* d_cspec, float* d_surface,
                           RowStat* d_rows, cudaStream_t stream) {
  const int grid = s.P * s.D;
  if (s.sets == 2) {
    cudaError_t e = set_smem(k_xcorr<N, true>, Cfg<N>::smem);
    if (e != cudaSuccess) return e;
    k_xcorr<N, true><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(d_Y, d_cspec, s.B, s.D, s.P, s.excl, d_surface,
                                                              d_rows);
  } else {
    cudaError_t e = set_smem(k_xcorr<N, false>, Cfg<N>::smem);
    if (e != cudaSuccess) return e;
    k_xcorr<N, false><<<grid, Cfg<N>::T, Cfg<N>::smem, stream>>>(d_Y, d_cspec, s.B, s.D, s.P, s.excl, d_surface,
                                                               d_rows);
  }
  return cudaGetLastError();
}

cudaError_t launch_xcorr(const AcqShape& s, const float2* d_Y, const float2* d_cspec, float* d_surface,
                         RowStat* d_rows, cudaStream_t stream) {
  GNSS_DISPATCH_N(s.N, return xcorr_n<NN>(s, d_Y, d_cspec, d_surface, d_rows, stream));
}

cudaError_t launch_peak(const AcqShape& s, const RowStat* d_rows, const int* d_prns, const float* d_surface,
                        gnss_detection* d_out, cudaStream_t stream) {
  k_peak<<<s.P, 32, 0, stream>>>(d_rows, d_prns, d_surface, s.P, s.D, s.N, s.sets, s.excl, s.dopp_min,
                                 s.dopp_step, s.threshold, s.second_whole, d_out);
  return cudaGetLastError();
}

}  // namespace gnss

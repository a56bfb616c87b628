// fft.cuh -- register-resident mixed-radix Stockham FFT for one CTA (sm_103a).
//
// The FFT / IFFT blocks of the acquisition channel (Section 3, Fig. 2).
// One CTA of T = N / E threads transforms one N-point complex vector.  Thread
// j always holds the E elements x[j + T r], r < E, in registers:
//   - every Stockham pass reads its butterfly inputs J + s N / R, which for
//     J = j + T q are exactly x[j + T (q + (E/R) s)], so the first pass of a
//     transform starts from registers without any shared-memory traffic;
//   - the last pass writes its outputs J + t N / R = j + T (q + (E/R) t),
//     again the thread's own registers, in natural order;
//   - the P - 1 passes in between exchange through shared memory (padded
//     index i + i/16, so the stride-16 writes of the first pass and the
//     unit-stride reads are free of bank conflicts).
// Radix-16 passes come first, then one radix-2/4/8 pass for the rest of N.
//
// Pass with sub-transform size NS and radix R (Stockham autosort): for
// butterfly J < N/R, k = J mod NS,
//   u[s] = x[J + s N/R] * W_{NS R}^{s k},   u <- DFT_R(u),
//   y[(J / NS) NS R + k + t NS] = u[t].
// Forward W = exp(-2 pi i / M) unscaled; inverse W = exp(+2 pi i / M), the
// caller applies 1/N.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gnss {

// Complex sums and differences as two-wide FP32 operations (add.f32x2: one
// instruction for both components; per component the same round-to-nearest
// result as the scalar form).  Complex products stay scalar: their packed
// form needs swapped operands and broadcast twiddle pairs, which cost more
// registers than the kernels have.
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 c_mulconj(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by the quarter-turn of the transform direction: -i (forward), +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 c_quarter(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos / sin of k pi / 8 (mathematical constants of the 16-point transform)
#define GNSS_C1 0.92387953251128675613f  // cos(pi/8)
#define GNSS_S1 0.38268343236508977173f  // sin(pi/8)
#define GNSS_R2 0.70710678118654752440f  // sqrt(2)/2

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = c_add(t, b);
  b = c_sub(t, b);
}

// 4-point DFT in place, natural order.
template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 s0 = c_add(x0, x2), d0 = c_sub(x0, x2);
  float2 s1 = c_add(x1, x3), d1 = c_quarter<INV>(c_sub(x1, x3));
  x0 = c_add(s0, s1);
  x2 = c_sub(s0, s1);
  x1 = c_add(d0, d1);
  x3 = c_sub(d0, d1);
}

// multiply by W_M^m with W_M = exp(-+2 pi i / M) for the constant angles of
// the 8- and 16-point transforms (m * 16 / M in 0..9 sixteenths of a turn).
template <bool INV, int SIXTEENTHS>
__device__ __forceinline__ float2 twiddle16(float2 a) {
  constexpr float sg = INV ? 1.f : -1.f;
  if constexpr (SIXTEENTHS == 0) return a;
  else if constexpr (SIXTEENTHS == 4) return c_quarter<INV>(a);
  else if constexpr (SIXTEENTHS == 2) {  // (1 + sg i) / sqrt 2
    return make_float2(GNSS_R2 * (a.x - sg * a.y), GNSS_R2 * (a.y + sg * a.x));
  } else if constexpr (SIXTEENTHS == 6) {  // (-1 + sg i) / sqrt 2
    return make_float2(GNSS_R2 * (-a.x - sg * a.y), GNSS_R2 * (-a.y + sg * a.x));
  } else {
    constexpr float c = SIXTEENTHS == 1 ? GNSS_C1 : SIXTEENTHS == 3 ? GNSS_S1 : -GNSS_C1;
    constexpr float s = SIXTEENTHS == 1 ? GNSS_S1 : SIXTEENTHS == 3 ? GNSS_C1 : -GNSS_S1;
    return c_mul(a, make_float2(c, sg * s));
  }
}

// 8-point DFT: n = n2 + 4 n1, k = k1 + 2 k2.  Radix-2 over n1, twiddle
// W8^(n2 k1), radix-4 over n2.  Output X[k1 + 2 k2] lands in v[4 k1 + k2];
// the caller-visible order is restored by the final register permutation.
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft2<INV>(v[n2], v[n2 + 4]);  // v[n2 + 4 k1]
  v[5] = twiddle16<INV, 2>(v[5]);
  v[6] = twiddle16<INV, 4>(v[6]);
  v[7] = twiddle16<INV, 6>(v[7]);
  dft4<INV>(v[0], v[1], v[2], v[3]);  // k1 = 0 -> X[2 k2]
  dft4<INV>(v[4], v[5], v[6], v[7]);  // k1 = 1 -> X[1 + 2 k2]
  float2 t[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 2 * k2] = t[4 * k1 + k2];
}

// 16-point DFT: n = n2 + 4 n1, k = k1 + 4 k2.  Radix-4 over n1, twiddle
// W16^(n2 k1), radix-4 over n2, then the 4x4 register transpose.
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);  // v[n2 + 4 k1]
  v[5] = twiddle16<INV, 1>(v[5]);
  v[6] = twiddle16<INV, 2>(v[6]);
  v[7] = twiddle16<INV, 3>(v[7]);
  v[9] = twiddle16<INV, 2>(v[9]);
  v[10] = twiddle16<INV, 4>(v[10]);
  v[11] = twiddle16<INV, 6>(v[11]);
  v[13] = twiddle16<INV, 3>(v[13]);
  v[14] = twiddle16<INV, 6>(v[14]);
  v[15] = twiddle16<INV, 9>(v[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

// a + w b with four FMAs.
__device__ __forceinline__ float2 c_fma(float2 a, float2 w, float2 b) {
  return make_float2(fmaf(w.x, b.x, fmaf(-w.y, b.y, a.x)), fmaf(w.x, b.y, fmaf(w.y, b.x, a.y)));
}
// 2 a - t (the other output of a butterfly whose first output t = a + u).
__device__ __forceinline__ float2 c_twice_minus(float2 a, float2 t) {
  return __ffma2_rn(make_float2(2.f, 2.f), a, make_float2(-t.x, -t.y));
}

// 4-point DFT of (x0, y x1, y^2 x2, y^3 x3) in place, given y1 = y and
// y2 = y^2, in FMA form:
//   p0 = x0 + y2 x2,  p1 = x0 - y2 x2,  q0 = x1 + y2 x3,  q1 = x1 - y2 x3,
//   X0 = p0 + y1 q0,  X2 = p0 - y1 q0,  X1 = p1 + W4 y1 q1,  X3 = p1 - W4 y1 q1
// (W4 = -i forward, +i inverse); every difference is formed as 2a - (a + b).
template <bool INV>
__device__ __forceinline__ void dft4_tw(float2& x0, float2& x1, float2& x2, float2& x3, float2 y1, float2 y2) {
  const float2 p0 = c_fma(x0, y2, x2);
  const float2 p1 = c_twice_minus(x0, p0);
  const float2 q0 = c_fma(x1, y2, x3);
  const float2 q1 = c_twice_minus(x1, q0);
  const float2 X0 = c_fma(p0, y1, q0);
  const float2 X2 = c_twice_minus(p0, X0);
  const float2 X1 = c_fma(p1, c_quarter<INV>(y1), q1);
  const float2 X3 = c_twice_minus(p1, X1);
  x0 = X0;
  x1 = X1;
  x2 = X2;
  x3 = X3;
}

// Twiddled 16-point stage of a Stockham pass: X[t] = sum_s u[s] w^s W16^(s t)
// with s = n2 + 4 n1, t = k1 + 4 k2:
//   stage 1 (per n2): a[n2][k1] = DFT4 over n1 of u[n2 + 4 n1] (w^4)^n1,
//   stage 2 (per k1): X[k1 + 4 k2] = DFT4 over n2 of a[n2][k1] z^n2,
//                     z = w W16^k1,
// both with dft4_tw; w1, w2, w4, w8 are w, w^2, w^4, w^8.  Natural order out.
template <bool INV>
__device__ __forceinline__ void dft16_tw(float2 (&v)[16], float2 w1, float2 w2, float2 w4, float2 w8) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4_tw<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12], w4, w8);  // v[n2 + 4 k1]
  dft4_tw<INV>(v[0], v[1], v[2], v[3], w1, w2);
  dft4_tw<INV>(v[4], v[5], v[6], v[7], twiddle16<INV, 1>(w1), twiddle16<INV, 2>(w2));
  dft4_tw<INV>(v[8], v[9], v[10], v[11], twiddle16<INV, 2>(w1), twiddle16<INV, 4>(w2));
  dft4_tw<INV>(v[12], v[13], v[14], v[15], twiddle16<INV, 3>(w1), twiddle16<INV, 6>(w2));
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

// The same without external twiddles (w = 1): stage 2 uses the constants
// z = W16^k1.
template <bool INV>
__device__ __forceinline__ void dft16_c(float2 (&v)[16]) {
  constexpr float sg = INV ? 1.f : -1.f;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  dft4<INV>(v[0], v[1], v[2], v[3]);
  dft4_tw<INV>(v[4], v[5], v[6], v[7], make_float2(GNSS_C1, sg * GNSS_S1), make_float2(GNSS_R2, sg * GNSS_R2));
  dft4_tw<INV>(v[8], v[9], v[10], v[11], make_float2(GNSS_R2, sg * GNSS_R2), make_float2(0.f, sg));
  dft4_tw<INV>(v[12], v[13], v[14], v[15], make_float2(GNSS_S1, sg * GNSS_C1), make_float2(-GNSS_R2, sg * GNSS_R2));
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

template <int R, bool INV>
__device__ __forceinline__ void dft_r(float2 (&u)[R]) {
  if constexpr (R == 2) dft2<INV>(u[0], u[1]);
  else if constexpr (R == 4) dft4<INV>(u[0], u[1], u[2], u[3]);
  else if constexpr (R == 8) dft8<INV>(u);
  else dft16_c<INV>(u);
}

// Padded shared-memory index (one spare slot every 16 elements).
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int N>
struct FftShape {
  static constexpr int smem_elems = N + N / 16;
};

// Radix of the pass with sub-transform size NS: RMAX (16, or E when a
// thread holds fewer than 16 elements) while RMAX divides what is left of
// N, then the remainder.
template <int N, int NS, int E = 16>
struct PassRadix {
  static constexpr int rmax = E < 16 ? E : 16;
  static constexpr int rem = N / NS;
  static constexpr int value = rem >= rmax ? rmax : rem;
};

// One butterfly set of a pass (thread-local), twiddled and transformed.
// Inputs/outputs in v[q + Q s] as described at the top of the file.
template <int N, int E, int R, int NS, bool INV>
__device__ __forceinline__ void pass_compute(float2 (&v)[E], int j) {
  constexpr int T = N / E;
  constexpr int Q = E / R;
  // Twiddle base W^k, k = (j + T q) mod NS, of each butterfly q.  T and NS
  // are powers of two: if NS <= T every q has k = j mod NS; otherwise
  // k = j + T (q mod NS/T), and W^k = W^j W^(T m) with W^(T m) a constant of
  // the pass.  One sincospif per pass and thread, then constant products.
  constexpr float scale = (INV ? 2.f : -2.f) / float(NS * R);
  float2 w0 = make_float2(1.f, 0.f);
  if constexpr (NS > 1) {
    float sn, cs;
    sincospif(scale * float(j & (NS - 1)), &sn, &cs);
    w0 = make_float2(cs, sn);
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float2 u[R];
#pragma unroll
    for (int s = 0; s < R; ++s) u[s] = v[q + Q * s];
    if constexpr (NS > 1) {
      float2 w = w0;
      if constexpr (NS > T) {
        const int m = q % (NS / T);
        if (m != 0) {
          float sn, cs;
          sincospif(scale * float(T * m), &sn, &cs);  // a constant of the pass
          w = c_mul(w0, make_float2(cs, sn));
        }
      }
      if constexpr (R == 16) {
        const float2 w2 = c_mul(w, w), w4 = c_mul(w2, w2), w8 = c_mul(w4, w4);
        dft16_tw<INV>(u, w, w2, w4, w8);
      } else {
        float2 wp = w;
#pragma unroll
        for (int s = 1; s < R; ++s) {
          u[s] = c_mul(u[s], wp);
          if (s + 1 < R) wp = c_mul(wp, w);
        }
        dft_r<R, INV>(u);
      }
    } else {
      dft_r<R, INV>(u);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) v[q + Q * t] = u[t];
  }
}

// Scatter the pass outputs to shared memory at their Stockham positions.
// NS is 1, 8 or a multiple of 16 (radix-16 passes come first; radix-8
// transforms have NS = 1, 8, 64, ...).  For NS = 1, base = R J keeps
// base mod 16 + t < 16; for NS = 8, base = 64 (J / 8) + J mod 8 has
// base mod 16 < 8, so base + 8 t crosses a multiple of 16 exactly t / 2
// times; for NS a multiple of 16 the steps are whole.  In every case
// pad16(base + t NS) = pad16(base) + t NS + (t NS) / 16, so each store is one
// per-butterfly address plus a compile-time offset.
template <int N, int E, int R, int NS>
__device__ __forceinline__ void pass_store(const float2 (&v)[E], int j, float2* __restrict__ buf) {
  static_assert(NS == 1 || NS % 16 == 0 || (NS == 8 && R == 8), "pass order: radix-16 (or 8) passes first");
  constexpr int T = N / E;
  constexpr int Q = E / R;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int J = j + T * q;
    const int k = J & (NS - 1);
    float2* b = buf + pad16((J / NS) * NS * R + k);
#pragma unroll
    for (int t = 0; t < R; ++t) b[t * NS + ((t * NS) >> 4)] = v[q + Q * t];
  }
}

// Element j + T r of the padded buffer; T is a multiple of 16, so the offset
// from pad16(j) is the compile-time T r + T r / 16.
template <int N, int E>
__device__ __forceinline__ void gather_regs(float2 (&v)[E], int j, const float2* __restrict__ buf) {
  constexpr int T = N / E;
  static_assert(T % 16 == 0, "T must be a multiple of 16");
  const float2* b = buf + pad16(j);
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = b[T * r + ((T * r) >> 4)];
}

template <int N, int E>
__device__ __forceinline__ void scatter_regs(const float2 (&v)[E], int j, float2* __restrict__ buf) {
  constexpr int T = N / E;
  static_assert(T % 16 == 0, "T must be a multiple of 16");
  float2* b = buf + pad16(j);
#pragma unroll
  for (int r = 0; r < E; ++r) b[T * r + ((T * r) >> 4)] = v[r];
}

// Whole transform.  On entry and exit thread j holds x[j + T r] in v[r].
// Shared-memory exchanges alternate between buf0 and buf1 when DOUBLE_BUF
// (one barrier per exchange); with a single buffer a second barrier guards
// the reuse.  'phase' carries the alternation across calls so that
// back-to-back transforms in one CTA never overwrite a buffer still being
// read.  Every thread of the CTA must call this.
template <int N, int E, bool INV, bool DOUBLE_BUF, int NS = 1>
__device__ __forceinline__ void fft_block(float2 (&v)[E], int j, float2* buf0, float2* buf1, int& phase) {
  constexpr int R = PassRadix<N, NS, E>::value;
  pass_compute<N, E, R, NS, INV>(v, j);
  if constexpr (NS * R < N) {
    float2* buf = (DOUBLE_BUF && phase) ? buf1 : buf0;
    if constexpr (!DOUBLE_BUF) __syncthreads();
    pass_store<N, E, R, NS>(v, j, buf);
    __syncthreads();
    gather_regs<N, E>(v, j, buf);
    if constexpr (DOUBLE_BUF) phase ^= 1;
    fft_block<N, E, INV, DOUBLE_BUF, NS * R>(v, j, buf0, buf1, phase);
  }
}

// ---------------------------------------------------------------------------
// Twiddle bases held across many transforms of one CTA.
//
// A pass with sub-transform size NS > 1 multiplies input s (1 <= s < R) by
// W^(s k), W = exp(-+2 pi i / (NS R)), k = J mod NS.  Writing s = 4 hi + lo,
// W^(s k) = W^(lo k) W^(4 hi k), so a thread keeps a[] = W^k, W^2k, W^3k and
// b[] = W^4k, W^8k, ... and forms each twiddle with at most one complex
// multiply.  These bases depend only on the thread, not on the data, so a
// kernel that runs many transforms computes them once.
// ---------------------------------------------------------------------------
template <int R>
struct TwBase {
  static_assert(R < 16, "radix-16 passes use TwBase16");
  static constexpr int NA = R >= 4 ? 3 : 1;
  static constexpr int NB = R >= 8 ? R / 4 - 1 : 0;
  float2 a[NA];
  float2 b[NB > 0 ? NB : 1];

  __device__ __forceinline__ void init(float turns2) {  // W^k = exp(i pi turns2)
    float sn, cs;
    sincospif(turns2, &sn, &cs);
    a[0] = make_float2(cs, sn);
    if constexpr (NA > 1) {
      a[1] = c_mul(a[0], a[0]);
      a[2] = c_mul(a[1], a[0]);
    }
    if constexpr (NB > 0) {
      const float2 w4 = c_mul(a[1], a[1]);
      b[0] = w4;
#pragma unroll
      for (int i = 1; i < NB; ++i) b[i] = c_mul(b[i - 1], w4);
    }
  }

  // Make the bases opaque to the optimiser for one loop iteration, so that the
  // twiddles formed from them are recomputed next to their use instead of
  // being hoisted out of the caller's loop into extra registers.
  __device__ __forceinline__ void launder() {
#pragma unroll
    for (int i = 0; i < NA; ++i) asm volatile("" : "+f"(a[i].x), "+f"(a[i].y));
    if constexpr (NB > 0) {
#pragma unroll
      for (int i = 0; i < NB; ++i) asm volatile("" : "+f"(b[i].x), "+f"(b[i].y));
    }
  }

  template <int S>
  __device__ __forceinline__ float2 get() const {
    constexpr int lo = S & 3, hi = S >> 2;
    if constexpr (hi == 0) return a[lo - 1];
    else if constexpr (lo == 0) return b[hi - 1];
    else return c_mul(a[lo - 1], b[hi - 1]);
  }
};

// Radix-16 passes keep w, w^2, w^4, w^8 for dft16_tw.
struct TwBase16 {
  float2 w1, w2, w4, w8;
  __device__ __forceinline__ void init(float turns2) {
    float sn, cs;
    sincospif(turns2, &sn, &cs);
    w1 = make_float2(cs, sn);
    w2 = c_mul(w1, w1);
    w4 = c_mul(w2, w2);
    w8 = c_mul(w4, w4);
  }
  __device__ __forceinline__ void launder() {
    asm volatile("" : "+f"(w1.x), "+f"(w1.y), "+f"(w2.x), "+f"(w2.y));
    asm volatile("" : "+f"(w4.x), "+f"(w4.y), "+f"(w8.x), "+f"(w8.y));
  }
};

template <int R>
struct TwSel {
  using type = TwBase<R>;
};
template <>
struct TwSel<16> {
  using type = TwBase16;
};

template <int R, int S, bool LAST>
struct TwApply {
  __device__ __forceinline__ static void run(float2 (&u)[R], const TwBase<R>& t) {
    u[S] = c_mul(u[S], t.template get<S>());
    if constexpr (!LAST) TwApply<R, S + 1, S + 2 == R>::run(u, t);
  }
};

// Twiddle bases of every pass of an N-point transform for thread j.
template <int N, int E, bool INV, int NS = 1>
struct FftTw {
  static constexpr int R = PassRadix<N, NS, E>::value;
  static constexpr int Q = E / R;
  static constexpr int T = N / E;
  typename TwSel<R>::type tw[NS > 1 ? Q : 1];
  FftTw<N, E, INV, NS * R> next;

  __device__ __forceinline__ void init(int j) {
    if constexpr (NS > 1) {
      constexpr float scale = (INV ? 2.f : -2.f) / float(NS * R);
#pragma unroll
      for (int q = 0; q < Q; ++q) tw[q].init(scale * float((j + T * q) & (NS - 1)));
    }
    next.init(j);
  }

  __device__ __forceinline__ void launder() {
    if constexpr (NS > 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) tw[q].launder();
    }
    next.launder();
  }
};

template <int N, int E, bool INV>
struct FftTw<N, E, INV, N> {
  __device__ __forceinline__ void init(int) {}
  __device__ __forceinline__ void launder() {}
};

template <int N, int E, int R, int NS, bool INV>
__device__ __forceinline__ void pass_compute_tw(float2 (&v)[E], const FftTw<N, E, INV, NS>& tw) {
  constexpr int Q = E / R;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float2 u[R];
#pragma unroll
    for (int s = 0; s < R; ++s) u[s] = v[q + Q * s];
    if constexpr (NS > 1 && R == 16) {
      dft16_tw<INV>(u, tw.tw[q].w1, tw.tw[q].w2, tw.tw[q].w4, tw.tw[q].w8);
    } else {
      if constexpr (NS > 1) TwApply<R, 1, R == 2>::run(u, tw.tw[q]);
      dft_r<R, INV>(u);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) v[q + Q * t] = u[t];
  }
}

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// fft_block with the twiddle bases precomputed in 'tw' (see FftTw).  'hook'
// runs once, right after the first CTA barrier of the transform: by then
// every thread has consumed the inputs it loaded before the transform.
template <int N, int E, bool INV, bool DOUBLE_BUF, int NS = 1, typename Hook = NoHook>
__device__ __forceinline__ void fft_block_tw(float2 (&v)[E], int j, float2* buf0, float2* buf1, int& phase,
                                             const FftTw<N, E, INV, NS>& tw, const Hook& hook = Hook()) {
  constexpr int R = PassRadix<N, NS, E>::value;
  pass_compute_tw<N, E, R, NS, INV>(v, tw);
  if constexpr (NS * R < N) {
    float2* buf = (DOUBLE_BUF && phase) ? buf1 : buf0;
    if constexpr (!DOUBLE_BUF) __syncthreads();
    pass_store<N, E, R, NS>(v, j, buf);
    __syncthreads();
    if constexpr (NS == 1) hook();
    gather_regs<N, E>(v, j, buf);
    if constexpr (DOUBLE_BUF) phase ^= 1;
    fft_block_tw<N, E, INV, DOUBLE_BUF, NS * R>(v, j, buf0, buf1, phase, tw.next);
  }
}

}  // namespace gnss

namespace gnss {

// ---------------------------------------------------------------------------
// Class-local schedule (16 elements per thread, T = N / 16 threads, N = 4096
// or 8192): one CTA-wide exchange per transform instead of P - 1.
//
// The first radix-16 pass (inputs at stride T, straight from registers)
// writes its output digit c into slot i with i mod 16 = c.  Every later
// Stockham pass reads x[J + T s'] and writes y[(J / NS) NS R + k + t NS] with
// NS a multiple of 16, so it maps slots of one residue class c = J mod 16 onto
// the same class: the rest of the transform is 16 independent T-point
// transforms, one per class.  In those passes thread t runs the butterflies
// J = jp + T q, jp = t / G + 16 (t mod G), G = T / 16, so class c = jp mod 16
// = t / G lives on the G lanes G c .. G c + G - 1 (half a warp at 4096, a
// warp at 8192); after
// the CTA barrier of the first exchange the later exchanges need only
// __syncwarp, in place in the same buffer (each class's lanes read its
// slots, then overwrite exactly them).  On exit thread t holds X[jp + T r]
// in v[r] at N = 4096.
//
// At N = 8192 the last pass is radix 2 (NS = 4096), and its two inputs
// y[m], y[m + 4096] come out of the radix-16 pass before it in the same
// register of lanes l and l ^ 16 (butterflies J and J + 256 of one class).
// The lane pair splits the 16 butterflies m = k + 256 t, k = jp mod 256: the
// low lane takes t < 8, the high lane t >= 8, and each sends the other the 8
// operands it needs by shuffle -- half the data moves, and no shared-memory
// exchange is left for that pass.  Thread t then holds X[b + 256 (r mod 8) +
// 4096 (r / 8)] in v[r], b = k + 2048 h, h = 1 on the high lane
// (ClassLocal::out_index).  Each butterfly keeps its twiddle (the same float
// argument of sincospif) and its arithmetic, so the results are those of the
// exchanged form bit for bit.
//
// Shared-memory slot of element i: i + i/16 + i/256.  The lanes of each
// half-warp then hit distinct bank pairs in every access of the schedule
// (first-pass stores at 16 t + u, class gathers at jp + T r, later stores at
// (J / NS) 16 NS + k + u NS), and every access is a per-thread base plus a
// compile-time offset.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad_cl(int i) { return i + (i >> 4) + (i >> 8); }
// pad_cl(x + d) - pad_cl(x) for the strides d of the schedule (no carries)
__host__ __device__ constexpr int cl_off(int d) { return d + d / 16 + d / 256; }

template <int N>
struct ClassLocal {
  static_assert(N == 4096 || N == 8192, "class-local schedule: N = 4096 or 8192, 16 per thread");
  static constexpr int E = 16, T = N / E, G = T / 16;
  static constexpr int smem_elems = N + N / 16 + N / 256;  // > pad_cl(N - 1)
  // thread of butterfly J (mod T) in the class passes (an involution when G = 16)
  __device__ __forceinline__ static int perm(int t) { return t / G + 16 * (t % G); }
  // first output of the lane-pair radix-2 butterflies of class index jp (N = 8192)
  __device__ __forceinline__ static int pair_base(int jp) { return (jp & 255) + 2048 * ((jp >> 8) & 1); }
  // element of X that class index jp holds in v[r] on exit: increasing in r,
  // and congruent to jp modulo 256 at both sizes
  __device__ __forceinline__ static int out_index(int jp, int r) {
    if constexpr (N == 8192) return pair_base(jp) + 256 * (r & 7) + 4096 * (r >> 3);
    else return jp + T * r;
  }
  // twiddle bases of every pass for class index jp; at 8192 the lane-pair
  // radix-2 pass runs butterflies pair_base(jp) + 256 i, i < 8
  template <bool INV>
  __device__ __forceinline__ static void init_twiddles(FftTw<N, 16, INV>& tw, int jp) {
    tw.init(jp);
    if constexpr (N == 8192) {
      auto& last = tw.next.next.next;  // NS = 4096, radix 2
      constexpr float scale = (INV ? 2.f : -2.f) / float(N);
      const int b = pair_base(jp);
#pragma unroll
      for (int i = 0; i < 8; ++i) last.tw[i].init(scale * float(b + 256 * i));
    }
  }
};

// ---------------------------------------------------------------------------
// Class-local schedule at N = 16384 (16 per thread, T = 1024 threads): radix
// 16, 16, 16, then 4.  After the first pass's CTA-wide exchange, class c =
// J mod 16 (1024 elements) lives on the 64 threads 64 c .. 64 c + 63 (warps
// 2c, 2c + 1), which run the NS = 16 and NS = 256 passes with one in-place
// exchange between them guarded by a barrier of those warps.  The NS = 256
// pass's butterflies J and J + 256 h (h < 4) write exactly the slots that the
// radix-4 butterflies m = J mod 256 + 256 t read, so the last exchange runs
// within those four threads -- placed on lanes l, l + 8, l + 16, l + 24 of
// one warp, it needs only __syncwarp.  The thread of quarter h = J / 256 then
// runs the radix-4 butterflies m = k + 256 (h + 4 i), i < 4, k = J mod 256,
// and ends holding X[m + 4096 s] in v[4 i + s] (out_index).
//
// Thread position p within the class runs butterfly J = c + 16 i', where i'
// takes p's bits in the order (0, 5, 1, 2, 4, 3); slot of element i:
// i + i/16 + i/256 + i/4096.  Every access of the schedule (first-pass
// stores at 16 t + u, class gathers at J + 1024 r, class stores at
// 256 (J / 16) + J mod 16 + 16 u, quad stores at 4096 h + k + 256 u, quad
// gathers at k + 256 (h + 4 i) + 4096 s) puts each half-warp on 16 distinct
// 8-byte bank pairs, and every offset from a thread's base is a compile-time
// constant (no carries); tests/test_class_local_schedules.py models the schedule on
// the host and checks both, the exchange groups and the output order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad_q(int i) { return i + (i >> 4) + (i >> 8) + (i >> 12); }
// pad_q(x + d) - pad_q(x) for the strides d of the 16384 schedule (no carries)
__host__ __device__ constexpr int q_off(int d) { return d + d / 16 + d / 256 + d / 4096; }

template <>
struct ClassLocal<16384> {
  static constexpr int N = 16384, E = 16, T = N / E, G = 64;
  static constexpr int smem_elems = N + N / 16 + N / 256 + N / 4096;  // > pad_q(N - 1)
  __device__ __forceinline__ static int perm(int t) {
    const int p = t & 63;
    const int ip = (p & 1) | (((p >> 5) & 1) << 1) | (((p >> 1) & 3) << 2) | (((p >> 4) & 1) << 4) |
                   (((p >> 3) & 1) << 5);
    return (t >> 6) + 16 * ip;
  }
  // the radix-4 butterfly i of class index jp
  __device__ __forceinline__ static int quad_m(int jp, int i) { return (jp & 255) + 256 * ((jp >> 8) + 4 * i); }
  __device__ __forceinline__ static int out_index(int jp, int r) { return quad_m(jp, r >> 2) + 4096 * (r & 3); }
  template <bool INV>
  __device__ __forceinline__ static void init_twiddles(FftTw<N, 16, INV>& tw, int jp) {
    tw.init(jp);  // the radix-16 passes (NS = 16, 256)
    auto& last = tw.next.next.next;  // NS = 4096, radix 4
    constexpr float scale = (INV ? 2.f : -2.f) / float(N);
#pragma unroll
    for (int i = 0; i < 4; ++i) last.tw[i].init(scale * float(quad_m(jp, i)));
  }
};

// ---------------------------------------------------------------------------
// Class-local schedule at N = 2048 (16 per thread, T = 128): radix 16, 16,
// then 8.  After the CTA-wide exchange class c = J mod 16 (128 elements)
// lives on 8 lanes of one warp, which run the NS = 16 pass and exchange in
// place under __syncwarp; the gather after it gives thread jp the inputs of
// its two radix-8 butterflies jp and jp + 128 of the last pass (x[jp + 128 r]),
// so that pass needs no exchange and ends with X[jp + 128 r] in v[r].
//
// Thread t's class index jp = c + 16 i takes c from t's bits (0, 1, 5, 6) and
// i from its bits (4, 2, 3); slot of element e: e + e/8 + e/128.  With these
// every access (first-pass stores at 16 t + u, class gathers at jp + 128 r,
// class stores at 256 (jp / 16) + jp mod 16 + 16 u) puts each half-warp on 16
// distinct 8-byte bank pairs and every offset from a thread's base is a
// compile-time constant (tests/test_class_local_schedules.py models it too).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad_2k(int e) { return e + (e >> 3) + (e >> 7); }
// pad_2k(x + d) - pad_2k(x) for the strides d of the 2048 schedule (no carries)
__host__ __device__ constexpr int off_2k(int d) { return d + d / 8 + d / 128; }

template <>
struct ClassLocal<2048> {
  static constexpr int N = 2048, E = 16, T = N / E, G = 8;
  static constexpr int smem_elems = N + N / 8 + N / 128;  // > pad_2k(N - 1)
  __device__ __forceinline__ static int perm(int t) {
    const int c = (t & 3) | (((t >> 5) & 3) << 2);
    const int i = ((t >> 4) & 1) | (((t >> 2) & 3) << 1);
    return c + 16 * i;
  }
  __device__ __forceinline__ static int out_index(int jp, int r) { return jp + T * r; }
  template <bool INV>
  __device__ __forceinline__ static void init_twiddles(FftTw<N, 16, INV>& tw, int jp) {
    tw.init(jp);  // NS = 16: k = jp mod 16; NS = 256 (radix 8): butterflies jp + 128 q
  }
};

// The radix-2 pass of N = 8192 across lanes l and l ^ 16 (see above).
template <bool INV>
__device__ __forceinline__ void lane_pair_radix2(float2 (&v)[16], int jp, const FftTw<8192, 16, INV, 4096>& tw) {
  const bool hi = (jp >> 8) & 1;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 send = hi ? v[i] : v[8 + i];
    float2 got;
    got.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
    got.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
    float2 u[2];
    u[0] = hi ? got : v[i];
    u[1] = hi ? v[8 + i] : got;
    TwApply<2, 1, true>::run(u, tw.tw[i]);
    dft_r<2, INV>(u);
    v[i] = u[0];
    v[8 + i] = u[1];
  }
}

template <int N, bool INV, int NS>
__device__ __forceinline__ void class_local_rest(float2 (&v)[16], int jp, float2* buf, const float2* g,
                                                 const FftTw<N, 16, INV, NS>& tw) {
  // g = buf + pad_cl(jp): both address the same exchange buffer (no restrict)
  constexpr int T = N / 16;
  constexpr int R = PassRadix<N, NS, 16>::value;
  constexpr int Q = 16 / R;
  pass_compute_tw<N, 16, R, NS, INV>(v, tw);
  if constexpr (N == 8192 && NS * R == N / 2) {
    lane_pair_radix2<INV>(v, jp, tw.next);
  } else if constexpr (NS * R < N) {
    __syncwarp();  // the class's lanes have read every slot of the class
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const unsigned J = (unsigned)(jp + T * q);
      float2* b = buf + pad_cl((int)((J / NS) * NS * R + (J & (NS - 1))));
#pragma unroll
      for (int t = 0; t < R; ++t) b[cl_off(t * NS)] = v[q + Q * t];
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = g[cl_off(T * r)];
    class_local_rest<N, INV, NS * R>(v, jp, buf, g, tw.next);
  }
}

template <int N, bool INV, typename Hook = NoHook>
__device__ __forceinline__ void fft_class_local(float2 (&v)[16], int t, float2* buf, const FftTw<N, 16, INV>& tw,
                                                const Hook& hook = Hook()) {
  constexpr int T = N / 16;
  // pass 1 (NS = 1): DFT16 over stride T; outputs to 16 t + u
  pass_compute_tw<N, 16, 16, 1, INV>(v, tw);
  {
    float2* b = buf + pad_cl(16 * t);
#pragma unroll
    for (int u = 0; u < 16; ++u) b[u] = v[u];
  }
  __syncthreads();
  hook();
  const int jp = ClassLocal<N>::perm(t);
  const float2* g = buf + pad_cl(jp);  // element jp + T r sits at g[cl_off(T r)]
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[cl_off(T * r)];
  class_local_rest<N, INV, 16>(v, jp, buf, g, tw.next);
}

}  // namespace gnss

namespace gnss {

// ---------------------------------------------------------------------------
// Two independent transforms per thread, interleaved.  Each pass runs the
// butterflies of both before either exchanges, and each exchange issues both
// transforms' stores (then loads) together, so the scheduler can overlap one
// transform's shared-memory latency and barrier with the other's arithmetic.
// Each transform's own operations are exactly those of the one-transform
// code, in the same order, so the results are bit-identical to it.
// ---------------------------------------------------------------------------
template <int N, bool INV, int NS>
__device__ __forceinline__ void class_local_rest2(float2 (&va)[16], float2 (&vb)[16], int jp, float2* bufa,
                                                  const float2* ga, float2* bufb, const float2* gb,
                                                  const FftTw<N, 16, INV, NS>& tw) {
  constexpr int T = N / 16;
  constexpr int R = PassRadix<N, NS, 16>::value;
  constexpr int Q = 16 / R;
  pass_compute_tw<N, 16, R, NS, INV>(va, tw);
  pass_compute_tw<N, 16, R, NS, INV>(vb, tw);
  if constexpr (N == 8192 && NS * R == N / 2) {
    lane_pair_radix2<INV>(va, jp, tw.next);
    lane_pair_radix2<INV>(vb, jp, tw.next);
  } else if constexpr (NS * R < N) {
    __syncwarp();  // the class's lanes have read every slot of the class
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const unsigned J = (unsigned)(jp + T * q);
      const int off = pad_cl((int)((J / NS) * NS * R + (J & (NS - 1))));
#pragma unroll
      for (int t = 0; t < R; ++t) {
        bufa[off + cl_off(t * NS)] = va[q + Q * t];
        bufb[off + cl_off(t * NS)] = vb[q + Q * t];
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      va[r] = ga[cl_off(T * r)];
      vb[r] = gb[cl_off(T * r)];
    }
    class_local_rest2<N, INV, NS * R>(va, vb, jp, bufa, ga, bufb, gb, tw.next);
  }
}

// Two class-local transforms (see fft_class_local) on buffers bufa, bufb.
// The caller guarantees that no thread still reads either buffer from an
// earlier transform (one CTA barrier before the first-pass stores below
// does that when the same two buffers serve every block).
template <int N, bool INV>
__device__ __forceinline__ void fft_class_local2(float2 (&va)[16], float2 (&vb)[16], int t, float2* bufa,
                                                 float2* bufb, const FftTw<N, 16, INV>& tw) {
  pass_compute_tw<N, 16, 16, 1, INV>(va, tw);
  pass_compute_tw<N, 16, 16, 1, INV>(vb, tw);
  __syncthreads();  // every thread has finished reading both buffers
  {
    float2* a = bufa + pad_cl(16 * t);
    float2* b = bufb + pad_cl(16 * t);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a[u] = va[u];
      b[u] = vb[u];
    }
  }
  __syncthreads();
  const int jp = ClassLocal<N>::perm(t);
  const float2* ga = bufa + pad_cl(jp);
  const float2* gb = bufb + pad_cl(jp);
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    va[r] = ga[cl_off((N / 16) * r)];
    vb[r] = gb[cl_off((N / 16) * r)];
  }
  class_local_rest2<N, INV, 16>(va, vb, jp, bufa, ga, bufb, gb, tw.next);
}

// Two Stockham transforms with cached twiddles (see fft_block_tw), on their
// own buffers; a CTA barrier guards each buffer's reuse.
template <int N, int E, bool INV, int NS = 1>
__device__ __forceinline__ void fft_block_tw2(float2 (&va)[E], float2 (&vb)[E], int j, float2* bufa, float2* bufb,
                                              const FftTw<N, E, INV, NS>& tw) {
  constexpr int R = PassRadix<N, NS, E>::value;
  pass_compute_tw<N, E, R, NS, INV>(va, tw);
  pass_compute_tw<N, E, R, NS, INV>(vb, tw);
  if constexpr (NS * R < N) {
    __syncthreads();  // both buffers are free
    pass_store<N, E, R, NS>(va, j, bufa);
    pass_store<N, E, R, NS>(vb, j, bufb);
    __syncthreads();
    gather_regs<N, E>(va, j, bufa);
    gather_regs<N, E>(vb, j, bufb);
    fft_block_tw2<N, E, INV, NS * R>(va, vb, j, bufa, bufb, tw.next);
  }
}

}  // namespace gnss

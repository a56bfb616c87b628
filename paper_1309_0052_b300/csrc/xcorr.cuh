// xcorr.cuh -- device pieces shared by the correlate kernels (sm_103a):
// launch configurations, programmatic dependent launch, the batched-launch
// request lookup, block reductions, per-row peak statistics and the per-PRN
// detection (second mixing + IFFT + detection of Section 3, Fig. 2).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fft.cuh"
#include "internal.h"

namespace gnss {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The carrier-FFT and correlate kernels are
// launched so that their CTAs may start while the kernel before them on the
// stream is still draining (launch latency and prologue overlap its tail);
// each waits for that kernel's completion and memory (griddep_wait) before
// it reads the kernel's output or writes anything.  The kernels before them
// allow this early launch as soon as they start (griddep_release): the
// dependent grid is scheduled only once every CTA of the primary has started,
// and it waits for all of them to finish.  Without the launch attribute the
// wait returns at once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Per-N launch configuration.  E = elements per thread, T = N / E threads.
// ---------------------------------------------------------------------------
template <int N>
struct Cfg {
  static constexpr int E = N >= 16384 ? 32 : 16;
  static constexpr int T = N / E;
  static constexpr bool TWC = (E <= 16);                        // twiddle bases cached in registers
  static constexpr size_t buf_bytes = sizeof(float2) * FftShape<N>::smem_elems;
  static constexpr bool DB = 2 * buf_bytes <= 160 * 1024;     // ping-pong exchange buffers
  static constexpr size_t smem = (DB ? 2 : 1) * buf_bytes;
  static constexpr int MINB = T <= 256 ? 2 : 1;
};

// Launch configuration of the correlate kernel with E elements per thread
// (a tuning choice: 8, 16 or 32, see xcorr_variant).  With ST the next block's
// spectrum is staged into shared memory by a bulk TMA copy (N * 8 bytes more).
// With CL the transform runs the class-local schedule (N = 4096 or 8192,
// E = 16: one CTA barrier per block; fft_class_local).
template <int N, int E, bool ST = false, bool CL = false>
struct XCfg {
  static_assert(!CL || ((N == 2048 || N == 4096 || N == 8192 || N == 16384) && E == 16 && !ST),
                "class-local schedule: N = 2048 ... 16384");
  static constexpr int T = N / E;
  static constexpr bool TWC = (E <= 16);                        // twiddle bases cached in registers
  static constexpr size_t buf_bytes =
      sizeof(float2) * (CL ? ClassLocal<(CL ? N : 4096)>::smem_elems : FftShape<N>::smem_elems);
  static constexpr bool DB = 2 * buf_bytes <= 160 * 1024;     // ping-pong exchange buffers
  static constexpr size_t stage_off = (DB || CL ? 2 : 1) * buf_bytes;
  // At 16384 with 32 per thread, sums 8-31 of each thread live in
  // thread-private shared memory (slot (r - 8) T + j, 48 KB): 32 data and 32
  // sum registers do not fit 128 with the passes' temporaries, and the
  // spills cost more than these slots (measured: 8 sums in registers beat
  // 4, 12, 16 and none).
  static constexpr bool SHACC = N == 16384 && E == 32 && !CL && !ST;
  static constexpr size_t sacc_off = stage_off + (ST ? sizeof(float2) * N : 0);
  static constexpr size_t smem = sacc_off + (SHACC ? sizeof(float) * (E - 8) * T : 0);
  // CTAs per SM the registers must allow: a budget of 128 registers per
  // thread (two 256-thread CTAs, four of 128, ...; registers are allocated
  // per warp, so CTAs under 32 threads count as one warp), 64 at 512 threads
  // with E = 8
  static constexpr int MINB = T <= 256 ? 512 / (T < 32 ? 32 : T) : (E <= 8 && T <= 512) ? 2 : 1;
  static_assert(stage_off % 16 == 0, "bulk copies need a 16-byte aligned destination");
};

// Staging is offered with 16 elements per thread when the CTA still fits.
template <int N>
struct StageFits {
  static constexpr bool value = XCfg<N, 16, true>::smem <= 227 * 1024;
};

// Request of a batched launch that owns CTA blockIdx.x: base[r] <= blockIdx.x
// < base[r + 1] (base ascending, base[0] = 0).  One probe per thread.
__device__ __forceinline__ int find_request(const uint32_t* __restrict__ base, int n, unsigned tile) {
  __shared__ int s_req;
  for (int r = threadIdx.x; r < n; r += blockDim.x)
    if (__ldg(base + r) <= tile && tile < __ldg(base + r + 1)) s_req = r;
  __syncthreads();
  return s_req;
}
__device__ __forceinline__ int find_request(const uint32_t* __restrict__ base, int n) {
  return find_request(base, n, blockIdx.x);
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

template <int T>
__device__ __forceinline__ uint32_t block_min_u32(uint32_t v, uint32_t* s_idx) {
  constexpr int W = (T + 31) / 32;
#pragma unroll
  for (int o = WarpShape<T>::first; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(WarpShape<T>::mask, v, o));
  if constexpr (W > 1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_idx[warp] = v;
    __syncthreads();
    v = s_idx[0];
#pragma unroll
    for (int w = 1; w < W; ++w) v = min(v, s_idx[w]);
  }
  return v;
}

// Row statistics of one (PRN, Doppler) row held as a[r] = S[j + T r]:
// peak = max S, tau = the smallest phase holding it, second = max S over the
// phases whose circular distance to tau exceeds excl (0 if none).  Only the
// threads whose own maximum is the peak search their phases for it, and only
// the threads that can hold a phase inside the band (their phases are
// congruent modulo a period P >= 2 excl + 1, so the band meets a thread only
// if its residue lies within excl of tau's) scan their cells for the second
// peak; every other thread's contribution is its own maximum.
// Phase held in accumulator r by the thread with butterfly index j: j + T r,
// or the class-local schedule's output order.  Phases grow with r, and all
// phases of a thread are congruent to j modulo 'period'.
template <int N, int E, bool CL>
struct PhaseMap {
  // with the lane-pair (8192) or quad (16384) last pass a thread's phases are
  // all congruent to its class index modulo 256
  static constexpr bool pairs = CL && (N == 8192 || N == 16384);
  static constexpr int period = pairs ? 256 : N / E;
  __device__ __forceinline__ static int at(int j, int r) {
    if constexpr (pairs) return ClassLocal<(pairs ? N : 8192)>::out_index(j, r);
    else return j + (N / E) * r;
  }
};

template <int N, int E, bool CL>
__device__ __forceinline__ void row_stats(const float (&a)[E], int j, int excl, float* s_val, uint32_t* s_idx,
                                          RowStat* out) {
  constexpr int T = N / E;
  using M = PhaseMap<N, E, CL>;
  float tmax = a[0];
#pragma unroll
  for (int r = 1; r < E; ++r) tmax = fmaxf(tmax, a[r]);
  const float best = block_max<T>(tmax, s_val);
  uint32_t bt = 0xffffffffu;
  if (tmax == best) {
#pragma unroll
    for (int r = E - 1; r >= 0; --r)
      if (a[r] == best) bt = (uint32_t)M::at(j, r);
  }
  bt = block_min_u32<T>(bt, s_idx);
  float sec = tmax;
  if (2 * excl + 1 > M::period || ((j - (int)bt + excl) & (M::period - 1)) <= 2 * excl) {
    sec = 0.f;  // every cell is >= 0
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int dist = abs(M::at(j, r) - (int)bt);
      dist = min(dist, N - dist);
      if (dist > excl) sec = fmaxf(sec, a[r]);
    }
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

// Per-PRN detection, run by the last CTA to finish a PRN (all its threads):
// best row over the Doppler bins (ties to the smallest bin), its second
// peak (or, with GNSS_SECOND_WHOLE, the largest surface cell outside the
// exclusion band around the peak phase), ratio, and the half-bit set with
// the larger ratio (ties to set 0).  Rows and surface cells written by other
// CTAs are read through L2.
template <int N, int T>
__device__ __forceinline__ void finalize_prn(const XcorrArgs& a, int p, int sets, float* s_val, uint32_t* s_idx) {
  float best_ratio = -1.f;
  gnss_detection rec;
  for (int s = 0; s < sets; ++s) {
    const RowStat* rs = a.rows + ((size_t)s * a.P + p) * a.D;
    float v = -1.f;
    uint32_t db = 0;
    for (int d = threadIdx.x; d < a.D; d += T) {
      const float pk = __ldcg(&rs[d].peak);
      if (pk > v) {
        v = pk;
        db = (uint32_t)d;
      }
    }
    block_argmax<T>(v, db, s_val, s_idx);
    const float4 raw = __ldcg(reinterpret_cast<const float4*>(rs + db));
    const float peak = raw.x;
    const uint32_t tau = __float_as_uint(raw.y);
    float second = raw.z;
    if (a.second_whole) {
      const float* S = a.surface + ((size_t)s * a.P + p) * a.D * (size_t)N;
      float m = 0.f;
      for (int idx = threadIdx.x; idx < a.D * N; idx += T) {
        const int t = idx & (N - 1);
        int dist = abs(t - (int)tau);
        dist = min(dist, N - dist);
        if (dist > a.excl) m = fmaxf(m, __ldcg(S + idx));
      }
      second = block_max<T>(m, s_val);
    }
    const float ratio = second > 0.f ? peak / second : INFINITY;
    if (s == 0 || ratio > best_ratio) {
      best_ratio = ratio;
      rec.prn = (uint8_t)a.prns[p];
      rec.set = (uint8_t)s;
      rec.flags = (uint8_t)__ldcg(a.counters + a.P);  // this call's status word
      rec.dopp_bin = (int32_t)db;
      rec.dopp_hz = a.dopp_min + (int32_t)db * a.dopp_step;
      rec.code_phase = tau;
      rec.peak = peak;
      rec.second = second;
      rec.ratio = ratio;
    }
  }
  rec.detected = (uint8_t)(best_ratio >= a.threshold);
  if (threadIdx.x == 0) a.out[p] = rec;
}

// Host side: dynamic shared memory above 48 KB, and the dependent launch.
template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Launch with programmatic stream serialization (see griddep_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                                   cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace gnss

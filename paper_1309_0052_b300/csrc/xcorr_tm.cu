// xcorr_tm.cu -- the correlate kernel (second mixing, IFFT, |.|^2 and the
// non-coherent sum of Section 3, Fig. 2, then the detection) with the SM's
// tensor memory as an extension of the register file (sm_103a).
//
// Every correlate CTA multiplies each block's spectrum Y by conj(C_p) of its
// PRN and adds |IFFT|^2 into per-thread sums.  In the register form C_p is
// re-read from L2 for every block (it shares the L1/shared-memory data path
// with the FFT's exchanges), the sums take registers, and the block's Y loads
// stall the CTA for an L2 round trip at every block start.  Here:
//   - C_p of the CTA's PRNs is written once into tensor memory (TMEM: 128
//     lanes x 512 columns of 32 bits per SM, beside the register file and
//     shared memory) and read back each block with tcgen05.ld, off the
//     L1/shared path;
//   - the registers this frees hold the NEXT block's Y, loaded right after
//     the current block's products are formed, so its L2 latency passes
//     under the current block's transform (16 elements per thread);
//   - where the registers cannot also hold the non-coherent sums (two PRNs
//     per CTA, 32 elements per thread at N = 16384, or the occupancy form)
//     those live in TMEM too (tcgen05.ld, add and tcgen05.st around each
//     block's |.|^2).
// A CTA can take K PRNs of one Doppler bin (one Y load feeds K products and
// K transforms) and M bins one after another (the code spectra stay in
// TMEM across bins).
//
// TMEM layout.  tcgen05.ld/st of shape 32x32b give lane i of warp w TMEM lane
// 32 (w % 4) + i, so the warps w, w + 4, ... share a lane quarter and take
// consecutive column slots: C_i (2E columns, E complex values in the thread's
// FFT input order) at 2E i and, with TMEM sums, the sums of PRN i (E columns)
// at 2E K + E i.  The CTA allocates the next power of two >= 32 of slots x
// slot width with tcgen05.alloc and frees them before it leaves.
// tcgen05.alloc waits while the SM's 512 columns are taken, so the host only
// offers a shape whose CTAs that fit on one SM together take at most 512
// columns, and a CTA allocates after its grid-dependency wait and waits for
// nothing while it holds columns (an allocation can then only wait for CTAs
// that run to their end).
//
// The arithmetic of a block is that of the register form operation for
// operation (the same products, transform and sums in the same order), so the
// surfaces and records are identical to it bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fft.cuh"
#include "internal.h"
#include "xcorr.cuh"

namespace gnss {

// ---------------------------------------------------------------------------
// tcgen05 primitives (one CTA, cta_group::1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tm_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Whole warp: allocate COLS columns (all 128 lanes); the TMEM address of the
// first column lands in *dst (shared memory).
template <int COLS>
__device__ __forceinline__ void tm_alloc(uint32_t* dst) {
  static_assert(COLS >= 32 && COLS <= 512 && (COLS & (COLS - 1)) == 0, "TMEM columns: a power of two in 32..512");
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tm_smem_addr(dst)),
               "n"(COLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Whole warp (the one that allocated): free them.
template <int COLS>
__device__ __forceinline__ void tm_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(COLS) : "memory");
}
// Order TMEM accesses before / after a CTA barrier.
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Wait until this thread's earlier tcgen05.st have completed.
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// TMEM columns [c, c + 16) of the warp's lane quarter -> r[0 .. 16) of each
// thread (lane i of the warp reads TMEM lane 32 (warp % 4) + i; ta carries
// that lane base and c).  Asynchronous: the values are valid after
// tm_wait_ld16(r).
__device__ __forceinline__ void tm_ld16(uint32_t ta, float (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
               "%14,%15}, [%16];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]),
               "=f"(r[6]), "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]),
               "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
               : "r"(ta));
}
// Wait for this thread's TMEM loads.  r is tied to the wait, so no use of
// the loaded values can be scheduled before it.
__device__ __forceinline__ void tm_wait_ld16(float (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]),
               "+f"(r[6]), "+f"(r[7]), "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]),
               "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15])
               :
               : "memory");
}
__device__ __forceinline__ void tm_st16(uint32_t ta, const float (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
               "%13,%14,%15,%16};"
               :
               : "r"(ta), "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]),
               "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]), "f"(r[10]), "f"(r[11]),
               "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
               : "memory");
}

// TMEM columns [c, c + 32) of the warp's lane quarter -> r[0 .. 32) of each
// thread (lane i of the warp reads TMEM lane 32 (warp % 4) + i; ta carries
// that lane base and c).  Asynchronous: the values are valid after
// tm_wait_ld32(r).
__device__ __forceinline__ void tm_ld32(uint32_t ta, float (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
               "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]),
               "=f"(r[6]), "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]),
               "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15]), "=f"(r[16]), "=f"(r[17]),
               "=f"(r[18]), "=f"(r[19]), "=f"(r[20]), "=f"(r[21]), "=f"(r[22]), "=f"(r[23]),
               "=f"(r[24]), "=f"(r[25]), "=f"(r[26]), "=f"(r[27]), "=f"(r[28]), "=f"(r[29]),
               "=f"(r[30]), "=f"(r[31])
               : "r"(ta));
}
// Wait for this thread's TMEM loads.  r is tied to the wait, so no use of
// the loaded values can be scheduled before it.
__device__ __forceinline__ void tm_wait_ld32(float (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]),
               "+f"(r[6]), "+f"(r[7]), "+f"(r[8]), "+f"(r[9]), "+f"(r[10]), "+f"(r[11]),
               "+f"(r[12]), "+f"(r[13]), "+f"(r[14]), "+f"(r[15]), "+f"(r[16]), "+f"(r[17]),
               "+f"(r[18]), "+f"(r[19]), "+f"(r[20]), "+f"(r[21]), "+f"(r[22]), "+f"(r[23]),
               "+f"(r[24]), "+f"(r[25]), "+f"(r[26]), "+f"(r[27]), "+f"(r[28]), "+f"(r[29]),
               "+f"(r[30]), "+f"(r[31])
               :
               : "memory");
}
__device__ __forceinline__ void tm_st32(uint32_t ta, const float (&r)[32]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
               "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
               :
               : "r"(ta), "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]),
               "f"(r[6]), "f"(r[7]), "f"(r[8]), "f"(r[9]), "f"(r[10]), "f"(r[11]),
               "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15]), "f"(r[16]), "f"(r[17]),
               "f"(r[18]), "f"(r[19]), "f"(r[20]), "f"(r[21]), "f"(r[22]), "f"(r[23]),
               "f"(r[24]), "f"(r[25]), "f"(r[26]), "f"(r[27]), "f"(r[28]), "f"(r[29]),
               "f"(r[30]), "f"(r[31])
               : "memory");
}
// 8 columns (the twiddle bases of one radix-16 pass): load and tied wait.
__device__ __forceinline__ void tm_ld8(uint32_t ta, float (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]),
               "=f"(r[6]), "=f"(r[7])
               : "r"(ta));
}
__device__ __forceinline__ void tm_wait_ld8(float (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3]), "+f"(r[4]), "+f"(r[5]),
               "+f"(r[6]), "+f"(r[7])
               :
               : "memory");
}

// ---------------------------------------------------------------------------
// Launch shape of the TMEM variant: E = 16 elements per thread (class-local
// schedule at 4096 and 8192, cached twiddles otherwise) with the next block
// prefetched into registers, or E = 32 at N = 16384 without the prefetch.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tm_pow2_cols(int c) { return c <= 32 ? 32 : 2 * tm_pow2_cols((c + 1) / 2); }

template <int N, int E, bool O = false>
struct TmShape {
  static constexpr bool CL = (N == 4096 || N == 8192 || ((N == 2048 || N == 16384) && O)) && E == 16;
  using X = XCfg<N, E, false, CL>;
  static constexpr int T = N / E;
  static_assert(T >= 32, "tcgen05.ld/st run on whole warps");
  static constexpr int WARPS = T / 32;
  static constexpr int SLOTS = WARPS >= 4 ? WARPS / 4 : 1;  // warps sharing a lane quarter
  // The occupancy form (O): more CTAs per SM, so more warps hide latency --
  // the sums in TMEM and no register prefetch.  Every size it is built for
  // runs the class-local schedule (ONEBUF) at 64 registers with ONE exchange
  // buffer per CTA (without it the form would cap registers at 80 for three
  // 256-thread CTAs): eight 128-thread CTAs at 2048 (8 x (18 + 8) KB of
  // shared memory: the buffer and the radix-8 pass's bases; 8 x 64 TMEM
  // columns), four 256-thread CTAs at 4096 (4 x 35 KB, 4 x 128 columns), two
  // 512-thread CTAs at 8192 (2 x (70 + 32) KB with the lane-pair pass's
  // twiddle table; 2 x 256 columns), one 1024-thread CTA at 16384 (140 + 32
  // KB; all 512 columns) -- 32 warps per SM in each case.  The buffer's reuse
  // by the next transform waits on an mbarrier that every thread arrives on
  // after its last read (fft_cl_tmtw), so the wait falls a whole pass after
  // the arrivals.
  static constexpr bool ONEBUF = O && CL;
  static constexpr int MINB = O ? (ONEBUF ? 65536 / (64 * T) : T <= 256 ? 768 / T : 1) : X::MINB;
  // last-pass twiddles per thread: float4 [4][T] at 8192 (the lane-pair
  // pass's W^(b + 256 i), i < 8), float4 [2][T] at 16384 (the radix-4 pass's
  // W^m of its four butterflies), float4 [4][T] at 2048 (the radix-8 pass's
  // bases w, w^2, w^3, w^4 of its two butterflies)
  static constexpr int lp_vec = ONEBUF ? (N == 8192 || N == 2048 ? 4 : N == 16384 ? 2 : 0) : 0;
  static constexpr size_t lp_bytes = (size_t)lp_vec * T * sizeof(float4);
  static constexpr size_t smem = ((X::DB || CL) && !ONEBUF ? 2 : 1) * X::buf_bytes + lp_bytes;
  template <int K>
  struct Cols {
    // sums in registers with one PRN of 16 elements; else E TMEM columns per PRN
    static constexpr bool acc_regs = E == 16 && K == 1 && !O;
    // the next block's Y prefetched into registers (one PRN of 16 per thread;
    // two PRNs run their transforms interleaved instead, see fft_class_local2)
    static constexpr bool prefetch = E == 16 && K == 1 && !O;
    static constexpr int per_prn = acc_regs ? 2 * E : 3 * E;
    // the class-local occupancy form keeps the two twiddled radix-16 passes'
    // bases (w, w^2, w^4, w^8 each: 16 floats) in TMEM too, after the PRNs'
    // columns
    static constexpr bool tw_tmem = O && CL;
    static constexpr int tw_cols = tw_tmem ? 16 : 0;
    static constexpr int stride = (K * per_prn + tw_cols + 31) / 32 * 32;  // columns of one warp slot
    static constexpr int alloc = tm_pow2_cols(SLOTS * stride);
    static_assert(alloc <= 512, "TMEM has 512 columns");
  };
};

// Element js + T r (r < E) of a spectrum row, js = j + ksh: only the last
// can wrap around the row (ksh < 16 <= T: spectrum classes are cut so).
template <int N, int E>
__device__ __forceinline__ void tm_load_row(float2 (&y)[E], const float2* __restrict__ row, int js) {
  constexpr int T = N / E;
  const float2* ys = row + js;
#pragma unroll
  for (int r = 0; r < E - 1; ++r) y[r] = __ldcg(ys + T * r);
  const int last = js + T * (E - 1);
  y[E - 1] = __ldcg(row + (last >= N ? last - N : last));
}

// v = y * conj(C) with C read from TMEM columns ta .. ta + 2E (y and v may
// be the same array).  With 16 elements one 32-column load; with 32, where
// the elements already fill half the registers, 16 columns at a time.
template <int E>
__device__ __forceinline__ void tm_product(uint32_t ta, const float2 (&y)[E], float2 (&v)[E]) {
  if constexpr (E == 16) {
    float c[32];
    tm_ld32(ta, c);
    tm_wait_ld32(c);
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = c_mulconj(y[q], make_float2(c[2 * q], c[2 * q + 1]));
  } else {
#pragma unroll
    for (int h = 0; h < E / 8; ++h) {
      float c[16];
      tm_ld16(ta + 16u * h, c);
      tm_wait_ld16(c);
#pragma unroll
      for (int q = 0; q < 8; ++q) v[8 * h + q] = c_mulconj(y[8 * h + q], make_float2(c[2 * q], c[2 * q + 1]));
    }
  }
}

// |v|^2 added to sums t (the register form's order of operations).
template <int E>
__device__ __forceinline__ void add_power(float (&t)[E], const float2 (&v)[E]) {
#pragma unroll
  for (int r = 0; r < E; ++r) t[r] = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, t[r]));
}

// Sums of E = 32 at TMEM columns ta .. ta + 32, 16 at a time: += |v|^2 (zero
// before the first block of a set).
__device__ __forceinline__ void tm_accumulate32(uint32_t ta, const float2 (&v)[32], bool first) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float t[16];
    if (first) {
#pragma unroll
      for (int q = 0; q < 16; ++q) t[q] = 0.f;
    } else {
      tm_wait_st();  // this thread's previous update of these columns has landed
      tm_ld16(ta + 16u * h, t);
      tm_wait_ld16(t);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float2 w = v[16 * h + q];
      t[q] = fmaf(w.x, w.x, fmaf(w.y, w.y, t[q]));
    }
    tm_st16(ta + 16u * h, t);
  }
}

template <int E>
__device__ __forceinline__ void tm_read_sums(uint32_t ta, float (&acc)[E]) {
  tm_wait_st();
#pragma unroll
  for (int h = 0; h < E / 16; ++h) {
    float t[16];
    tm_ld16(ta + 16u * h, t);
    tm_wait_ld16(t);
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[16 * h + q] = t[q];
  }
}

// The class-local 4096- or 8192-point inverse transform (fft_class_local,
// the same passes and operations) with each twiddled radix-16 pass's bases
// read from TMEM columns ta .. ta + 8 (pass NS = 16) and ta + 8 .. ta + 16
// (NS = 256) right before the pass, and at 8192 the lane-pair radix-2 pass's
// eight twiddles read from this thread's column of a shared-memory table:
// 16 (32) registers fewer live through the transform.
__device__ __forceinline__ TwBase16 tw_unpack(const float (&w)[8]) {
  TwBase16 b;
  b.w1 = make_float2(w[0], w[1]);
  b.w2 = make_float2(w[2], w[3]);
  b.w4 = make_float2(w[4], w[5]);
  b.w8 = make_float2(w[6], w[7]);
  return b;
}

__device__ __forceinline__ void tw_to_tmem(const TwBase16& a, const TwBase16& b, uint32_t ta) {
  const float w[16] = {a.w1.x, a.w1.y, a.w2.x, a.w2.y, a.w4.x, a.w4.y, a.w8.x, a.w8.y,
                       b.w1.x, b.w1.y, b.w2.x, b.w2.y, b.w4.x, b.w4.y, b.w8.x, b.w8.y};
  tm_st16(ta, w);
}

//
// With one exchange buffer per CTA (TmShape::ONEBUF) the first-pass stores of
// a transform must not land while another warp still reads the previous
// transform's classes.  An mbarrier of T arrivals per transform orders them:
// each thread arrives right after its last read of the buffer (the class
// gathers before the NS = 256 pass) and waits for that phase only before its
// next first-pass stores, so the wait spans the NS = 256 pass, the sums,
// the next block's loads and products and the next first pass.  Each wait
// polls at most g_buf_wait_limit times; one that gives up marks the call's
// status word (GNSS_DET_WAIT_TIMEOUT: the call's results are not valid) and
// goes on, so the CTA still finishes and frees its TMEM.  (The limit is
// lowered only by the testing entry point: at 0 every wait gives up at once
// and the CTA's warps race on the buffer -- in bounds, results flagged.)
__device__ unsigned g_buf_wait_limit = 1u << 22;

struct BufRelease {
  uint64_t* bar;     // the CTA's mbarrier (shared memory), T arrivals per phase
  unsigned* status;  // the call's status word
  uint32_t n;        // transforms this thread has run
};

__device__ __forceinline__ uint32_t tm_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void buf_release_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tm_smem_u32(bar)), "r"(count) : "memory");
}

// release: this thread's reads of the buffer are ordered before the arrival
__device__ __forceinline__ void buf_release_arrive(BufRelease& rel) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tm_smem_u32(rel.bar)) : "memory");
  ++rel.n;
}

// acquire: every thread's reads of the previous transform precede this
// thread's stores (no wait before a CTA's first transform)
__device__ __forceinline__ void buf_release_wait(const BufRelease& rel) {
  if (rel.n == 0) return;
  const uint32_t parity = (rel.n - 1) & 1u;
  const unsigned limit = g_buf_wait_limit;
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(tm_smem_u32(rel.bar)), "r"(parity)
        : "memory");
    if (done) return;
  }
  atomicOr(rel.status, (unsigned)GNSS_DET_WAIT_TIMEOUT);
}

template <int N, bool ONEBUF>
__device__ __forceinline__ void fft_cl_tmtw(float2 (&v)[16], int t, float2* buf, uint32_t ta_tw, BufRelease& rel,
                                            const float4* lp) {
  constexpr int T = N / 16;
  {
    FftTw<N, 16, true, 1> none;  // pass 1 (NS = 1) takes no twiddles
    pass_compute_tw<N, 16, 16, 1, true>(v, none);
  }
  if constexpr (ONEBUF) buf_release_wait(rel);
  {
    float2* b = buf + pad_cl(16 * t);
#pragma unroll
    for (int u = 0; u < 16; ++u) b[u] = v[u];
  }
  // each pass's bases are requested one exchange ahead, so the TMEM load
  // completes under the barrier and the gathers
  float w[8];
  tm_ld8(ta_tw, w);
  __syncthreads();
  const int jp = ClassLocal<N>::perm(t);
  const float2* g = buf + pad_cl(jp);  // element jp + T r sits at g[cl_off(T r)]
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[cl_off(T * r)];
  {
    tm_wait_ld8(w);
    FftTw<N, 16, true, 16> tw;
    tw.tw[0] = tw_unpack(w);
    pass_compute_tw<N, 16, 16, 16, true>(v, tw);
  }
  tm_ld8(ta_tw + 8u, w);
  __syncwarp();  // the class's lanes have read every slot of the class
  {
    // butterfly jp of the NS = 16 pass writes y[(jp / 16) 256 + (jp mod 16) + 16 u]
    float2* b = buf + pad_cl((jp / 16) * 256 + (jp & 15));
#pragma unroll
    for (int u = 0; u < 16; ++u) b[cl_off(16 * u)] = v[u];
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[cl_off(T * r)];
  if constexpr (ONEBUF) buf_release_arrive(rel);  // the last read of the buffer in this transform
  {
    tm_wait_ld8(w);
    FftTw<N, 16, true, 256> tw;
    tw.tw[0] = tw_unpack(w);
    pass_compute_tw<N, 16, 16, 256, true>(v, tw);
  }
  if constexpr (N == 8192) {
    FftTw<N, 16, true, 4096> lt;
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float4 x = lp[T * h + t];
      lt.tw[2 * h].a[0] = make_float2(x.x, x.y);
      lt.tw[2 * h + 1].a[0] = make_float2(x.z, x.w);
    }
    lane_pair_radix2<true>(v, jp, lt);
  }
}

// Barrier of the four warps 4 g .. 4 g + 3 (the two 16384-point classes 2 g,
// 2 g + 1): named barrier 1 + g of 128 threads.
__device__ __forceinline__ void class_pair_sync(int warp) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + (warp >> 2)) : "memory");
}

// The class-local 16384-point inverse transform (ClassLocal<16384>): the
// radix-16 passes NS = 16 and 256 with their bases from TMEM columns ta ..
// ta + 16, the radix-4 pass with W^m of its four butterflies from this
// thread's column of the shared-memory table (W^2m, W^3m formed as in
// TwBase<4>::init).  One CTA barrier, one barrier of the class's warps and two
// __syncwarp per transform; the buffer's reuse waits on 'rel' as above.
__device__ __forceinline__ void fft16384_cl_tmtw(float2 (&v)[16], int t, float2* buf, uint32_t ta_tw,
                                                 BufRelease& rel, const float4* lp) {
  constexpr int N = 16384, T = N / 16;
  using CLq = ClassLocal<N>;
  {
    FftTw<N, 16, true, 1> none;  // pass 1 (NS = 1) takes no twiddles
    pass_compute_tw<N, 16, 16, 1, true>(v, none);
  }
  buf_release_wait(rel);
  {
    float2* b = buf + pad_q(16 * t);
#pragma unroll
    for (int u = 0; u < 16; ++u) b[u] = v[u];
  }
  float w[8];
  tm_ld8(ta_tw, w);
  __syncthreads();
  const int jp = CLq::perm(t);
  const float2* g = buf + pad_q(jp);  // element jp + T r sits at g[q_off(T r)]
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[q_off(T * r)];
  {
    tm_wait_ld8(w);
    FftTw<N, 16, true, 16> tw;
    tw.tw[0] = tw_unpack(w);
    pass_compute_tw<N, 16, 16, 16, true>(v, tw);
  }
  tm_ld8(ta_tw + 8u, w);
  const int warp = t >> 5;
  class_pair_sync(warp);  // the class's warps have read every slot of the class
  {
    // butterfly jp of the NS = 16 pass writes y[(jp / 16) 256 + (jp mod 16) + 16 u]
    float2* b = buf + pad_q((jp >> 4) * 256 + (jp & 15));
#pragma unroll
    for (int u = 0; u < 16; ++u) b[q_off(16 * u)] = v[u];
  }
  class_pair_sync(warp);
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[q_off(T * r)];
  {
    tm_wait_ld8(w);
    FftTw<N, 16, true, 256> tw;
    tw.tw[0] = tw_unpack(w);
    pass_compute_tw<N, 16, 16, 256, true>(v, tw);
  }
  const int h = jp >> 8, k = jp & 255;
  __syncwarp();  // the four lanes of this k have read their slots
  {
    // butterfly jp of the NS = 256 pass writes y[4096 h + k + 256 u]
    float2* b = buf + pad_q(4096 * h + k);
#pragma unroll
    for (int u = 0; u < 16; ++u) b[q_off(256 * u)] = v[u];
  }
  __syncwarp();
  {
    // radix-4 butterfly i: m = k + 256 (h + 4 i), inputs x[m + 4096 s]
    const float2* q = buf + pad_q(k + 256 * h);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int s = 0; s < 4; ++s) v[4 * i + s] = q[q_off(1024 * i + 4096 * s)];
  }
  buf_release_arrive(rel);  // the last read of the buffer in this transform
  FftTw<N, 16, true, 4096> lt;
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const float4 x = lp[T * hh + t];
    lt.tw[2 * hh].a[0] = make_float2(x.x, x.y);
    lt.tw[2 * hh + 1].a[0] = make_float2(x.z, x.w);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    lt.tw[i].a[1] = c_mul(lt.tw[i].a[0], lt.tw[i].a[0]);
    lt.tw[i].a[2] = c_mul(lt.tw[i].a[1], lt.tw[i].a[0]);
    float2 u[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) u[s] = v[4 * i + s];
    TwApply<4, 1, false>::run(u, lt.tw[i]);
    dft_r<4, true>(u);
#pragma unroll
    for (int s = 0; s < 4; ++s) v[4 * i + s] = u[s];
  }
}

// The class-local 2048-point inverse transform (ClassLocal<2048>): the
// NS = 16 pass's bases from TMEM columns ta .. ta + 8, the radix-8 NS = 256
// pass's bases (w, w^2, w^3 and w^4 of butterflies jp and jp + 128) from this
// thread's column of the shared-memory table.  One CTA barrier and two
// __syncwarp per transform; the buffer's reuse waits on 'rel'.
__device__ __forceinline__ void fft2048_cl_tmtw(float2 (&v)[16], int t, float2* buf, uint32_t ta_tw,
                                                BufRelease& rel, const float4* lp) {
  constexpr int N = 2048, T = N / 16;
  {
    FftTw<N, 16, true, 1> none;  // pass 1 (NS = 1) takes no twiddles
    pass_compute_tw<N, 16, 16, 1, true>(v, none);
  }
  buf_release_wait(rel);
  {
    float2* b = buf + pad_2k(16 * t);
#pragma unroll
    for (int u = 0; u < 16; ++u) b[off_2k(u)] = v[u];
  }
  float w[8];
  tm_ld8(ta_tw, w);
  __syncthreads();
  const int jp = ClassLocal<N>::perm(t);
  const float2* g = buf + pad_2k(jp);  // element jp + T r sits at g[off_2k(T r)]
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[off_2k(T * r)];
  {
    tm_wait_ld8(w);
    FftTw<N, 16, true, 16> tw;
    tw.tw[0] = tw_unpack(w);
    pass_compute_tw<N, 16, 16, 16, true>(v, tw);
  }
  __syncwarp();  // the class's eight lanes have read every slot of the class
  {
    // butterfly jp of the NS = 16 pass writes y[(jp / 16) 256 + (jp mod 16) + 16 u]
    float2* b = buf + pad_2k((jp >> 4) * 256 + (jp & 15));
#pragma unroll
    for (int u = 0; u < 16; ++u) b[off_2k(16 * u)] = v[u];
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = g[off_2k(T * r)];
  buf_release_arrive(rel);  // the last read of the buffer in this transform
  FftTw<N, 16, true, 256> lt;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float4 x0 = lp[T * (2 * q) + t], x1 = lp[T * (2 * q + 1) + t];
    lt.tw[q].a[0] = make_float2(x0.x, x0.y);
    lt.tw[q].a[1] = make_float2(x0.z, x0.w);
    lt.tw[q].a[2] = make_float2(x1.x, x1.y);
    lt.tw[q].b[0] = make_float2(x1.z, x1.w);
  }
  pass_compute_tw<N, 16, 8, 256, true>(v, lt);
}

// ---------------------------------------------------------------------------
// One CTA: PRNs p0 .. p0 + kk - 1 (kk <= K) of the tile rows u0 .. u0 + mm - 1
// (mm <= M; a row is a Doppler bin, or the bin bin_order names).  Each bin
// runs its blocks set by set (with half-bit sets the even blocks, then the
// odd ones); within a block the K PRNs share the Y that was loaded during the
// previous block.  The sums stay in registers with one PRN of 16 elements
// per thread (except in the occupancy form); otherwise they live in TMEM
// (with two PRNs of 16 per thread the block's sums are fetched before its
// transform, in the occupancy form after it, and updated after it).
// ---------------------------------------------------------------------------
template <int N, int E, bool HALF, int K, int M, bool O>
__device__ __forceinline__ void xcorr_tile_tm(const XcorrArgs& a, int cta, float2* sm) {
  using Sh = TmShape<N, E, O>;
  using X = typename Sh::X;
  using Cl = typename Sh::template Cols<K>;
  constexpr int T = Sh::T, S = HALF ? 2 : 1;
  constexpr bool CL = Sh::CL, RACC = Cl::acc_regs;
  float2* buf0 = sm;
  float2* buf1 = ((X::DB || CL) && !Sh::ONEBUF) ? sm + X::buf_bytes / sizeof(float2) : sm;
  __shared__ float s_val[32];
  __shared__ uint32_t s_idx[32];
  __shared__ uint32_t s_tmem;
  __shared__ unsigned s_last[K];
  const int j = threadIdx.x, warp = j >> 5;
  // thread j ends each transform holding |R|^2 of phases PhaseMap::at(jo, r)
  const int jo = CL ? ClassLocal<(CL ? N : 4096)>::perm(j) : j;
  const int PK = (a.P + K - 1) / K;
  const int p0 = (cta % PK) * K, kk = min(K, a.P - p0);
  const int u0 = (cta / PK) * M, mm = min(M, a.D - u0);
  FftTw<N, E, true> tw;
  // the first pass has no twiddles; later passes run butterfly jo
  if constexpr (CL) ClassLocal<(CL ? N : 4096)>::init_twiddles(tw, jo);
  else if constexpr (X::TWC) tw.init(jo);
  griddep_wait();  // the spectra and the cleared counters are complete and visible
  // Columns are taken only now: a CTA never holds TMEM while it waits for
  // another kernel, and between here and the release below it waits for
  // nothing, so an allocation can at worst wait for CTAs that run on.
  __shared__ uint64_t s_release;
  BufRelease rel{&s_release, a.counters + a.P, 0};
  if constexpr (Sh::ONEBUF) {
    if (j == 0) buf_release_init(&s_release, (unsigned)T);  // visible after the barrier below
  }
  if (warp == 0) tm_alloc<Cl::alloc>(&s_tmem);
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  // this warp's slot: lane quarter 32 (warp % 4), columns stride (warp / 4) ..
  const uint32_t tq = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * Cl::stride);
  const uint32_t tsum = tq + (uint32_t)(2 * E * K);  // sums of PRN i at tsum + E i (TMEM sums)
  // code spectra C_i[j + T r] of the CTA's PRNs, once
#pragma unroll
  for (int i = 0; i < K; ++i) {
    if (i < kk) {
      const float2* cp = a.cspec + (size_t)(p0 + i) * N + j;
#pragma unroll
      for (int h = 0; h < E / 16; ++h) {
        float c[32];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float2 w = __ldg(cp + T * (16 * h + q));
          c[2 * q] = w.x;
          c[2 * q + 1] = w.y;
        }
        tm_st32(tq + (uint32_t)(2 * E * i + 32 * h), c);
      }
    }
  }
  // with the twiddle bases in TMEM: the two twiddled passes' bases, after the PRNs' columns
  const uint32_t ttw = tq + (uint32_t)(K * Cl::per_prn);
  if constexpr (Cl::tw_tmem) {
    if constexpr (N == 2048) tw_to_tmem(tw.next.tw[0], tw.next.tw[0], ttw);  // (the NS = 16 bases only)
    else tw_to_tmem(tw.next.tw[0], tw.next.next.tw[0], ttw);
  }
  // and the lane-pair twiddles of N = 8192 into this thread's table column
  // (read back only by this thread)
  float4* lp = reinterpret_cast<float4*>(sm + X::buf_bytes / sizeof(float2));
  if constexpr (Cl::tw_tmem && N == 2048) {
    const auto& lt = tw.next.next;  // NS = 256, radix 8: w, w^2, w^3 and w^4 of two butterflies
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      lp[T * (2 * q) + j] = make_float4(lt.tw[q].a[0].x, lt.tw[q].a[0].y, lt.tw[q].a[1].x, lt.tw[q].a[1].y);
      lp[T * (2 * q + 1) + j] = make_float4(lt.tw[q].a[2].x, lt.tw[q].a[2].y, lt.tw[q].b[0].x, lt.tw[q].b[0].y);
    }
  } else if constexpr (Cl::tw_tmem && Sh::lp_vec > 0) {
    const auto& lt = tw.next.next.next;
#pragma unroll
    for (int h = 0; h < Sh::lp_vec; ++h)
      lp[T * h + j] = make_float4(lt.tw[2 * h].a[0].x, lt.tw[2 * h].a[0].y, lt.tw[2 * h + 1].a[0].x,
                                  lt.tw[2 * h + 1].a[0].y);
  }
  tm_wait_st();  // the first block reads them back
  auto bin_at = [&](int u) { return a.bin_order ? __ldg(a.bin_order + u) : u; };
  // bin d's spectrum: its own row, or its class's row read K bins further
  // (Y_{f + 1000 K}[k] = Y_f[k + K]: a whole kHz is one bin of a 1 ms FFT)
  auto row_at = [&](int d) { return a.Y + (size_t)(a.bin_cls ? __ldg(a.bin_cls + d) : d) * a.B * N; };
  auto shift_at = [&](int d) { return a.bin_shift ? __ldg(a.bin_shift + d) : 0; };
  int d = bin_at(u0);
  const float2* yd = row_at(d);
  int js = j + shift_at(d);
  float2 y[E];
  if constexpr (Cl::prefetch) tm_load_row<N, E>(y, yd, js);  // block 0 of set 0
  int phase = 0;
#pragma unroll 1
  for (int ui = 0; ui < mm; ++ui) {
    // the CTA's next bin: its first block follows this bin's last one
    int dn = d, jsn = js;
    const float2* ydn = nullptr;
    if constexpr (M > 1) {
      if (ui + 1 < mm) {
        dn = bin_at(u0 + ui + 1);
        ydn = row_at(dn);
        jsn = j + shift_at(dn);
      }
    }
#pragma unroll 1
    for (int set = 0; set < S; ++set) {
      const int nb = (a.B - set + S - 1) / S;  // blocks set, set + S, ...
      float racc[RACC ? E : 1];
      if constexpr (RACC) {
#pragma unroll
        for (int r = 0; r < E; ++r) racc[r] = 0.f;
      }
      const float2* yb = yd + (size_t)set * N;
#pragma unroll 1
      for (int t = 0; t < nb; ++t, yb += S * N) {
        // where the next block's spectrum comes from: this set's next block,
        // the first block of the next set, or the first of the next bin
        const float2* nrow = ydn;
        int njs = jsn;
        if constexpr (Cl::prefetch) {
          if (t + 1 < nb) {
            nrow = yb + S * N;
            njs = js;
          } else if (set + 1 < S && set + 1 < a.B) {
            nrow = yd + (size_t)(set + 1) * N;
            njs = js;
          }
        }
        if constexpr (K == 2 && E == 16) {
          if (kk == 2) {
            // both PRNs' transforms interleaved in each thread, one Y load
            tw.launder();
            float2 va[E], vb[E];
            tm_load_row<N, E>(va, yb, js);
            tm_product<E>(tq + (uint32_t)(2 * E), va, vb);
            tm_product<E>(tq, va, va);
            if constexpr (CL) fft_class_local2<N, true>(va, vb, j, buf0, buf1, tw);
            else fft_block_tw2<N, E, true>(va, vb, j, buf0, buf1, tw);
            float sa[16], sb[16];
            if (t > 0) {
              tm_wait_st();
              tm_ld16(tsum, sa);
              tm_ld16(tsum + (uint32_t)E, sb);
              tm_wait_ld16(sa);
              tm_wait_ld16(sb);
            } else {
#pragma unroll
              for (int r = 0; r < 16; ++r) sa[r] = sb[r] = 0.f;
            }
            add_power<16>(sa, va);
            add_power<16>(sb, vb);
            tm_st16(tsum, sa);
            tm_st16(tsum + (uint32_t)E, sb);
            continue;
          }
        }
        if constexpr (K == 1) {
          // one PRN: straight-line block
          if constexpr (X::TWC && !Cl::tw_tmem) tw.launder();
          float2 v[E];
          if constexpr (Cl::prefetch) {
            tm_product<E>(tq, y, v);
            if (nrow != nullptr) tm_load_row<N, E>(y, nrow, njs);  // under this transform
          } else {
            tm_load_row<N, E>(v, yb, js);
            tm_product<E>(tq, v, v);
          }
          if constexpr (Cl::tw_tmem) {
            if constexpr (N == 16384) fft16384_cl_tmtw(v, j, buf0, ttw, rel, lp);
            else if constexpr (N == 2048) fft2048_cl_tmtw(v, j, buf0, ttw, rel, lp);
            else fft_cl_tmtw<N, Sh::ONEBUF>(v, j, phase ? buf1 : buf0, ttw, rel, lp);
            phase ^= 1;
          } else if constexpr (CL) {
            fft_class_local<N, true>(v, j, phase ? buf1 : buf0, tw);
            phase ^= 1;
          } else if constexpr (X::TWC) {
            fft_block_tw<N, E, true, X::DB>(v, j, buf0, buf1, phase, tw);
          } else {
            fft_block<N, E, true, X::DB>(v, j, buf0, buf1, phase);
          }
          if constexpr (RACC) {
            add_power<E>(racc, v);
          } else if constexpr (E == 16) {
            // the sums are fetched only now: 16 registers fewer live through
            // the transform (the occupancy form runs at 64 registers)
            float s16[16];
            if (t > 0) {
              tm_wait_st();
              tm_ld16(tsum, s16);
              tm_wait_ld16(s16);
            } else {
#pragma unroll
              for (int r = 0; r < 16; ++r) s16[r] = 0.f;
            }
            add_power<16>(s16, v);
            tm_st16(tsum, s16);
          } else {
            tm_accumulate32(tsum, v, t == 0);
          }
          continue;
        }
        if constexpr (K > 1) {  // (one PRN per CTA always takes the block above)
#pragma unroll 1
        for (int i = 0; i < kk; ++i) {
          if constexpr (X::TWC) tw.launder();
          float2 v[E];
          if constexpr (Cl::prefetch) {
            tm_product<E>(tq + (uint32_t)(2 * E * i), y, v);
            // the K products are formed: Y of the next block loads now, under this transform
            if (i == kk - 1 && nrow != nullptr) tm_load_row<N, E>(y, nrow, njs);
          } else {
            tm_load_row<N, E>(v, yb, js);
            tm_product<E>(tq + (uint32_t)(2 * E * i), v, v);
          }
          // TMEM sums of 16 per thread: fetched now, used after the transform
          float s16[RACC || E != 16 ? 1 : 16];
          if constexpr (!RACC && E == 16) {
            if (t > 0) {
              tm_wait_st();
              tm_ld16(tsum + (uint32_t)(E * i), s16);
            } else {
#pragma unroll
              for (int r = 0; r < 16; ++r) s16[r] = 0.f;
            }
          }
          if constexpr (CL) {
            // one buffer per transform, alternating: the next transform's
            // first-pass stores go to the other buffer
            fft_class_local<N, true>(v, j, phase ? buf1 : buf0, tw);
            phase ^= 1;
          } else if constexpr (X::TWC) {
            fft_block_tw<N, E, true, X::DB>(v, j, buf0, buf1, phase, tw);
          } else {
            fft_block<N, E, true, X::DB>(v, j, buf0, buf1, phase);
          }
          if constexpr (RACC) {
            add_power<E>(racc, v);
          } else if constexpr (E == 16) {
            tm_wait_ld16(s16);
            add_power<16>(s16, v);
            tm_st16(tsum + (uint32_t)(E * i), s16);
          } else {
            tm_accumulate32(tsum + (uint32_t)(E * i), v, t == 0);
          }
        }
        }
      }
      // R = IFFT / N, so |R|^2 = |.|^2 / N^2 (an exact power of two)
      constexpr float sc = 1.f / ((float)N * (float)N);
#pragma unroll 1
      for (int i = 0; i < kk; ++i) {
        const int p = p0 + i;
        float acc[E];
        if constexpr (RACC) {
#pragma unroll
          for (int r = 0; r < E; ++r) acc[r] = racc[r];
        } else if (nb > 0) {
          tm_read_sums<E>(tsum + (uint32_t)(E * i), acc);
        } else {
#pragma unroll
          for (int r = 0; r < E; ++r) acc[r] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < E; ++r) acc[r] *= sc;
        if (a.surface != nullptr) {
          float* row = a.surface + (((size_t)set * a.P + p) * a.D + d) * (size_t)N;
#pragma unroll
          for (int r = 0; r < E; ++r) row[PhaseMap<N, E, CL>::at(jo, r)] = acc[r];
        }
        row_stats<N, E, CL>(acc, jo, a.excl, s_val, s_idx, a.rows + ((size_t)set * a.P + p) * a.D + d);
      }
    }
    d = dn;
    yd = ydn;
    js = jsn;
  }
  // Every TMEM access of the CTA has completed (each thread waited for its
  // loads, and for its stores before its last loads).  The barrier also
  // orders every row and surface write of the CTA before thread 0's fence and
  // counts (release), as in the register form.
  tm_fence_before();
  __syncthreads();
  if (warp == 0) {
    tm_fence_after();
    tm_dealloc<Cl::alloc>(s_tmem);
  }
  // Each of the CTA's PRNs gains mm rows; the CTA that completes a PRN's D
  // rows runs its detection, after a fence (acquire).
  if (a.second_whole) {
    // the whole-surface second peak scans D N cells per set: all threads
    if (j == 0) {
      __threadfence();
      for (int i = 0; i < kk; ++i)
        s_last[i] = (atomicAdd(a.counters + p0 + i, (unsigned)mm) + (unsigned)mm == (unsigned)a.D) ? 1u : 0u;
    }
    __syncthreads();
    for (int i = 0; i < kk; ++i) {
      if (s_last[i]) {
        __threadfence();
        finalize_prn<N, T>(a, p0 + i, S, s_val, s_idx);
      }
    }
    return;
  }
  // otherwise warp 0 alone counts and detects; the other warps leave now
  if (j >= 32) return;
  unsigned last = 0;
  if (j == 0) {
    __threadfence();
    for (int i = 0; i < kk; ++i)
      if (atomicAdd(a.counters + p0 + i, (unsigned)mm) + (unsigned)mm == (unsigned)a.D) last |= 1u << i;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    for (int i = 0; i < kk; ++i)
      if ((last >> i) & 1u) finalize_prn<N, 32>(a, p0 + i, S, s_val, s_idx);
  }
}

template <int N, int E, bool HALF, int K, int M, bool O>
__global__ void __launch_bounds__(TmShape<N, E, O>::T, TmShape<N, E, O>::MINB) k_xcorr_tm(const XcorrArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  xcorr_tile_tm<N, E, HALF, K, M, O>(a, blockIdx.x, sm);
}

template <int N, int E, bool HALF, int K, int M, bool O>
__global__ void __launch_bounds__(TmShape<N, E, O>::T, TmShape<N, E, O>::MINB)
    k_xcorr_tm_batch(const BatchReq* __restrict__ reqs, const uint32_t* __restrict__ base, int n) {
  extern __shared__ __align__(16) float2 sm[];
  const int r = find_request(base, n);
  xcorr_tile_tm<N, E, HALF, K, M, O>(reqs[r].xc, (int)(blockIdx.x - __ldg(base + r)), sm);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
cudaError_t set_buf_wait_limit(unsigned iters, cudaStream_t stream) {
  cudaError_t e = cudaMemcpyToSymbolAsync(g_buf_wait_limit, &iters, sizeof(unsigned), 0, cudaMemcpyHostToDevice,
                                          stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(stream);
}

int xcorr_tm_prns(int code) { return (code & (int)GNSS_TUNE_TMEM) ? ((code >> 12) & 3) + 1 : 1; }
int xcorr_tm_bins(int code) { return (code & (int)GNSS_TUNE_TMEM) ? ((code >> 14) & 3) + 1 : 1; }

uint32_t xcorr_ctas(int code, int P, int D) {
  const int K = xcorr_tm_prns(code), M = xcorr_tm_bins(code);
  return (uint32_t)(((P + K - 1) / K) * ((D + M - 1) / M));
}

// A shape is offered only if the CTAs of its kernel that fit on one SM
// together (registers, shared memory, threads) take at most the SM's 512
// TMEM columns, so its allocations do not wait for one another.  (Where
// CTAs of different correlate launches share an SM, an allocation can at
// most wait for a CTA that is running to its end: none waits for anything
// while it holds columns.)
template <typename Kern>
static bool tm_cols_fit(Kern k, int T, size_t smem, int cols) {
  int occ = 0;
  if (set_smem(k, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, T, smem) != cudaSuccess) {
    cudaGetLastError();  // a refused shape leaves no error for a later launch check to pick up
    return false;
  }
  return occ >= 1 && occ * cols <= 512;
}

template <int N, int E, int K, int M, bool O>
static bool tm_fits() {
  using Sh = TmShape<N, E, O>;
  constexpr int cols = Sh::template Cols<K>::alloc;
  return tm_cols_fit(k_xcorr_tm<N, E, false, K, M, O>, Sh::T, Sh::smem, cols) &&
         tm_cols_fit(k_xcorr_tm<N, E, true, K, M, O>, Sh::T, Sh::smem, cols) &&
         tm_cols_fit(k_xcorr_tm_batch<N, E, false, K, M, O>, Sh::T, Sh::smem, cols) &&
         tm_cols_fit(k_xcorr_tm_batch<N, E, true, K, M, O>, Sh::T, Sh::smem, cols);
}

template <int N, int E, int K, int M, bool O>
static cudaError_t tm_launch(const AcqShape& s, const XcorrArgs& a, cudaStream_t stream) {
  using Sh = TmShape<N, E, O>;
  const unsigned grid = (unsigned)(((s.P + K - 1) / K) * ((s.D + M - 1) / M));
  cudaError_t e;
  if (s.sets == 2) {
    if ((e = set_smem(k_xcorr_tm<N, E, true, K, M, O>, Sh::smem)) != cudaSuccess) return e;
    return launch_dependent(k_xcorr_tm<N, E, true, K, M, O>, grid, Sh::T, Sh::smem, stream, a);
  }
  if ((e = set_smem(k_xcorr_tm<N, E, false, K, M, O>, Sh::smem)) != cudaSuccess) return e;
  return launch_dependent(k_xcorr_tm<N, E, false, K, M, O>, grid, Sh::T, Sh::smem, stream, a);
}

template <int N, int E, int K, int M, bool O>
static cudaError_t tm_launch_batch(const BatchGroup& g, cudaStream_t stream) {
  using Sh = TmShape<N, E, O>;
  cudaError_t e;
  if (g.sets == 2) {
    if ((e = set_smem(k_xcorr_tm_batch<N, E, true, K, M, O>, Sh::smem)) != cudaSuccess) return e;
    return launch_dependent(k_xcorr_tm_batch<N, E, true, K, M, O>, g.xc_ctas, Sh::T, Sh::smem, stream, g.reqs,
                            g.xc_base, g.n);
  }
  if ((e = set_smem(k_xcorr_tm_batch<N, E, false, K, M, O>, Sh::smem)) != cudaSuccess) return e;
  return launch_dependent(k_xcorr_tm_batch<N, E, false, K, M, O>, g.xc_ctas, Sh::T, Sh::smem, stream, g.reqs,
                          g.xc_base, g.n);
}

// Every (N, E, K, M, O) the variant is built for, as CALL(N, E, K, M, O).
#define GNSS_TM_SHAPES(CALL)                                                                              \
  CALL(2048, 16, 1, 1, false) CALL(2048, 16, 2, 1, false) CALL(2048, 16, 1, 2, false)                      \
  CALL(2048, 16, 2, 2, false) CALL(2048, 16, 1, 1, true)                                                   \
  CALL(4096, 16, 1, 1, false) CALL(4096, 16, 2, 1, false) CALL(4096, 16, 1, 2, false)                      \
  CALL(4096, 16, 2, 2, false) CALL(4096, 16, 1, 1, true)                                                   \
  CALL(8192, 16, 1, 1, false) CALL(8192, 16, 2, 1, false) CALL(8192, 16, 1, 2, false)                      \
  CALL(8192, 16, 2, 2, false) CALL(8192, 16, 1, 1, true)                                                  \
  CALL(16384, 32, 1, 1, false) CALL(16384, 32, 1, 2, false) CALL(16384, 16, 1, 1, true)

static bool tm_shape(int N, int code, int* E, int* K, int* M, bool* O) {
  if (!(code & (int)GNSS_TUNE_TMEM)) return false;
  const int e = code & 0xff, k = xcorr_tm_prns(code), m = xcorr_tm_bins(code);
  const bool o = (code & (int)GNSS_TUNE_OCC) != 0;
  if ((code & ~(0xff | (int)GNSS_TUNE_TMEM | (int)GNSS_TUNE_OCC | (3 << 12) | (3 << 14))) != 0) return false;
  bool known = false;
#define GNSS_TM_MATCH(NN, EE, KK, MM, OO) known = known || (N == NN && e == EE && k == KK && m == MM && o == OO);
  GNSS_TM_SHAPES(GNSS_TM_MATCH)
#undef GNSS_TM_MATCH
  if (!known) return false;
  *E = e;
  *K = k;
  *M = m;
  *O = o;
  return true;
}

bool xcorr_tm_valid(int N, int code) {
  int E, K, M;
  bool O;
  if (!tm_shape(N, code, &E, &K, &M, &O)) return false;
#define GNSS_TM_FITS(NN, EE, KK, MM, OO) \
  if (N == NN && E == EE && K == KK && M == MM && O == OO) return tm_fits<NN, EE, KK, MM, OO>();
  GNSS_TM_SHAPES(GNSS_TM_FITS)
#undef GNSS_TM_FITS
  return false;
}

cudaError_t launch_xcorr_tm(int code, const AcqShape& s, const XcorrArgs& a, cudaStream_t stream) {
  int E, K, M;
  bool O;
  if (!tm_shape(s.N, code, &E, &K, &M, &O)) return cudaErrorInvalidValue;
#define GNSS_TM_LAUNCH(NN, EE, KK, MM, OO) \
  if (s.N == NN && E == EE && K == KK && M == MM && O == OO) return tm_launch<NN, EE, KK, MM, OO>(s, a, stream);
  GNSS_TM_SHAPES(GNSS_TM_LAUNCH)
#undef GNSS_TM_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t launch_xcorr_tm_batch(int code, const BatchGroup& g, cudaStream_t stream) {
  int E, K, M;
  bool O;
  if (!tm_shape(g.N, code, &E, &K, &M, &O)) return cudaErrorInvalidValue;
#define GNSS_TM_LAUNCH(NN, EE, KK, MM, OO) \
  if (g.N == NN && E == EE && K == KK && M == MM && O == OO) return tm_launch_batch<NN, EE, KK, MM, OO>(g, stream);
  GNSS_TM_SHAPES(GNSS_TM_LAUNCH)
#undef GNSS_TM_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace gnss

/*
 * gnss.h -- C ABI of a B300 (sm_103a) GPS L1 C/A acquisition library.
 *
 * The library implements the acquisition channel of "Accelerating a
 * Cloud-Based Software GNSS Receiver" (Karimi, Pamir, Afzal), Section 3,
 * Fig. 2, as an FFT parallel code-phase search over a whole client
 * recording: code NCO (Gold code + replica), carrier NCO and first mixing
 * (wipe-off), FFT of the mixed signal and of the replica, frequency-domain
 * second mixing, IFFT, |.|^2 summed non-coherently over blocks, and signal
 * detection (peak against second peak).  The paper runs each ~1 ms FFT as a
 * separate GPU call from many CPU threads (Section 5, Listing 3a); here a
 * whole recording, all PRNs and all Doppler bins go to the device in one
 * batched call (the batch mode of Listing 3b).
 *
 * Conventions shared by every entry point
 *  - Status: every function returns a gnss_status; on failure
 *    gnss_last_error() returns a message for the calling thread.  No C++
 *    exception crosses this boundary.
 *  - Ownership: the caller owns every buffer it passes.  Plans own their
 *    device code tables; the library never hands out memory the caller must
 *    free.  Scratch memory comes from a library-owned stream-ordered pool
 *    (cudaMallocAsync) and is released in stream order.
 *  - Streams: 'stream' is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Device-side work is enqueued on it; see each function
 *    for when results are valid on the host.
 *  - Devices: a plan belongs to the device that was current when it was
 *    created; calls must be made with that device current.
 *  - Recordings: complex baseband samples in one of two formats (below).
 *    A device pointer to samples must be 16-byte aligned.
 *  - Sample rate: fs is a multiple of 1000 Hz and N = fs / 1000 (the
 *    samples of one 1 ms code period, the FFT size) is a power of two in
 *    [256, 16384].
 */
#ifndef GNSS_H
#define GNSS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GNSS_API __attribute__((visibility("default")))
#else
#define GNSS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GNSS_OK = 0,
  GNSS_EINVAL = 1,     /* bad argument, descriptor or length              */
  GNSS_ENOMEM = 2,     /* host or device allocation failed                */
  GNSS_ECUDA = 3,      /* a CUDA call failed (message in gnss_last_error) */
  GNSS_EBUSY = 4,      /* over the server's memory budget / queue full    */
  GNSS_EAGAIN = 5,     /* result not ready yet                            */
  GNSS_ETIMEOUT = 6,   /* a bounded wait gave up                          */
  GNSS_ECANCELLED = 7  /* request cancelled                               */
} gnss_status;

/* Recording formats.
 * GNSS_FMT_I8_IQ:   int8 I, Q interleaved, 2 bytes per complex sample.
 * GNSS_FMT_2BIT_IQ: 2-bit I/Q, two complex samples per byte,
 *                   byte = I0 | Q0 << 2 | I1 << 4 | Q1 << 6, code c is the
 *                   level 2c - 3 (-3, -1, +1, +3). */
typedef enum { GNSS_FMT_I8_IQ = 0, GNSS_FMT_2BIT_IQ = 1 } gnss_format;

/* Plan flags. */
#define GNSS_HALF_BIT 0x1u     /* two non-coherent sets: even and odd blocks */
#define GNSS_SECOND_WHOLE 0x2u /* second peak over the whole surface instead
                                  of the peak's Doppler row (needs a surface) */
/* Code-Doppler compensation of the non-coherent sum.  The code NCO of the
 * receiver (Section 3, Fig. 2) runs at the nominal chip rate, while a signal
 * at Doppler f carries its code f / 1540 chips per second faster (1540
 * carrier cycles per chip at L1), so over a long non-coherent sum its
 * correlation peak walks by f t fs / f_L1 samples (f_L1 = 1540 x 1.023 MHz).
 * With this flag, block b of bin f enters the sum circularly shifted by
 *   sigma_b = floor(f b L / f_L1 + 1/2)  samples (exact integer arithmetic),
 *   S[tau] += |R_b[(tau - sigma_b) mod N]|^2,
 * so the peaks of all blocks line up on the code phase of block 0.  The paper
 * does not treat code Doppler; without the flag no compensation is made. */
#define GNSS_CODE_DOPPLER 0x4u

/* Acquisition plan descriptor (Section 3, Fig. 2: sample rate and coherent
 * length set the replica loop length fs * T; Doppler grid and PRN set define
 * the search).
 *  fs_hz        sample rate, multiple of 1000, fs/1000 a power of two 256..16384
 *  coh_ms       coherent milliseconds per block T_coh >= 1 (folded before the FFT)
 *  noncoh       blocks to sum non-coherently; 0 = every whole block recorded
 *  dopp_min_hz, dopp_step_hz, n_dopp
 *               Doppler bins f_d = dopp_min_hz + d * dopp_step_hz, d < n_dopp
 *               (integer Hz; n_dopp >= 1, step >= 1 when n_dopp > 1)
 *  prn_mask     bit p-1 set = search PRN p (1..32); at least one bit
 *  threshold    detected = peak / second >= threshold (e.g. 2.0)
 *  flags        GNSS_HALF_BIT | GNSS_SECOND_WHOLE | GNSS_CODE_DOPPLER
 *  format       gnss_format of the recordings this plan will see */
typedef struct {
  uint32_t fs_hz;
  uint32_t coh_ms;
  uint32_t noncoh;
  int32_t dopp_min_hz;
  uint32_t dopp_step_hz;
  uint32_t n_dopp;
  uint64_t prn_mask;
  float threshold;
  uint32_t flags;
  uint32_t format;
  uint32_t reserved;
} gnss_plan_desc;

/* Detection record, one per searched PRN in ascending PRN order.
 *  detected   peak / second >= threshold
 *  set        non-coherent set the record comes from (0, or 1 = odd blocks
 *             with GNSS_HALF_BIT; the set with the larger ratio, ties to 0)
 *  dopp_bin   index d of the peak, dopp_hz its frequency
 *  code_phase peak code phase in samples [0, N) (replica delay; with
 *             GNSS_CODE_DOPPLER the delay of block 0)
 *  peak, second, ratio: surface values (sample units squared) and their ratio
 *  flags      GNSS_DET_* bits of the call that produced the record */
#define GNSS_DET_STAGE_TIMEOUT 0x01u /* a bounded wait of the staged correlate variant gave up in this call: its
                                        CTA read the spectra from global memory instead and the results are
                                        complete, but a copy may have outlived its CTA (see gnss_autotune) */
#define GNSS_DET_WAIT_TIMEOUT 0x02u  /* a bounded wait between the warps of a correlate CTA (the shared-memory
                                        exchange buffer's release) gave up in this call: the CTA went on
                                        without it and the call's records and surfaces are not valid */
#define GNSS_DET_TIMEOUTS (GNSS_DET_STAGE_TIMEOUT | GNSS_DET_WAIT_TIMEOUT)
typedef struct {
  uint8_t prn;
  uint8_t detected;
  uint8_t set;
  uint8_t flags;
  int32_t dopp_bin;
  int32_t dopp_hz;
  uint32_t code_phase;
  float peak;
  float second;
  float ratio;
} gnss_detection;

/* Sizes a plan resolved from its descriptor. */
typedef struct {
  uint32_t N;          /* FFT size = fs / 1000                  */
  uint32_t n_prn;      /* PRNs searched                         */
  uint32_t n_dopp;     /* Doppler bins                          */
  uint32_t n_sets;     /* 1, or 2 with GNSS_HALF_BIT            */
  uint32_t excl;       /* second-peak exclusion half-width, ceil(N/1023) samples */
  uint32_t block_len;  /* L = coh_ms * N samples per block      */
  uint32_t xcorr_variant; /* correlate-kernel variant code used for N on the
                             current device now (see gnss_autotune)   */
} gnss_plan_info;

typedef struct gnss_plan gnss_plan;

/* Create a plan on the current device: validates the descriptor, generates
 * the Gold codes of the searched PRNs on the device (G1 = 1 + x^3 + x^10,
 * G2 = 1 + x^2 + x^3 + x^6 + x^8 + x^9 + x^10, both seeded all ones, two-tap
 * G2 phase selector per PRN), samples each replica at fs
 * (c_s[m] = c[floor(m * 1023 / N)]) and keeps its FFT resident (the code
 * replica FFT of Fig. 2, computed once per plan instead of once per call).
 * Synchronous.  On success *out owns device memory until gnss_plan_destroy.
 * Errors: GNSS_EINVAL (descriptor), GNSS_ENOMEM, GNSS_ECUDA. */
GNSS_API gnss_status gnss_plan_create(const gnss_plan_desc* desc, gnss_plan** out);

/* Release a plan (NULL is accepted).  The caller must make sure no work that
 * uses the plan is still in flight. */
GNSS_API gnss_status gnss_plan_destroy(gnss_plan* plan);

/* Resolved sizes of a plan into *out (host). */
GNSS_API gnss_status gnss_plan_get_info(const gnss_plan* plan, gnss_plan_info* out);

/* Copy the plan's Gold codes to host memory: int8 [n_prn][1023] of +-1 chips
 * (chip = 1 - 2 * bit), PRNs ascending.  cap = bytes available at out.
 * Synchronous.  Errors: GNSS_EINVAL when cap < n_prn * 1023. */
GNSS_API gnss_status gnss_plan_codes(const gnss_plan* plan, int8_t* out, size_t cap);

/* Copy the plan's code spectra C_p[k] = FFT_N(c_s,p) (forward, unscaled) to
 * device memory: float [n_prn][N][2] (re, im).  cap = bytes available.
 * Enqueued on 'stream'. */
GNSS_API gnss_status gnss_plan_code_spectra(const gnss_plan* plan, float* out_dev, size_t cap, void* stream);

/* Bytes of the sample buffer that gnss_acquire reads for n_samples samples
 * (only the B * L samples of whole blocks are read). */
GNSS_API size_t gnss_recording_bytes(uint32_t format, size_t n_samples);

/* Acquire every planned PRN over one recording (Section 3, Fig. 2, batched
 * over the whole recording):
 *   y_{f,b}[m] = sum_{i < T_coh} x[bL + iN + m] exp(-j 2 pi ((f (bL+iN+m)) mod fs) / fs)
 *   R_{p,f,b}  = IFFT_N( FFT_N(y_{f,b}) * conj(C_p) ),   (inverse scaled 1/N)
 *   S^{(s)}_{p,f}[tau] = sum over blocks b of set s of |R_{p,f,b}[tau]|^2,
 * then per PRN the peak (largest cell, ties to the smallest Doppler-major
 * index), the second peak (largest cell of the peak's Doppler row whose
 * circular distance from the peak phase exceeds ceil(N/1023) samples) and
 * their ratio.  B = floor(n_samples / L) blocks (capped by noncoh); trailing
 * samples are ignored.
 *  samples            recording in the plan's format; host memory, or device
 *                     memory (16-byte aligned) when samples_on_device != 0
 *  n_samples          complex samples in the recording (>= L)
 *  out                host array of n_prn records (PRN ascending)
 *  surface_dev        NULL, or device float [n_sets][n_prn][n_dopp][N] that
 *                     receives the surfaces S
 *  stream             work is enqueued on it; 'out' is valid once the stream
 *                     has synchronised (a NULL stream is synchronised before
 *                     the call returns)
 * Errors: GNSS_EINVAL (n_samples < L, misaligned device pointer, NULL
 * arguments), GNSS_ENOMEM, GNSS_ECUDA; with a NULL stream also
 * GNSS_ETIMEOUT when a bounded wait inside the correlate kernel gave up
 * during this call (the records carry GNSS_DET_STAGE_TIMEOUT or
 * GNSS_DET_WAIT_TIMEOUT; every entry point reports such a wait through the
 * flags of its records, and the server fails the request's ticket with
 * GNSS_ETIMEOUT, keeping its records). */
GNSS_API gnss_status gnss_acquire(gnss_plan* plan, const void* samples, size_t n_samples, int samples_on_device,
                         gnss_detection* out, float* surface_dev, void* stream);

/* Device-resident form of gnss_acquire: samples_dev and out_dev are device
 * pointers; nothing is copied to or from the host and the call never
 * synchronises.  Same arithmetic and errors. */
GNSS_API gnss_status gnss_acquire_device(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                gnss_detection* out_dev, float* surface_dev, void* stream);

/* gnss_acquire_device with stage timing (a tracing aid: the paper profiles
 * its GPU path as a timeline of short bursts, Section 5, Fig. 12).  events
 * holds four caller-owned CUDA events (cudaEvent_t passed as void*, created
 * with timing enabled; a NULL entry is skipped) that the call records on
 * 'stream': [0] before the unpack/fold launch, [1] before the carrier +
 * forward FFT launch, [2] before the correlate launch, [3] after it, so
 * cudaEventElapsedTime of (2, 3) is the device time of the correlate stage
 * of this very acquisition.  Same arithmetic, outputs and errors as
 * gnss_acquire_device; GNSS_EINVAL if events is NULL. */
GNSS_API gnss_status gnss_acquire_device_traced(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                       gnss_detection* out_dev, float* surface_dev, void* stream,
                                       void* const* events);

/* One request of a batched acquisition. */
typedef struct {
  gnss_plan* plan;          /* plan of this request (fs, coherent length, Doppler grid, PRNs, format, flags) */
  const void* samples_dev;  /* device recording in the plan's format, 16-byte aligned */
  size_t n_samples;         /* complex samples (>= the plan's block length) */
  gnss_detection* out_dev;  /* device, n_prn records of this plan */
  float* surface_dev;       /* NULL or device [n_sets][n_prn][n_dopp][N] */
} gnss_request;

/* Acquire many recordings of uneven length, sample rate, Doppler grid and
 * coherent length with one launch triple per group of requests that share
 * FFT size, format and half-bit setting -- the batch mode of Section 5,
 * Listing 3b, over whole requests.  Within a group the requests run longest
 * first; groups are split into waves whose scratch (folded blocks, spectra,
 * row statistics) stays within scratch_budget bytes (0 = 16 GiB; a request
 * larger than the budget runs in a wave of its own).  Every request gets the
 * same records and surfaces as gnss_acquire_device alone.  Asynchronous on
 * 'stream'; device outputs are valid once it has synchronised.
 * Errors: GNSS_EINVAL (any invalid request; nothing is launched),
 * GNSS_ENOMEM, GNSS_ECUDA. */
GNSS_API gnss_status gnss_acquire_batch(const gnss_request* reqs, size_t n_req, size_t scratch_budget, void* stream);

/* The batch above captured once into a CUDA graph and replayed with one
 * launch: the batch mode of Section 5 (one batched GPU call in place of many
 * small ones, Listing 3b) for a service that refills fixed recording slots.
 * gnss_batch_graph_create validates the requests exactly as
 * gnss_acquire_batch does, allocates the graph's own scratch (one region of
 * the largest wave's size, reused by the waves in order, plus the launch
 * tables), writes the launch tables and captures every wave's launches;
 * it is synchronous.  The requests' plans, sample, output and surface
 * pointers are baked in: they must stay valid, and unchanged in size, while
 * the graph lives; their contents may change between launches (a new
 * recording in the same buffer gives that recording's results).
 * gnss_batch_graph_launch enqueues one replay on 'stream' (asynchronous;
 * outputs are valid once the stream has synchronised); replays on one stream
 * run in order, replays that overlap on the GPU race on the graph's scratch.
 * Errors: GNSS_EINVAL (NULL or empty, any invalid request, a graph of
 * another device), GNSS_ENOMEM, GNSS_ECUDA. */
typedef struct gnss_batch_graph gnss_batch_graph;
GNSS_API gnss_status gnss_batch_graph_create(const gnss_request* reqs, size_t n_req, size_t scratch_budget,
                                             gnss_batch_graph** out);
GNSS_API gnss_status gnss_batch_graph_launch(gnss_batch_graph* graph, void* stream);
GNSS_API gnss_status gnss_batch_graph_destroy(gnss_batch_graph* graph);

/* Second-stage fine Doppler search around coarse detections.  For each of
 * the n_det host records in det (typically the detected ones of a
 * gnss_acquire on this plan and recording), the acquisition of Section 3,
 * Fig. 2 is run again for that PRN alone on a grid zoom times finer,
 * spanning +-span coarse steps around the record's Doppler:
 *   f_k = det.dopp_hz + (k - span * zoom) * dopp_step_hz / zoom,
 *   k < 2 * span * zoom + 1,
 * with the plan's sample rate, coherent length, blocks, format, flags and
 * threshold, in one batched launch over all detections (the code spectra are
 * the plan's own).  out_dev[i] (device) receives the record of detection i
 * on its fine grid (dopp_bin indexes that grid); surface_dev, when not NULL,
 * receives detection i's surface [n_sets][1][2 span zoom + 1][N] at offset
 * i * n_sets * (2 span zoom + 1) * N floats.  Each record equals what
 * gnss_acquire_device gives for a plan with that fine grid and that PRN.
 * Asynchronous on 'stream'.  Errors: GNSS_EINVAL (NULL arguments, zoom not
 * in [2, 1000] or not dividing dopp_step_hz, span not in [1, 100], a PRN not
 * in the plan, more than 4096 detections, any invalid request),
 * GNSS_ENOMEM, GNSS_ECUDA. */
GNSS_API gnss_status gnss_acquire_zoom(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                       const gnss_detection* det, size_t n_det, uint32_t zoom, uint32_t span,
                                       gnss_detection* out_dev, float* surface_dev, void* stream);

/* Acquisition that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at
 * request time -- services that must keep a fixed device footprint after
 * start-up, or processes where another allocator (a framework's caching
 * allocator, a reserved arena) owns the device memory, so that cudaMalloc or
 * cudaMallocAsync is forbidden or may fail.  It computes exactly what
 * gnss_acquire_device computes, with the same kernels, but takes its scratch
 * (folded blocks, blocks * N * 8 bytes of spectra per class of bins a whole
 * kHz apart -- per bin with GNSS_CODE_DOPPLER -- and the per-row statistics)
 * from one fixed 32 MiB device array inside the library, which every GPU
 * that loads the library holds until the process exits.
 *  - Inputs and outputs are the caller's, as in gnss_acquire_device:
 *    samples_dev (16-byte aligned), out_dev (n_prn records), surface_dev
 *    (NULL or [n_sets][n_prn][n_dopp][N]).  Calls no cudaMalloc, cudaFree or
 *    other allocating routine.
 *  - A request whose scratch exceeds 32 MiB is rejected with GNSS_EINVAL and
 *    a message giving the bytes it needs; nothing is launched.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    device's primary context: like plans, it does not survive
 *    cudaDeviceReset, after which this entry point must not be called.
 *  - All calls on a device share the one array and it keeps the last call's
 *    contents (every value a call reads is written by that call first).
 *    Calls whose work overlaps on the GPU (other streams, or other threads)
 *    race on it: serialise them, e.g. on one stream. */
GNSS_API gnss_status gnss_acquire_noalloc(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                          gnss_detection* out_dev, float* surface_dev, void* stream);

/* Stage entry points (one launch each) for stage-level checks and for the
 * one-stage-per-launch comparison.
 * gnss_stage_wipe_fft: carrier wipe-off, coherent fold and forward FFT of
 *   every (Doppler, block): spectra_dev = float [n_dopp][n_blocks][N][2],
 *   Y_{f,b} = FFT_N(y_{f,b}).  n_blocks <= floor(n_samples / L).  With
 *   GNSS_CODE_DOPPLER, y_{f,b} is the block rotated by sigma_b samples
 *   (y'[n] = y[(n - sigma_b) mod N]), which rotates its correlation alike.
 * gnss_stage_correlate: conj-multiply with every code spectrum, IFFT, |.|^2
 *   and the non-coherent sums over n_blocks blocks of spectra_dev; writes
 *   surface_dev (may be NULL) and the per-PRN detections (device). */
GNSS_API gnss_status gnss_stage_wipe_fft(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                uint32_t n_blocks, float* spectra_dev, void* stream);
GNSS_API gnss_status gnss_stage_correlate(gnss_plan* plan, const float* spectra_dev, uint32_t n_blocks,
                                 float* surface_dev, gnss_detection* out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Fine acquisition.  The paper hands the coarse Doppler and code phase of an
 * acquisition channel to tracking for fine tuning (Section 3, Fig. 1); here
 * the fine tuning is gradient ascent on the coherent power of a window of
 * L = coh_ms * N samples from the start of the recording:
 *   z(f, tau) = sum_{n<L} x[n] exp(-j 2 pi f n / fs) ctilde(n * 1023 / N - tau - 1/2)
 *   ctilde(u) = (1 - a) c[k mod 1023] + a c[(k+1) mod 1023],  k = floor(u), a = u - k
 *   P(f, tau) = |z|^2     (f in Hz, tau in chips; chip k's value sits at its
 *                          centre, so nodes are interpolated between centres)
 * with the analytic gradient
 *   dP/df   = 2 Re(conj(z) sum x e^{-j theta_n} (-j 2 pi n / fs) ctilde)
 *   dP/dtau = 2 Re(conj(z) sum x e^{-j theta_n} (-(c[k+1] - c[k])))
 * (the slope of the replica segment each sample lies on).  Sums in FP32.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint8_t prn;         /* PRN 1..32, must be in the plan's PRN set */
  uint8_t reserved[7];
  double f_hz;         /* start Doppler (Hz)                     */
  double tau_chips;    /* start code delay (chips)               */
} gnss_candidate;

typedef struct {
  double f_hz;         /* refined Doppler                         */
  double tau_chips;    /* refined code delay                      */
  float power;         /* P at the refined point                  */
  uint32_t iters;      /* accepted steps                          */
  int32_t status;      /* 0 converged (Newton step < 1e-3 Hz, tau step < 1e-5 chip), 1 stuck, 2 max_iter */
  uint16_t n_eval;     /* evaluations of P alone (pre-search, tau trials), saturating at 65535 */
  uint16_t n_eval_grad; /* evaluations of P with its gradient (f trials, after accepted tau steps) */
} gnss_refined;

/* P and its gradient for n (PRN, f, tau) points, one CTA per point.
 *  samples_dev  device recording in the plan's format (16-byte aligned),
 *               n_samples >= coh_ms * N
 *  prn_dev      int32 [n]; f_dev, tau_dev double [n] (device)
 *  P_dev        float [n] (device); dPdf_dev, dPdtau_dev float [n] or NULL
 * Asynchronous on 'stream'.  Errors: GNSS_EINVAL, GNSS_ECUDA. */
GNSS_API gnss_status gnss_refine_eval(gnss_plan* plan, const void* samples_dev, size_t n_samples, uint32_t coh_ms,
                                      const int32_t* prn_dev, const double* f_dev, const double* tau_dev, size_t n,
                                      float* P_dev, float* dPdf_dev, float* dPdtau_dev, void* stream);

/* Gradient ascent from each candidate, entirely on the device (one CTA per
 * candidate).
 *  Doppler pre-search: with search_hz > 0, P is first evaluated at
 *   f0 + k d, d = fs / (2 L) (half the main-lobe width), k = -1, +1, ...,
 *   +-floor(search_hz / d), and the ascent starts from the first largest
 *   value (f0 itself first).  A coarse Doppler bin wider than the coherent
 *   window's main lobe (1 / T) needs search_hz of about half the bin.
 *  Each iteration then moves f, then tau:
 *   f:   Newton step g_f / (P (2 pi)^2 T^2 / 6) (closed-form peak curvature,
 *        T = L / fs); trials alpha = 1, 1/2, ... (up to 20 halvings), taking
 *        the first that satisfies Armijo (c1 = 1e-4) or that reduces |dP/df|
 *        while losing at most 1e-5 of P (near the peak a change of P is below
 *        single-precision resolution but the gradient still resolves it);
 *   tau: sign step s_tau sign(g_tau), s_tau starting at 0.05 chip and
 *        shrinking by the accepted backtracking factor, with Armijo; when
 *        every trial fails, the opposite direction is tried (the segment
 *        slope is one-sided where samples sit exactly on a kink); when both
 *        fail, tau sits on the kink of the peak and s_tau shrinks by 2^20.
 *  Converged (status 0) when the Newton step in f is below 1e-3 Hz and s_tau
 *  below 1e-5 chip; stuck (status 1) when neither coordinate moves; status 2
 *  after max_iter iterations.
 *  samples            host recording, or device (16-byte aligned) when samples_on_device
 *  cands, out         host arrays of n_cand records
 * 'out' is valid once the stream has synchronised (a NULL stream is
 * synchronised before the call returns).  Errors: GNSS_EINVAL (window longer
 * than the recording, search_hz outside [0, 1e6], NULL), GNSS_ENOMEM,
 * GNSS_ECUDA. */
GNSS_API gnss_status gnss_refine(gnss_plan* plan, const void* samples, size_t n_samples, int samples_on_device,
                                 const gnss_candidate* cands, size_t n_cand, uint32_t coh_ms, uint32_t max_iter,
                                 double search_hz, gnss_refined* out, void* stream);

/* Device-resident form of gnss_refine: samples_dev, cands_dev and out_dev
 * are device pointers; never synchronises. */
GNSS_API gnss_status gnss_refine_device(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                        const gnss_candidate* cands_dev, size_t n_cand, uint32_t coh_ms,
                                        uint32_t max_iter, double search_hz, gnss_refined* out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Tracking channels (Section 3, Fig. 3).  A tracking channel shares the
 * carrier and code NCOs and the first mixing stage with acquisition, but
 * correlates in the time domain at early / prompt / late code offsets and
 * closes a carrier loop and a code loop around them.  The paper gives the
 * channel as a block diagram; the loop design here is this library's
 * reading, built like a hardware receiver's:
 *   NCOs in fixed point: carrier phase Phi (uint32, 2^32 = one cycle), word
 *     Wc = round(f 2^32 / fs) (two's complement); code position P in units of
 *     2^-32 chip in [0, 1023 2^32), word Wk = round(f_code 2^32 / fs)
 *     (rounding half away from zero).
 *   Interval k = samples kL + i, i < L = coh_ms N:
 *     s_i   = x[kL + i] exp(-j 2 pi (Phi + i Wc) / 2^32),
 *     Z_E/P/L = sum s_i c[floor((P + i Wk + {+h, 0, -h}) / 2^32) mod 1023],
 *     h = round(spacing / 2 * 2^32); the record's delay is (-P / 2^32) mod 1023
 *     chips at the interval start; then Phi += L Wc, P += L Wk.
 *   e_phi = atan(Q_P / I_P) / (2 pi) cycles (Costas; 0 when Z_P = 0),
 *   e_tau = (1 - spacing / 2) (|Z_L| - |Z_E|) / (|Z_L| + |Z_E|) chips.
 *   PLL, 2nd order, zeta = 1/sqrt(2), w_n = 8 zeta B_pll / (4 zeta^2 + 1):
 *     f_int += w_n^2 T e_phi,  f = f_int + 2 zeta w_n e_phi  (T = L / fs).
 *   DLL, 1st order, carrier aided: f_code = R_c (1 + f / f_L1) - 4 B_dll e_tau,
 *     f_L1 = 1540 R_c.
 *   Start: f_int = f = f0 (channel f_hz), Phi = 0, P = round(-tau0 2^32) mod.
 * Correlator sums in FP32, loop state in double.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint32_t coh_ms;       /* integration interval (ms), 1..1000                     */
  uint32_t n_int;        /* intervals to run from the recording start, >= 1         */
  float spacing_chips;   /* early-late spacing in (0, 1]                            */
  float pll_bw_hz;       /* PLL noise bandwidth, 0..1000 (0 = carrier NCO free-runs) */
  float dll_bw_hz;       /* DLL noise bandwidth, 0..1000 (0 = carrier aiding only)   */
  uint32_t reserved;
} gnss_track_config;

typedef struct {
  double f_hz;          /* carrier NCO frequency of the interval (Hz), Wc fs / 2^32 */
  double tau_chips;     /* replica code delay at the interval start, [0, 1023)     */
  float ze[2];          /* early correlator (I, Q)                                  */
  float zp[2];          /* prompt correlator                                       */
  float zl[2];          /* late correlator                                         */
  float e_phi;          /* Costas discriminator (cycles)                            */
  float e_tau;          /* DLL discriminator (chips)                                */
  int32_t status;       /* 0; -1 PRN not in the plan; -2 an NCO left its range     */
                        /* (the channel stops and its later records say -2)        */
  uint32_t reserved;
} gnss_track_rec;       /* 56 bytes */

/* Track n_chan channels over one recording: channel c starts from
 * chans_dev[c] (PRN, f_hz, tau_chips: e.g. refined acquisition results) and
 * writes out_dev[c * n_int + k] for intervals k < n_int.  The plan supplies
 * fs (N >= 2048: under one chip per sample), the recording format and the
 * PRN codes.  samples_dev, chans_dev and out_dev are device pointers; the
 * work is enqueued on 'stream' (one CTA per channel).  Errors: GNSS_EINVAL
 * (NULL arguments, fs < 2.048 MHz, configuration out of range, n_int * L >
 * n_samples, misaligned samples), GNSS_ECUDA. */
GNSS_API gnss_status gnss_track(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                const gnss_candidate* chans_dev, size_t n_chan, const gnss_track_config* cfg,
                                gnss_track_rec* out_dev, void* stream);

/* ------------------------------------------------------------------------
 * Serving.  The paper's cloud deployment runs many receiver instances per
 * server and rates throughput by the effective running time of concurrent
 * instances (Section 4); for the GPU it names fewer, larger operations as the
 * cure for per-thread GPU calls serialising (Section 5, Listing 3b).  The
 * server keeps plans and code spectra resident, admits submitted recordings
 * while their device memory fits the budget, and batches every admitted
 * request into one launch (continuous batching), with several batches in
 * flight so that new requests overlap with running ones.
 * ------------------------------------------------------------------------ */
typedef struct gnss_server gnss_server;

typedef struct {
  size_t device_mem_budget;   /* device bytes held by requests in flight (0 = 16 GiB) */
  size_t host_staging_bytes;  /* pinned host bytes for queued recordings and records (0 = 1 GiB) */
  uint32_t max_batch;         /* requests per batched launch (0 = 64) */
  uint32_t streams;           /* streams carrying batches, two in flight each (0 = 2, at most 16) */
  uint32_t queue_timeout_ms;  /* fail requests still queued after this long with GNSS_ETIMEOUT (0 = never) */
  uint32_t max_queue_wait_ms; /* admission bound: refuse with GNSS_EBUSY a request whose projected wait
                                 (the work queued and in flight ahead of it, plus its own, at the server's
                                 measured throughput) exceeds this (0 = no bound) */
} gnss_server_config;

typedef struct {
  uint64_t submitted;
  uint64_t completed;
  uint64_t failed;
  uint64_t batches;               /* batched launches so far */
  uint64_t queued;                /* requests waiting for admission now */
  uint32_t batches_in_flight;
  uint32_t refused;               /* submissions refused by the admission bound (saturating) */
  size_t device_bytes_reserved;   /* device bytes of batches in flight now */
} gnss_server_stats;

/* Start a server on the current device (cfg NULL = defaults): allocates the
 * pinned staging arena and the streams and starts the dispatcher thread.
 * Errors: GNSS_EINVAL, GNSS_ENOMEM, GNSS_ECUDA. */
GNSS_API gnss_status gnss_server_create(const gnss_server_config* cfg, gnss_server** out);

/* Fail still-queued requests with GNSS_ECANCELLED, wait for batches in
 * flight, release everything (NULL is accepted). */
GNSS_API gnss_status gnss_server_destroy(gnss_server* srv);

/* Queue one recording (host memory, copied before return: the caller may
 * free it) for acquisition with the plan 'desc' describes; *ticket names it.
 * Thread-safe.  Errors: GNSS_EINVAL (descriptor, length, GNSS_SECOND_WHOLE),
 * GNSS_EBUSY (host staging full, the request alone exceeds the device
 * budget, or -- with max_queue_wait_ms -- its projected wait exceeds that
 * bound: the work of the requests queued and in flight plus its own, in
 * algorithmic FLOPs of the acquisition, over the throughput the server has
 * achieved while busy; no bound applies before the first batch completes),
 * GNSS_ECANCELLED (server shutting down). */
GNSS_API gnss_status gnss_submit(gnss_server* srv, const gnss_plan_desc* desc, const void* host_samples,
                                 size_t n_samples, uint64_t* ticket);

/* Result of a request: GNSS_EAGAIN while queued or running; otherwise its
 * status (GNSS_OK with *n records copied to out, at most cap; or the error
 * that ended it) -- and the ticket is released. */
GNSS_API gnss_status gnss_poll(gnss_server* srv, uint64_t ticket, gnss_detection* out, size_t cap, size_t* n);

/* gnss_poll that blocks up to timeout_ms; GNSS_ETIMEOUT if the request is
 * still queued or running then (it keeps running; poll again later). */
GNSS_API gnss_status gnss_wait(gnss_server* srv, uint64_t ticket, uint32_t timeout_ms, gnss_detection* out,
                               size_t cap, size_t* n);

/* Cancel a request: a queued one is dropped, a running one has its records
 * discarded; its poll then returns GNSS_ECANCELLED. */
GNSS_API gnss_status gnss_cancel(gnss_server* srv, uint64_t ticket);

/* Counters of the server. */
GNSS_API gnss_status gnss_server_get_stats(gnss_server* srv, gnss_server_stats* out);


/* Launch-shape autotuner of the correlate kernel (the FFT-heavy stage).  It
 * can hold 8, 16 or 32 FFT elements per thread (N/8, N/16 or N/32 threads
 * per FFT; 8 needs N <= 8192 and runs radix-8 passes, 32 needs N >= 1024,
 * 16 needs N <= 16384), and with 16 it can stage the
 * next block's spectrum into shared memory by a bulk TMA copy while the
 * current block is transformed (variant code 16 | GNSS_TUNE_STAGED, offered
 * where the CTA's shared memory still fits: N <= 8192).  At N = 4096 and
 * 8192 the 16-per-thread form can also run the class-local pass schedule
 * (variant code 16 | GNSS_TUNE_CLASS_LOCAL, the default there): after the
 * first radix-16 pass the transform splits into 16 independent N/16-point
 * transforms, each on half a warp (4096) or a warp (8192), so one CTA
 * barrier per block instead of two or three.  At N = 16384 variant code
 * 32 | GNSS_TUNE_CLASS_LOCAL splits each transform by
 * decimation in time into two 8192-point class-local transforms, run by the
 * two CTAs of a thread-block cluster (one per output parity, 16 elements
 * and 16 sums per thread), which merge their row statistics through
 * distributed shared memory.
 *
 * GNSS_TUNE_TMEM (N = 2048, 4096, 8192 with 16 per thread, N = 16384 with
 * 32) keeps the code spectra and the non-coherent sums in the SM's tensor
 * memory instead of re-reading C_p from L2 every block and holding the sums
 * in registers; with 16 per thread the freed registers hold the next block's
 * spectrum, loaded under the current block's transform.  Its CTA shape is
 * part of the code: GNSS_TUNE_PRNS(k) PRNs per CTA (k = 1 or 2; one spectrum
 * load feeds k products and transforms; 1 at 16384) and GNSS_TUNE_BINS(m)
 * Doppler bins per CTA (m = 1 or 2, run one after another with the code
 * spectra kept).  It gives the register form's surfaces and records bit for
 * bit.  GNSS_TUNE_OCC (one PRN and bin per CTA; N = 2048, 4096, 8192, 16384
 * with 16 per thread) is its occupancy form: the sums read from tensor memory
 * only after each transform and no prefetch, so more CTAs fit an SM: the
 * class-local schedule at 64 registers with one shared-memory exchange
 * buffer per CTA (eight CTAs of 128 threads at 2048, four of 256, two of
 * 512, one of 1024: 32 warps per SM), the twiddle bases in tensor memory
 * too; the default at 4096, 8192 and 16384.  Bit-identical to the register
 * form at 2048-8192; at 16384 it factors the transform as
 * radix 16-16-16-4 (the register forms there use 32 per thread), so its
 * surfaces agree with the others to rounding.  A shape is valid only where
 * the tensor-memory columns of the CTAs that fit one SM together (registers,
 * shared memory, threads) total at most 512, so co-resident CTAs never wait
 * for columns.
 *
 * With force_elems = 0 every valid variant is timed on a probe shaped like
 * the plan (its Doppler bins up to 32, its sets, 8 blocks) and the fastest
 * is recorded for the plan's FFT size on the current device; with
 * force_elems = a variant code that variant is recorded without timing
 * (GNSS_EINVAL if it is not valid for N).  Later launches of that FFT size
 * (single, batched, served) use it.  Synchronous.  out may be NULL. */
#define GNSS_TUNE_STAGED 0x100u
#define GNSS_TUNE_CLASS_LOCAL 0x200u
#define GNSS_TUNE_TMEM 0x400u
#define GNSS_TUNE_OCC 0x800u /* TMEM variant, one PRN and bin: the occupancy form (more CTAs per SM) */
#define GNSS_TUNE_PRNS(k) ((((uint32_t)(k)) - 1u) << 12) /* PRNs per CTA (TMEM variant) */
#define GNSS_TUNE_BINS(m) ((((uint32_t)(m)) - 1u) << 14) /* Doppler bins per CTA (TMEM variant) */
typedef struct {
  uint32_t N;             /* FFT size tuned                                 */
  uint32_t n_variants;    /* variants timed                                 */
  uint32_t elems[16];     /* variant code of each timed variant: elements   */
                          /* per thread | GNSS_TUNE_STAGED,                 */
                          /* GNSS_TUNE_CLASS_LOCAL or GNSS_TUNE_TMEM with   */
                          /* its GNSS_TUNE_PRNS / GNSS_TUNE_BINS            */
  float ms[16];           /* median probe time of each (ms)                 */
  uint32_t chosen;        /* variant code now in use for N                  */
  uint32_t prns_per_cta;  /* PRNs one correlate CTA takes under 'chosen'    */
  uint32_t bins_per_cta;  /* Doppler bins one correlate CTA takes           */
  uint32_t reserved;
} gnss_tune_result;

GNSS_API gnss_status gnss_autotune(gnss_plan* plan, uint32_t force_elems, gnss_tune_result* out);


/* Message of the last failed call on this thread ("" if none). */
GNSS_API const char* gnss_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GNSS_H */

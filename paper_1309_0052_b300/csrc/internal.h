// internal.h -- private declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gnss_testing.h"

namespace gnss {

// Per-row statistics of one (set, PRN, Doppler) row of a power surface:
// the row maximum, its code phase (smallest on ties) and the largest cell
// whose circular distance from that phase exceeds the exclusion half-width.
struct RowStat {
  float peak;
  uint32_t tau;
  float second;
  uint32_t pad;
};

// One acquisition problem as the kernels see it.
struct AcqShape {
  int fs;          // Hz
  int N;           // samples per ms (FFT size)
  int coh;         // coherent ms per block
  int B;           // blocks processed
  int D;           // Doppler bins
  int G;           // fold groups (bins sharing f mod 1000; 1 when coh == 1)
  int P;           // PRNs
  int sets;        // 1, or 2 with half-bit sets
  int excl;        // second-peak exclusion half-width (samples)
  int dopp_min;    // Hz
  int dopp_step;   // Hz
  int format;      // gnss_format
  int code_dopp;   // GNSS_CODE_DOPPLER
  int second_whole;
  float threshold;
  // Spectrum classes: bins whose frequencies differ by whole kHz share one
  // forward spectrum, circularly shifted (Y_{f + 1000 K}[k] = Y_f[k + K]).
  // C = 0: one spectrum per bin (the stage entry points, code Doppler).
  int C;                  // classes
  const int* cls_fgroup;  // [C] fold group of each class
  const int* cls_base;    // [C] frequency (Hz) of each class's spectrum
  const int* bin_cls;     // [D] class of each bin
  const int* bin_shift;   // [D] (f_d - cls_base) / 1000
  const int* bin_order;   // [D] bins class by class: the order correlate tiles run in
};

// Kernel arguments of the correlate + detection kernel.
struct XcorrArgs {
  const float2* Y;        // [D or C][B][N] spectra of the wiped, folded blocks
  const int* bin_cls;     // NULL (row d of Y) or [D] spectrum row of each bin
  const int* bin_shift;   // NULL or [D] circular shift of that row (bins)
  const int* bin_order;   // NULL (tiles bin by bin) or [D] bin of each tile row
  const float2* cspec;    // [P][N] code spectra
  int B, D, P, excl;
  float* surface;         // NULL or [sets][P][D][N]
  RowStat* rows;          // [sets][P][D]
  unsigned* counters;     // [P + 1] zero on entry: CTAs finished per PRN, then this
                          // call's status word (GNSS_DET_* bits for the records)
  const int* prns;        // [P]
  gnss_detection* out;    // [P]
  int dopp_min, dopp_step;
  float threshold;
  int second_whole;
};

// Kernel arguments of the fold kernel (k_fold): one request.
struct FoldArgs {
  const uint8_t* samples;  // recording
  const int* gkey;         // [G] f mod 1000 per fold group
  float2* Z;               // [G][B][N] folded blocks
  unsigned* counters;      // NULL or [P + 1] per-PRN counters and status word to clear
  int coh, B, P;
};

// Kernel arguments of the carrier + forward FFT kernel (k_carrier_fft).
struct CarrierArgs {
  const float2* Z;         // [G][B][N]
  const int* group;        // [D] fold group per Doppler bin
  const int* cls_fgroup;   // NULL (one spectrum per bin) or [C] fold group per class
  const int* cls_base;     // [C] frequency of each class (with cls_fgroup)
  float2* Y;               // [D or C][B][N]
  int fs, coh, B, dopp_min, dopp_step;
  int code_dopp;           // GNSS_CODE_DOPPLER: rotate block b by sigma_b samples
};

// One request of a batched launch.
struct BatchReq {
  FoldArgs fold;
  CarrierArgs car;
  XcorrArgs xc;
};

// One batched launch triple: n requests sharing N, format and sets; the CTAs
// of request r in each kernel are [base[r], base[r + 1]).
struct BatchGroup {
  int N, format, sets, n;
  int variant;                // correlate variant the CTA offsets were counted for
  const BatchReq* reqs;       // device [n]
  const uint32_t* fold_base;  // device [n + 1]
  const uint32_t* car_base;   // device [n + 1]
  const uint32_t* xc_base;    // device [n + 1]
  uint32_t fold_ctas, car_ctas, xc_ctas;
};

FoldArgs fold_args(const AcqShape& s, const uint8_t* d_samples, const int* d_gkey, float2* d_Z, unsigned* d_counters);
CarrierArgs carrier_args(const AcqShape& s, const int* d_group, const float2* d_Z, float2* d_Y);
XcorrArgs xcorr_args(const AcqShape& s, const float2* d_Y, const float2* d_cspec, const int* d_prns,
                     float* d_surface, RowStat* d_rows, unsigned* d_counters, gnss_detection* d_out);
cudaError_t launch_batch(const BatchGroup& g, cudaStream_t stream);
uint32_t fold_ctas_per_block(int N);

// Byte offsets of one acquisition's scratch (each piece 256-byte aligned).
struct AcqScratch {
  size_t z;         // float2 [G][B][N]  folded blocks
  size_t y;         // float2 [D][B][N]  spectra
  size_t rows;      // RowStat [sets][P][D]
  size_t counters;  // unsigned [P + 1]: per-PRN CTA counters, then the call's status word
  size_t total;
};
AcqScratch scratch_layout(const AcqShape& s);

// Launchers (acq.cu).  All are asynchronous on 'stream'.
cudaError_t launch_gold(const int* d_prns, int P, int8_t* d_codes, cudaStream_t stream);
cudaError_t launch_code_spectra(const int8_t* d_codes, int P, int N, float2* d_cspec, cudaStream_t stream);
// k_fold + k_carrier_fft: Y from the recording.  d_counters (may be NULL) is
// cleared for the k_xcorr launch that follows on the same stream.
// Upload the fold kernel's per-millisecond factors to the current device
// (once per device; plan creation calls it).
cudaError_t ensure_fold_roots();
// fold, then carrier + forward FFT; 'between' (may be NULL) is recorded on
// the stream between the two launches.
cudaError_t launch_wipe_fft(const AcqShape& s, const uint8_t* d_samples, const int* d_group, const int* d_gkey,
                            float2* d_Z, float2* d_Y, unsigned* d_counters, cudaStream_t stream,
                            cudaEvent_t between = nullptr);
// k_xcorr: surfaces, row statistics and per-PRN detections.  d_counters must
// be zero on entry.
cudaError_t launch_xcorr(const AcqShape& s, const float2* d_Y, const float2* d_cspec, const int* d_prns,
                         float* d_surface, RowStat* d_rows, unsigned* d_counters, gnss_detection* d_out,
                         cudaStream_t stream);
bool supported_fft_size(int N);

// Correlate-kernel variant (elements per thread E) per device and FFT size.
int xcorr_variant(int N);
int xcorr_default_e(int N);
bool xcorr_valid_e(int N, int code);
// Iterations a staged-correlate wait polls before it gives up (testing).
cudaError_t set_stage_wait_limit(unsigned iters, cudaStream_t stream);
cudaError_t set_buf_wait_limit(unsigned iters, cudaStream_t stream);
void set_xcorr_variant(int N, int E);
// Correlate CTAs of one request (P PRNs, D bins) under variant 'code': one
// per (PRN, bin), or per group of PRNs and bins (GNSS_TUNE_TMEM shapes).
uint32_t xcorr_ctas(int code, int P, int D);

// The TMEM correlate variant (xcorr_tm.cu): variant codes
// E | GNSS_TUNE_TMEM | GNSS_TUNE_PRNS(K) | GNSS_TUNE_BINS(M).
bool xcorr_tm_valid(int N, int code);
int xcorr_tm_prns(int code);
int xcorr_tm_bins(int code);
cudaError_t launch_xcorr_tm(int code, const AcqShape& s, const XcorrArgs& a, cudaStream_t stream);
cudaError_t launch_xcorr_tm_batch(int code, const BatchGroup& g, cudaStream_t stream);

// Fine acquisition (refine.cu).
struct RefineJob {
  const uint8_t* samples;  // device recording, 16-byte aligned
  int format;
  int N;                   // samples per ms
  int L;                   // samples in the coherent window (from the recording start)
  double fs;
  double inv_fs;           // 1 / fs
  const int8_t* codes;     // [P][1023] +-1
  const int* prn_index;    // [33] plan index of PRN 1..32 (-1 = not in the plan)
};
cudaError_t launch_refine_eval(const RefineJob& J, int n, const int* prn, const double* f, const double* tau,
                               float* P, float* dPdf, float* dPdtau, cudaStream_t s);
cudaError_t launch_refine(const RefineJob& J, int n, const gnss_candidate* cands, int max_iter, double search_hz,
                          gnss_refined* out, cudaStream_t s);

// Shared C-ABI helpers (capi.cu): thread-local error message, status from a
// CUDA error, current-device check and scratch from the library pool.
gnss_status fail_status(gnss_status st, const std::string& msg);
gnss_status cuda_status(cudaError_t e, const char* where);
gnss_status check_plan_device(const gnss_plan* plan);
gnss_status scratch_alloc(int dev, size_t bytes, cudaStream_t stream, void** out);

// Fold groups of a plan's Doppler grid (bins sharing f mod 1000; one group
// when coh_ms == 1): group[d] for every bin, gkey[g] = f mod 1000.  Returns G.
int fold_groups(const gnss_plan_desc& d, std::vector<int>& group, std::vector<int>& gkey);
// Spectrum classes of a plan's grid (bins with equal f mod 1000): packed as
// fold group [C], base frequency [C], class [D], shift [D].  Returns C.
int spectrum_classes(const gnss_plan_desc& d, const std::vector<int>& group, std::vector<int>& packed);
}  // namespace gnss
struct gnss_plan;
namespace gnss {
// Set the spectrum-class fields of a shape from its plan.
void spectrum_args(const gnss_plan* plan, AcqShape* s);
// Whole blocks of a recording under a plan (capped by noncoh and INT32_MAX),
// and the kernels' view of one acquisition of B blocks (capi.cu; every entry
// point that launches an acquisition builds its shape with these).
int blocks_of(const gnss_plan* plan, size_t n_samples);
AcqShape shape_of(const gnss_plan* plan, int B);

// Last-error message (thread-local), set by the C-ABI layer.
void set_error(const std::string& msg);

}  // namespace gnss

struct gnss_plan {
  gnss_plan_desc desc;
  int device;
  int N;
  int P;
  int D;
  int sets;
  int excl;
  int prns[32];
  int G;              // fold groups
  int* d_prns;        // [P]
  int* d_group;       // [D] fold group of each Doppler bin
  int* d_gkey;        // [G] f mod 1000 of each group (0 when coh_ms == 1)
  int* d_prn_index;   // [33] plan index of PRN 1..32, -1 when not searched
  int C;              // spectrum classes (0 with GNSS_CODE_DOPPLER: one per bin)
  int* d_cls;         // [2 C + 3 D]: fold group [C], base Hz [C], class [D], shift [D], tile order [D]
  int8_t* d_codes;    // [P][1023] +-1 chips
  float2* d_cspec;    // [P][N] FFT of the sampled replica
};

// internal.h -- private declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "gnss.h"

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
  int P;           // PRNs
  int sets;        // 1, or 2 with half-bit sets
  int excl;        // second-peak exclusion half-width (samples)
  int dopp_min;    // Hz
  int dopp_step;   // Hz
  int format;      // gnss_format
  int second_whole;
  float threshold;
};

// Launchers (acq.cu).  All are asynchronous on 'stream'.
cudaError_t launch_gold(const int* d_prns, int P, int8_t* d_codes, cudaStream_t stream);
cudaError_t launch_code_spectra(const int8_t* d_codes, int P, int N, float2* d_cspec, cudaStream_t stream);
cudaError_t launch_wipe_fft(const AcqShape& s, const uint8_t* d_samples, float2* d_Y, cudaStream_t stream);
cudaError_t launch_xcorr(const AcqShape& s, const float2* d_Y, const float2* d_cspec, float* d_surface,
                         RowStat* d_rows, cudaStream_t stream);
cudaError_t launch_peak(const AcqShape& s, const RowStat* d_rows, const int* d_prns, const float* d_surface,
                        gnss_detection* d_out, cudaStream_t stream);
bool supported_fft_size(int N);

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
  int* d_prns;        // [P]
  int8_t* d_codes;    // [P][1023] +-1 chips
  float2* d_cspec;    // [P][N] FFT of the sampled replica
};

// tune.cu -- autotuner of the correlate kernel's launch shape.
//
// The correlate kernel (conj-multiply, IFFT, |.|^2, non-coherent sum) can
// hold E = 8, 16 or 32 FFT elements per thread: N / E threads per FFT,
// different register budgets, occupancy and exchange costs; with E = 16 it
// can also stage the next block by a bulk TMA copy (more shared memory) or
// run the class-local pass schedule, and the TMEM form keeps the code
// spectra and sums in tensor memory with a CTA shape of 1-2 PRNs and 1-2
// Doppler bins.  Which one is faster depends on the FFT size (and the GPU),
// so gnss_autotune times every valid choice on a probe shaped like the plan
// and records the fastest for that FFT size on the current device; every
// later launch (single or batched) uses it.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

using namespace gnss;

extern "C" GNSS_API gnss_status gnss_autotune(gnss_plan* plan, uint32_t force_elems, gnss_tune_result* out) {
  if (!plan) return fail_status(GNSS_EINVAL, "NULL argument");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  const int N = plan->N;
  gnss_tune_result res;
  memset(&res, 0, sizeof(res));
  res.N = (uint32_t)N;
  const int TM = (int)GNSS_TUNE_TMEM;
  const int cand[] = {16,
                      32,
                      16 | (int)GNSS_TUNE_STAGED,
                      8,
                      16 | (int)GNSS_TUNE_CLASS_LOCAL,
                      32 | (int)GNSS_TUNE_CLASS_LOCAL,
                      16 | TM,
                      16 | TM | (int)GNSS_TUNE_PRNS(2),
                      16 | TM | (int)GNSS_TUNE_BINS(2),
                      16 | TM | (int)GNSS_TUNE_PRNS(2) | (int)GNSS_TUNE_BINS(2),
                      16 | TM | (int)GNSS_TUNE_OCC,
                      32 | TM,
                      32 | TM | (int)GNSS_TUNE_BINS(2)};
  constexpr int n_cand = (int)(sizeof(cand) / sizeof(cand[0]));
  static_assert(n_cand <= 16, "gnss_tune_result holds 16 variants");
  if (force_elems) {
    if (force_elems > 0xffffu || !xcorr_valid_e(N, (int)force_elems))
      return fail_status(GNSS_EINVAL, "variant must be 8 (N <= 8192), 16 (N <= 16384), 32 (N >= 1024), 16 | GNSS_TUNE_STAGED "
                                      "(N <= 8192), 16 | GNSS_TUNE_CLASS_LOCAL (N = 4096 or 8192), "
                                      "32 | GNSS_TUNE_CLASS_LOCAL (N = 16384), or 16 | GNSS_TUNE_TMEM (N = 2048, "
                                      "4096, 8192; GNSS_TUNE_PRNS 1-2, GNSS_TUNE_BINS 1-2; or GNSS_TUNE_OCC alone at "
                                      "2048 and 4096) or 32 | GNSS_TUNE_TMEM (N = 16384; GNSS_TUNE_BINS 1-2) where "
                                      "its tensor-memory columns fit");
    set_xcorr_variant(N, (int)force_elems);
    res.chosen = force_elems;
    res.prns_per_cta = (uint32_t)xcorr_tm_prns((int)force_elems);
    res.bins_per_cta = (uint32_t)xcorr_tm_bins((int)force_elems);
    if (out) *out = res;
    return GNSS_OK;
  }
  // probe: the plan's Doppler bins (at most 32) and sets, 8 blocks of zeros
  AcqShape s;
  memset(&s, 0, sizeof(s));
  s.fs = (int)plan->desc.fs_hz;
  s.N = N;
  s.coh = (int)plan->desc.coh_ms;
  s.B = 8;
  s.D = std::min(plan->D, 32);
  s.G = 1;
  s.P = plan->P;
  s.sets = plan->sets;
  s.excl = plan->excl;
  s.threshold = plan->desc.threshold;
  const AcqScratch lay = scratch_layout(s);
  const size_t det = ((size_t)s.P * sizeof(gnss_detection) + 255) & ~(size_t)255;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_status(e, "cudaStreamCreate");
  char* ws = nullptr;
  st = scratch_alloc(plan->device, lay.total + det, cs, (void**)&ws);
  if (st != GNSS_OK) {
    cudaStreamDestroy(cs);
    return st;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMemsetAsync(ws, 0, lay.total + det, cs);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int prev = xcorr_variant(N);
  float best = 0.f;
  int best_e = prev;
  for (int k = 0; k < n_cand && e == cudaSuccess; ++k) {
    const int E = cand[k];
    if (!xcorr_valid_e(N, E)) continue;
    set_xcorr_variant(N, E);
    std::vector<float> t;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
      e = cudaMemsetAsync(ws + lay.counters, 0, sizeof(unsigned) * (s.P + 1), cs);
      if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
      if (e == cudaSuccess)
        e = launch_xcorr(s, reinterpret_cast<const float2*>(ws + lay.y), plan->d_cspec, plan->d_prns, nullptr,
                         reinterpret_cast<RowStat*>(ws + lay.rows), reinterpret_cast<unsigned*>(ws + lay.counters),
                         reinterpret_cast<gnss_detection*>(ws + lay.total), cs);
      if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) t.push_back(ms);  // the first run warms up
    }
    if (e != cudaSuccess) break;
    std::sort(t.begin(), t.end());
    const float med = t[t.size() / 2];
    res.elems[res.n_variants] = (uint32_t)E;
    res.ms[res.n_variants] = med;
    res.n_variants++;
    if (best == 0.f || med < best) {
      best = med;
      best_e = E;
    }
  }
  set_xcorr_variant(N, e == cudaSuccess ? best_e : prev);
  res.chosen = (uint32_t)xcorr_variant(N);
  res.prns_per_cta = (uint32_t)xcorr_tm_prns((int)res.chosen);
  res.bins_per_cta = (uint32_t)xcorr_tm_bins((int)res.chosen);
  cudaFreeAsync(ws, cs);
  cudaStreamSynchronize(cs);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return cuda_status(e, "gnss_autotune");
  if (out) *out = res;
  return GNSS_OK;
}

// zoom.cu -- second-stage fine Doppler search around coarse detections.
//
// The coarse grid of an acquisition plan is as wide as the search needs and
// as fine as its cost allows; a detected satellite's Doppler is only known to
// the grid step.  The zoom re-runs the acquisition channel (Section 3,
// Fig. 2: wipe-off, FFT, conj-multiply, IFFT, |.|^2, non-coherent sum,
// peak / second peak) for each detection alone, on a grid zoom times finer
// spanning +-span coarse steps around the detected bin:
//   f_k = f_det + (k - span zoom) step / zoom,   k < 2 span zoom + 1.
// Each detection becomes one request of a batched launch whose plan is
// derived from the coarse one: same sample rate, coherent length, format,
// flags and threshold; one PRN, whose code and code spectrum rows are the
// coarse plan's own (nothing is recomputed); its own fine grid and fold
// groups.  Every zoomed record is exactly what gnss_acquire_device returns
// for a plan created with that fine grid and that single PRN.
#include <cuda_runtime.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.h"

using namespace gnss;

extern "C" GNSS_API gnss_status gnss_acquire_zoom(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                                  const gnss_detection* det, size_t n_det, uint32_t zoom,
                                                  uint32_t span, gnss_detection* out_dev, float* surface_dev,
                                                  void* stream) {
  if (!plan || !samples_dev || !out_dev || (n_det && !det)) return fail_status(GNSS_EINVAL, "NULL argument");
  if (n_det == 0) return GNSS_OK;
  if (n_det > 4096) return fail_status(GNSS_EINVAL, "at most 4096 detections per call");
  if (zoom < 2 || zoom > 1000) return fail_status(GNSS_EINVAL, "zoom must be in [2, 1000]");
  if (span < 1 || span > 100) return fail_status(GNSS_EINVAL, "span must be in [1, 100]");
  const gnss_plan_desc& pd = plan->desc;
  if (pd.dopp_step_hz == 0 || pd.dopp_step_hz % zoom != 0)
    return fail_status(GNSS_EINVAL, "the plan's Doppler step must be a positive multiple of zoom");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  const uint32_t fine = pd.dopp_step_hz / zoom;
  const uint32_t D = 2 * span * zoom + 1;
  std::vector<gnss_plan> sub(n_det);
  std::vector<std::vector<int>> groups(n_det), gkeys(n_det);
  std::vector<size_t> off(n_det);
  size_t bytes = 0;
  for (size_t i = 0; i < n_det; ++i) {
    const int prn = det[i].prn;
    int row = -1;
    for (int k = 0; k < plan->P; ++k)
      if (plan->prns[k] == prn) row = k;
    if (row < 0) return fail_status(GNSS_EINVAL, "detection " + std::to_string(i) + ": PRN not in the plan");
    const int64_t fmin = (int64_t)det[i].dopp_hz - (int64_t)span * pd.dopp_step_hz;
    if (fmin < INT32_MIN / 2 || fmin + (int64_t)(D - 1) * fine > INT32_MAX / 2)
      return fail_status(GNSS_EINVAL, "detection " + std::to_string(i) + ": Doppler out of range");
    gnss_plan& p = sub[i];
    memset(&p, 0, sizeof(p));
    p.desc = pd;
    p.desc.dopp_min_hz = (int32_t)fmin;
    p.desc.dopp_step_hz = fine;
    p.desc.n_dopp = D;
    p.desc.prn_mask = 1ull << (prn - 1);
    p.device = plan->device;
    p.N = plan->N;
    p.P = 1;
    p.D = (int)D;
    p.sets = plan->sets;
    p.excl = plan->excl;
    p.prns[0] = prn;
    p.G = fold_groups(p.desc, groups[i], gkeys[i]);
    p.d_codes = plan->d_codes + (size_t)row * 1023;
    p.d_cspec = plan->d_cspec + (size_t)row * plan->N;
    off[i] = bytes;  // prn, then group[D], then gkey[G], 16-byte aligned per detection
    bytes += ((1 + D + (size_t)p.G) * sizeof(int) + 15) & ~(size_t)15;
  }
  std::vector<int> host(bytes / sizeof(int), 0);
  for (size_t i = 0; i < n_det; ++i) {
    int* h = host.data() + off[i] / sizeof(int);
    h[0] = sub[i].prns[0];
    memcpy(h + 1, groups[i].data(), sizeof(int) * D);
    memcpy(h + 1 + D, gkeys[i].data(), sizeof(int) * sub[i].G);
  }
  cudaStream_t cs = (cudaStream_t)stream;
  char* ws = nullptr;
  st = scratch_alloc(plan->device, bytes, cs, (void**)&ws);
  if (st != GNSS_OK) return st;
  cudaError_t e = cudaMemcpyAsync(ws, host.data(), bytes, cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) {
    cudaFreeAsync(ws, cs);
    return cuda_status(e, "gnss_acquire_zoom");
  }
  std::vector<gnss_request> reqs(n_det);
  const size_t surf_each = (size_t)plan->sets * D * plan->N;
  for (size_t i = 0; i < n_det; ++i) {
    int* d = reinterpret_cast<int*>(ws + off[i]);
    sub[i].d_prns = d;
    sub[i].d_group = d + 1;
    sub[i].d_gkey = d + 1 + D;
    reqs[i].plan = &sub[i];
    reqs[i].samples_dev = samples_dev;
    reqs[i].n_samples = n_samples;
    reqs[i].out_dev = out_dev + i;
    reqs[i].surface_dev = surface_dev ? surface_dev + i * surf_each : nullptr;
  }
  st = gnss_acquire_batch(reqs.data(), n_det, 0, stream);
  cudaFreeAsync(ws, cs);
  return st;
}

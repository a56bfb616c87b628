// capi.cu -- C ABI of the acquisition library (include/gnss.h): plans,
// acquisition entry points, stage entry points, errors and scratch memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace gnss {

static thread_local std::string t_error;

void set_error(const std::string& msg) { t_error = msg; }

static gnss_status fail(gnss_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

static gnss_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GNSS_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Library-owned stream-ordered pool per device, keeping freed blocks cached
// so that repeated acquisitions do not return memory to the driver.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[128];
static bool g_pool_ok[128];

static cudaError_t device_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool_ok[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    g_pool_ok[dev] = true;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

gnss_status scratch_alloc(int dev, size_t bytes, cudaStream_t stream, void** out) {
  cudaMemPool_t pool;
  cudaError_t e = device_pool(dev, &pool);
  if (e != cudaSuccess) return cuda_fail(e, "memory pool");
  e = cudaMallocFromPoolAsync(out, bytes, pool, stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(GNSS_ENOMEM, "device scratch allocation of " + std::to_string(bytes) + " bytes failed");
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync");
  return GNSS_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

gnss_status fail_status(gnss_status st, const std::string& msg) { return fail(st, msg); }
gnss_status cuda_status(cudaError_t e, const char* where) { return cuda_fail(e, where); }
gnss_status check_plan_device(const gnss_plan* plan);

gnss_status check_plan_device(const gnss_plan* plan) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return fail(GNSS_EINVAL, "plan belongs to another device than the current one");
  return GNSS_OK;
}

AcqShape shape_of(const gnss_plan* plan, int B) {
  AcqShape s;
  s.fs = (int)plan->desc.fs_hz;
  s.N = plan->N;
  s.coh = (int)plan->desc.coh_ms;
  s.B = B;
  s.D = plan->D;
  s.G = plan->G;
  s.P = plan->P;
  s.sets = plan->sets;
  s.excl = plan->excl;
  s.dopp_min = plan->desc.dopp_min_hz;
  s.dopp_step = (int)plan->desc.dopp_step_hz;
  s.format = (int)plan->desc.format;
  s.second_whole = (plan->desc.flags & GNSS_SECOND_WHOLE) ? 1 : 0;
  s.code_dopp = (plan->desc.flags & GNSS_CODE_DOPPLER) ? 1 : 0;
  s.threshold = plan->desc.threshold;
  spectrum_args(plan, &s);
  return s;
}

int blocks_of(const gnss_plan* plan, size_t n_samples) {
  const size_t L = (size_t)plan->desc.coh_ms * plan->N;
  size_t B = n_samples / L;
  if (plan->desc.noncoh && B > plan->desc.noncoh) B = plan->desc.noncoh;
  if (B > (size_t)INT32_MAX) B = INT32_MAX;
  return (int)B;
}

static size_t rec_bytes(uint32_t format, size_t n) {
  return format == GNSS_FMT_I8_IQ ? 2 * n : (n + 1) / 2;
}

// Shared body of gnss_acquire / gnss_acquire_device.
static gnss_status acquire_impl(gnss_plan* plan, const void* samples, size_t n_samples, int samples_on_device,
                                gnss_detection* out_host, gnss_detection* out_dev, float* surface_dev,
                                cudaStream_t stream, void* const* events = nullptr) {
  if (!plan || !samples || (!out_host && !out_dev)) return fail(GNSS_EINVAL, "NULL argument");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  const int B = blocks_of(plan, n_samples);
  if (B < 1) return fail(GNSS_EINVAL, "n_samples is shorter than one coherent block");
  if (samples_on_device && ((uintptr_t)samples & 15u)) return fail(GNSS_EINVAL, "device samples must be 16-byte aligned");
  if ((plan->desc.flags & GNSS_SECOND_WHOLE) && !surface_dev)
    return fail(GNSS_EINVAL, "GNSS_SECOND_WHOLE needs a surface buffer");
  const AcqShape s = shape_of(plan, B);
  const AcqScratch lay = scratch_layout(s);
  const size_t smp_bytes = samples_on_device ? 0 : align256(rec_bytes(plan->desc.format, (size_t)B * s.coh * s.N));
  const size_t det_bytes = out_dev ? 0 : align256((size_t)s.P * sizeof(gnss_detection));
  char* ws = nullptr;
  st = scratch_alloc(plan->device, lay.total + det_bytes + smp_bytes, stream, (void**)&ws);
  if (st != GNSS_OK) return st;
  float2* d_Z = reinterpret_cast<float2*>(ws + lay.z);
  float2* d_Y = reinterpret_cast<float2*>(ws + lay.y);
  RowStat* d_rows = reinterpret_cast<RowStat*>(ws + lay.rows);
  unsigned* d_cnt = reinterpret_cast<unsigned*>(ws + lay.counters);
  gnss_detection* d_det = out_dev ? out_dev : reinterpret_cast<gnss_detection*>(ws + lay.total);
  const uint8_t* d_smp = reinterpret_cast<const uint8_t*>(samples);
  cudaError_t e = cudaSuccess;
  if (!samples_on_device) {
    uint8_t* dst = reinterpret_cast<uint8_t*>(ws + lay.total + det_bytes);
    e = cudaMemcpyAsync(dst, samples, rec_bytes(plan->desc.format, (size_t)B * s.coh * s.N),
                        cudaMemcpyHostToDevice, stream);
    d_smp = dst;
  }
  // stage-boundary events of the traced entry point (caller-owned)
  auto mark = [&](int k) {
    if (e == cudaSuccess && events && events[k]) e = cudaEventRecord((cudaEvent_t)events[k], stream);
  };
  mark(0);
  if (e == cudaSuccess)
    e = launch_wipe_fft(s, d_smp, plan->d_group, plan->d_gkey, d_Z, d_Y, d_cnt, stream,
                        events ? (cudaEvent_t)events[1] : nullptr);
  mark(2);
  if (e == cudaSuccess)
    e = launch_xcorr(s, d_Y, plan->d_cspec, plan->d_prns, surface_dev, d_rows, d_cnt, d_det, stream);
  mark(3);
  if (e == cudaSuccess && out_host)
    e = cudaMemcpyAsync(out_host, d_det, (size_t)s.P * sizeof(gnss_detection), cudaMemcpyDeviceToHost, stream);
  cudaError_t ef = cudaFreeAsync(ws, stream);
  if (e != cudaSuccess) return cuda_fail(e, "acquire");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  if (stream == nullptr && out_host) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int p = 0; p < s.P; ++p)
      if (out_host[p].flags & GNSS_DET_TIMEOUTS)
        return fail(GNSS_ETIMEOUT, (out_host[p].flags & GNSS_DET_WAIT_TIMEOUT)
                                       ? "a bounded wait between the warps of a correlate CTA gave up (records "
                                         "flagged GNSS_DET_WAIT_TIMEOUT, not valid)"
                                       : "a bounded wait of the staged correlate kernel gave up (records complete, "
                                         "flagged GNSS_DET_STAGE_TIMEOUT)");
  }
  return GNSS_OK;
}

}  // namespace gnss

namespace gnss {

// Spectrum classes: bins whose frequencies differ by whole kHz have forward
// spectra that are circular shifts of one another (a kHz is one cycle per
// 1 ms block, one bin of its FFT), so each class keeps one spectrum per
// block, the one of its lowest frequency, and bin d reads it shifted by
// (f_d - base) / 1000.  A class spans under 16 kHz (shift < 16), which keeps
// the shift below the correlate kernel's thread count.  The class's fold group is its bins' (fold groups
// partition by f mod 1000 too, or hold every bin when coh_ms = 1).
int spectrum_classes(const gnss_plan_desc& d, const std::vector<int>& group, std::vector<int>& packed) {
  const int D = (int)d.n_dopp;
  std::vector<int> key_of_class, fgroup, base, cls(D), shift(D);
  for (int k = 0; k < D; ++k) {
    const int64_t f = (int64_t)d.dopp_min_hz + (int64_t)k * d.dopp_step_hz;
    const int key = (int)(((f % 1000) + 1000) % 1000);
    int c = -1;  // the class of this residue whose base is within 15 kHz below f
    for (size_t q = 0; q < key_of_class.size(); ++q)
      if (key_of_class[q] == key && f - base[q] < 16 * 1000) c = (int)q;
    if (c < 0) {  // bins ascend in frequency, so the first bin of a class is its lowest
      c = (int)key_of_class.size();
      key_of_class.push_back(key);
      fgroup.push_back(group[k]);
      base.push_back((int)f);
    }
    cls[k] = c;
    shift[k] = (int)((f - base[c]) / 1000);
  }
  const int C = (int)key_of_class.size();
  // correlate tiles run class by class, so that CTAs resident together read
  // the blocks of few spectrum rows (L2 locality for long recordings)
  std::vector<int> order;
  for (int c = 0; c < C; ++c)
    for (int k = 0; k < D; ++k)
      if (cls[k] == c) order.push_back(k);
  packed.clear();
  packed.insert(packed.end(), fgroup.begin(), fgroup.end());
  packed.insert(packed.end(), base.begin(), base.end());
  packed.insert(packed.end(), cls.begin(), cls.end());
  packed.insert(packed.end(), shift.begin(), shift.end());
  packed.insert(packed.end(), order.begin(), order.end());
  return C;
}

void spectrum_args(const gnss_plan* plan, AcqShape* s) {
  s->C = plan->C;
  s->cls_fgroup = plan->C ? plan->d_cls : nullptr;
  s->cls_base = plan->C ? plan->d_cls + plan->C : nullptr;
  s->bin_cls = plan->C ? plan->d_cls + 2 * plan->C : nullptr;
  s->bin_shift = plan->C ? plan->d_cls + 2 * plan->C + plan->D : nullptr;
  s->bin_order = plan->C ? plan->d_cls + 2 * plan->C + 2 * plan->D : nullptr;
}

// Fold groups: the per-millisecond wipe-off factor exp(-j 2 pi (f i mod 1000) / 1000)
// depends on f only through f mod 1000 (and not at all with one coherent ms).
int fold_groups(const gnss_plan_desc& d, std::vector<int>& group, std::vector<int>& gkey) {
  group.assign(d.n_dopp, 0);
  gkey.clear();
  for (uint32_t k = 0; k < d.n_dopp; ++k) {
    const int64_t f = (int64_t)d.dopp_min_hz + (int64_t)k * d.dopp_step_hz;
    const int key = d.coh_ms == 1 ? 0 : (int)(((f % 1000) + 1000) % 1000);
    int gi = -1;
    for (size_t q = 0; q < gkey.size(); ++q)
      if (gkey[q] == key) gi = (int)q;
    if (gi < 0) {
      gi = (int)gkey.size();
      gkey.push_back(key);
    }
    group[k] = gi;
  }
  return (int)gkey.size();
}

}  // namespace gnss

using namespace gnss;

extern "C" {

const char* gnss_last_error(void) { return t_error.c_str(); }

size_t gnss_recording_bytes(uint32_t format, size_t n_samples) { return rec_bytes(format, n_samples); }

gnss_status gnss_plan_create(const gnss_plan_desc* desc, gnss_plan** out) {
  if (!desc || !out) return fail(GNSS_EINVAL, "NULL argument");
  *out = nullptr;
  const gnss_plan_desc& d = *desc;
  if (d.fs_hz == 0 || d.fs_hz % 1000) return fail(GNSS_EINVAL, "fs_hz must be a positive multiple of 1000");
  const int N = (int)(d.fs_hz / 1000);
  if (!supported_fft_size(N)) return fail(GNSS_EINVAL, "fs_hz / 1000 must be a power of two in [256, 16384]");
  if (d.coh_ms < 1 || d.coh_ms > 100000) return fail(GNSS_EINVAL, "coh_ms must be in [1, 100000]");
  if (d.n_dopp < 1 || d.n_dopp > 100000) return fail(GNSS_EINVAL, "n_dopp must be in [1, 100000]");
  if (d.n_dopp > 1 && d.dopp_step_hz < 1) return fail(GNSS_EINVAL, "dopp_step_hz must be >= 1");
  const int64_t fmax = (int64_t)d.dopp_min_hz + (int64_t)(d.n_dopp - 1) * d.dopp_step_hz;
  if (fmax > INT32_MAX / 2 || (int64_t)d.dopp_min_hz < INT32_MIN / 2) return fail(GNSS_EINVAL, "Doppler grid out of range");
  if ((d.prn_mask & 0xFFFFFFFFull) == 0 || (d.prn_mask >> 32)) return fail(GNSS_EINVAL, "prn_mask must select PRNs within 1..32");
  if (d.format != GNSS_FMT_I8_IQ && d.format != GNSS_FMT_2BIT_IQ) return fail(GNSS_EINVAL, "unknown format");
  if (d.flags & ~(GNSS_HALF_BIT | GNSS_SECOND_WHOLE | GNSS_CODE_DOPPLER)) return fail(GNSS_EINVAL, "unknown flags");
  if (!(d.threshold >= 0.f) || isinf(d.threshold)) return fail(GNSS_EINVAL, "threshold must be finite and >= 0");

  gnss_plan* p = new (std::nothrow) gnss_plan;
  if (!p) return fail(GNSS_ENOMEM, "host allocation failed");
  memset(p, 0, sizeof(*p));
  p->desc = d;
  p->N = N;
  p->D = (int)d.n_dopp;
  p->sets = (d.flags & GNSS_HALF_BIT) ? 2 : 1;
  p->excl = (N + 1022) / 1023;
  for (int prn = 1; prn <= 32; ++prn)
    if (d.prn_mask >> (prn - 1) & 1ull) p->prns[p->P++] = prn;
  std::vector<int> group, gkey, cls;
  p->G = fold_groups(d, group, gkey);
  // shared spectra unless code-Doppler rotations make every bin's spectrum its own
  p->C = (d.flags & GNSS_CODE_DOPPLER) ? 0 : spectrum_classes(d, group, cls);
  if (p->C >= p->D) p->C = 0;  // nothing shared: keep one spectrum per bin
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = ensure_fold_roots();
  // settle the correlate variant of this FFT size on this device now (its
  // default asks the runtime for occupancies), outside any later stream capture
  if (e == cudaSuccess) (void)xcorr_variant(N);
  cudaStream_t st = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_prns, sizeof(int) * p->P);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_codes, (size_t)p->P * 1023);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_cspec, (size_t)p->P * N * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_group, sizeof(int) * p->D);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_gkey, sizeof(int) * p->G);
  if (e == cudaSuccess && p->C) e = cudaMalloc(&p->d_cls, sizeof(int) * cls.size());
  int prn_index[33];
  for (int k = 0; k < 33; ++k) prn_index[k] = -1;
  for (int k = 0; k < p->P; ++k) prn_index[p->prns[k]] = k;
  if (e == cudaSuccess) e = cudaMalloc(&p->d_prn_index, sizeof(prn_index));
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_prn_index, prn_index, sizeof(prn_index), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_prns, p->prns, sizeof(int) * p->P, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_group, group.data(), sizeof(int) * p->D, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_gkey, gkey.data(), sizeof(int) * p->G, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && p->C)
    e = cudaMemcpyAsync(p->d_cls, cls.data(), sizeof(int) * cls.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_gold(p->d_prns, p->P, p->d_codes, st);
  if (e == cudaSuccess) e = launch_code_spectra(p->d_codes, p->P, N, p->d_cspec, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    gnss_status r = (e == cudaErrorMemoryAllocation) ? fail(GNSS_ENOMEM, "device allocation failed")
                                                      : cuda_fail(e, "gnss_plan_create");
    cudaFree(p->d_prns);
    cudaFree(p->d_codes);
    cudaFree(p->d_cspec);
    cudaFree(p->d_group);
    cudaFree(p->d_gkey);
    cudaFree(p->d_cls);
    cudaFree(p->d_prn_index);
    delete p;
    return r;
  }
  *out = p;
  return GNSS_OK;
}

gnss_status gnss_plan_destroy(gnss_plan* plan) {
  if (!plan) return GNSS_OK;
  cudaFree(plan->d_prns);
  cudaFree(plan->d_codes);
  cudaFree(plan->d_cspec);
  cudaFree(plan->d_group);
  cudaFree(plan->d_gkey);
  cudaFree(plan->d_cls);
  cudaFree(plan->d_prn_index);
  delete plan;
  return GNSS_OK;
}

gnss_status gnss_plan_get_info(const gnss_plan* plan, gnss_plan_info* out) {
  if (!plan || !out) return fail(GNSS_EINVAL, "NULL argument");
  out->N = (uint32_t)plan->N;
  out->n_prn = (uint32_t)plan->P;
  out->n_dopp = (uint32_t)plan->D;
  out->n_sets = (uint32_t)plan->sets;
  out->excl = (uint32_t)plan->excl;
  out->block_len = plan->desc.coh_ms * (uint32_t)plan->N;
  out->xcorr_variant = (uint32_t)xcorr_variant(plan->N);
  return GNSS_OK;
}

gnss_status gnss_plan_codes(const gnss_plan* plan, int8_t* out, size_t cap) {
  if (!plan || !out) return fail(GNSS_EINVAL, "NULL argument");
  if (cap < (size_t)plan->P * 1023) return fail(GNSS_EINVAL, "output too small");
  cudaError_t e = cudaMemcpy(out, plan->d_codes, (size_t)plan->P * 1023, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_plan_codes");
  return GNSS_OK;
}

gnss_status gnss_plan_code_spectra(const gnss_plan* plan, float* out_dev, size_t cap, void* stream) {
  if (!plan || !out_dev) return fail(GNSS_EINVAL, "NULL argument");
  const size_t bytes = (size_t)plan->P * plan->N * sizeof(float2);
  if (cap < bytes) return fail(GNSS_EINVAL, "output too small");
  cudaError_t e = cudaMemcpyAsync(out_dev, plan->d_cspec, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_plan_code_spectra");
  return GNSS_OK;
}

gnss_status gnss_acquire(gnss_plan* plan, const void* samples, size_t n_samples, int samples_on_device,
                         gnss_detection* out, float* surface_dev, void* stream) {
  return acquire_impl(plan, samples, n_samples, samples_on_device, out, nullptr, surface_dev, (cudaStream_t)stream);
}

gnss_status gnss_acquire_device(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                gnss_detection* out_dev, float* surface_dev, void* stream) {
  if (!out_dev) return fail(GNSS_EINVAL, "NULL argument");
  return acquire_impl(plan, samples_dev, n_samples, 1, nullptr, out_dev, surface_dev, (cudaStream_t)stream);
}

gnss_status gnss_acquire_device_traced(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                       gnss_detection* out_dev, float* surface_dev, void* stream,
                                       void* const* events) {
  if (!out_dev || !events) return fail(GNSS_EINVAL, "NULL argument");
  return acquire_impl(plan, samples_dev, n_samples, 1, nullptr, out_dev, surface_dev, (cudaStream_t)stream,
                      events);
}

gnss_status gnss_stage_wipe_fft(gnss_plan* plan, const void* samples_dev, size_t n_samples, uint32_t n_blocks,
                                float* spectra_dev, void* stream) {
  if (!plan || !samples_dev || !spectra_dev) return fail(GNSS_EINVAL, "NULL argument");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  if ((uintptr_t)samples_dev & 15u) return fail(GNSS_EINVAL, "device samples must be 16-byte aligned");
  const size_t L = (size_t)plan->desc.coh_ms * plan->N;
  if (n_blocks < 1 || (size_t)n_blocks > n_samples / L) return fail(GNSS_EINVAL, "n_blocks out of range");
  AcqShape s = shape_of(plan, (int)n_blocks);
  s.C = 0;  // the stage layout is one spectrum per bin
  const AcqScratch lay = scratch_layout(s);
  cudaStream_t cs = (cudaStream_t)stream;
  float2* d_Z = nullptr;
  st = scratch_alloc(plan->device, lay.y - lay.z, cs, (void**)&d_Z);
  if (st != GNSS_OK) return st;
  cudaError_t e = launch_wipe_fft(s, (const uint8_t*)samples_dev, plan->d_group, plan->d_gkey, d_Z,
                                  (float2*)spectra_dev, nullptr, cs);
  cudaError_t ef = cudaFreeAsync(d_Z, cs);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_stage_wipe_fft");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return GNSS_OK;
}

gnss_status gnss_stage_correlate(gnss_plan* plan, const float* spectra_dev, uint32_t n_blocks, float* surface_dev,
                                 gnss_detection* out_dev, void* stream) {
  if (!plan || !spectra_dev || !out_dev || n_blocks < 1) return fail(GNSS_EINVAL, "bad argument");
  if ((uintptr_t)spectra_dev & 15u) return fail(GNSS_EINVAL, "spectra_dev must be 16-byte aligned");
  gnss_status st = check_plan_device(plan);
  if (st != GNSS_OK) return st;
  if ((plan->desc.flags & GNSS_SECOND_WHOLE) && !surface_dev)
    return fail(GNSS_EINVAL, "GNSS_SECOND_WHOLE needs a surface buffer");
  AcqShape s = shape_of(plan, (int)n_blocks);
  s.C = 0;  // the stage layout is one spectrum per bin
  const AcqScratch lay = scratch_layout(s);
  cudaStream_t cs = (cudaStream_t)stream;
  char* ws = nullptr;
  st = scratch_alloc(plan->device, lay.total - lay.rows, cs, (void**)&ws);
  if (st != GNSS_OK) return st;
  RowStat* rows = reinterpret_cast<RowStat*>(ws);
  unsigned* cnt = reinterpret_cast<unsigned*>(ws + (lay.counters - lay.rows));
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (s.P + 1), cs);
  if (e == cudaSuccess)
    e = launch_xcorr(s, (const float2*)spectra_dev, plan->d_cspec, plan->d_prns, surface_dev, rows, cnt, out_dev, cs);
  cudaError_t ef = cudaFreeAsync(ws, cs);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_stage_correlate");
  if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  return GNSS_OK;
}

}  // extern "C"

namespace gnss {

// Batched acquisition, planned once on the host: requests are validated and
// grouped by (FFT size, format, sets); each group runs longest first and is
// cut into waves whose scratch fits the budget.  A wave's device tables are
// its BatchReq records and the three CTA-offset arrays.
struct Wave {
  int N, format, sets;
  std::vector<size_t> idx;  // requests of the wave, in launch order
  size_t bytes;             // scratch of its requests
};

static size_t wave_desc_bytes(size_t n) {
  return align256(sizeof(BatchReq) * n) + align256(3 * sizeof(uint32_t) * (n + 1));
}

static gnss_status plan_batch(const gnss_request* reqs, size_t n_req, size_t scratch_budget, int dev,
                              std::vector<AcqShape>& shape, std::vector<AcqScratch>& lay, std::vector<Wave>& waves) {
  if (!reqs) return fail(GNSS_EINVAL, "NULL argument");
  if (n_req > (size_t)INT32_MAX) return fail(GNSS_EINVAL, "too many requests");
  if (scratch_budget == 0) scratch_budget = (size_t)16 << 30;
  shape.assign(n_req, AcqShape());
  lay.assign(n_req, AcqScratch());
  std::map<std::tuple<int, int, int>, std::vector<size_t>> groups;
  for (size_t i = 0; i < n_req; ++i) {
    const gnss_request& r = reqs[i];
    const std::string at = "request " + std::to_string(i) + ": ";
    if (!r.plan || !r.samples_dev || !r.out_dev) return fail(GNSS_EINVAL, at + "NULL plan, samples or output");
    if (r.plan->device != dev) return fail(GNSS_EINVAL, at + "plan belongs to another device than the current one");
    if ((uintptr_t)r.samples_dev & 15u) return fail(GNSS_EINVAL, at + "device samples must be 16-byte aligned");
    if ((r.plan->desc.flags & GNSS_SECOND_WHOLE) && !r.surface_dev)
      return fail(GNSS_EINVAL, at + "GNSS_SECOND_WHOLE needs a surface buffer");
    const int B = blocks_of(r.plan, r.n_samples);
    if (B < 1) return fail(GNSS_EINVAL, at + "n_samples is shorter than one coherent block");
    shape[i] = shape_of(r.plan, B);
    lay[i] = scratch_layout(shape[i]);
    groups[std::make_tuple(shape[i].N, shape[i].format, shape[i].sets)].push_back(i);
  }
  waves.clear();
  for (auto& kv : groups) {
    std::vector<size_t>& idx = kv.second;
    // longest correlate CTAs (most blocks) first, so the tail is short ones
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return shape[a].B > shape[b].B; });
    size_t pos = 0;
    while (pos < idx.size()) {
      size_t end = pos, bytes = 0;
      while (end < idx.size() && (end == pos || bytes + lay[idx[end]].total <= scratch_budget)) bytes += lay[idx[end++]].total;
      Wave w;
      w.N = std::get<0>(kv.first);
      w.format = std::get<1>(kv.first);
      w.sets = std::get<2>(kv.first);
      w.idx.assign(idx.begin() + pos, idx.begin() + end);
      w.bytes = bytes;
      // CTA counts of the three launches must fit the 32-bit offsets
      uint64_t nf = 0, nc = 0, nx = 0;
      const uint32_t cpb = fold_ctas_per_block(w.N);
      for (size_t i : w.idx) {
        const AcqShape& sh = shape[i];
        nf += (uint64_t)sh.G * sh.B * cpb;
        nc += (uint64_t)(sh.C ? sh.C : sh.D) * sh.B;
        nx += (uint64_t)xcorr_ctas(xcorr_variant(w.N), sh.P, sh.D);
      }
      if (nf > INT32_MAX || nc > INT32_MAX || nx > INT32_MAX)
        return fail(GNSS_EINVAL, "a wave needs more than 2^31 CTAs; lower scratch_budget");
      waves.push_back(std::move(w));
      pos = end;
    }
  }
  return GNSS_OK;
}

// Host tables of one wave whose request scratch starts at 'scratch' and whose
// device tables will be copied to 'desc'; g describes the launch triple.
static void fill_wave(const Wave& w, const gnss_request* reqs, const std::vector<AcqShape>& shape,
                      const std::vector<AcqScratch>& lay, char* scratch, char* desc, std::vector<BatchReq>& hr,
                      std::vector<uint32_t>& hb, BatchGroup& g) {
  const int n = (int)w.idx.size();
  hr.assign(n, BatchReq());
  hb.assign(3 * (size_t)(n + 1), 0u);
  uint32_t* fb = hb.data();
  uint32_t* cb = fb + (n + 1);
  uint32_t* xb = cb + (n + 1);
  char* cur = scratch;
  const uint32_t cpb = fold_ctas_per_block(w.N);
  const int variant = xcorr_variant(w.N);
  for (int k = 0; k < n; ++k) {
    const size_t i = w.idx[k];
    const gnss_request& r = reqs[i];
    const AcqShape& sh = shape[i];
    const AcqScratch& L = lay[i];
    float2* Z = reinterpret_cast<float2*>(cur + L.z);
    float2* Y = reinterpret_cast<float2*>(cur + L.y);
    RowStat* rows = reinterpret_cast<RowStat*>(cur + L.rows);
    unsigned* cnt = reinterpret_cast<unsigned*>(cur + L.counters);
    hr[k].fold = fold_args(sh, (const uint8_t*)r.samples_dev, r.plan->d_gkey, Z, cnt);
    hr[k].car = carrier_args(sh, r.plan->d_group, Z, Y);
    hr[k].xc = xcorr_args(sh, Y, r.plan->d_cspec, r.plan->d_prns, r.surface_dev, rows, cnt, r.out_dev);
    fb[k + 1] = fb[k] + (uint32_t)(sh.G * sh.B * cpb);
    cb[k + 1] = cb[k] + (uint32_t)((sh.C ? sh.C : sh.D) * sh.B);  // carrier tiles
    xb[k + 1] = xb[k] + xcorr_ctas(variant, sh.P, sh.D);
    cur += L.total;
  }
  BatchReq* d_reqs = reinterpret_cast<BatchReq*>(desc);
  uint32_t* d_base = reinterpret_cast<uint32_t*>(desc + align256(sizeof(BatchReq) * n));
  g.N = w.N;
  g.format = w.format;
  g.sets = w.sets;
  g.n = n;
  g.variant = variant;
  g.reqs = d_reqs;
  g.fold_base = d_base;
  g.car_base = d_base + (n + 1);
  g.xc_base = d_base + 2 * (n + 1);
  g.fold_ctas = fb[n];
  g.car_ctas = cb[n];
  g.xc_ctas = xb[n];
}

}  // namespace gnss

extern "C" {

gnss_status gnss_acquire_batch(const gnss_request* reqs, size_t n_req, size_t scratch_budget, void* stream) {
  if (n_req == 0) return GNSS_OK;
  if (!reqs) return fail(GNSS_EINVAL, "NULL argument");
  cudaStream_t cs = (cudaStream_t)stream;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  // validate everything before launching anything
  std::vector<AcqShape> shape;
  std::vector<AcqScratch> lay;
  std::vector<Wave> waves;
  gnss_status st = plan_batch(reqs, n_req, scratch_budget, dev, shape, lay, waves);
  if (st != GNSS_OK) return st;
  std::vector<BatchReq> hr;
  std::vector<uint32_t> hb;
  for (const Wave& w : waves) {
    const size_t desc_bytes = wave_desc_bytes(w.idx.size());
    char* ws = nullptr;
    st = scratch_alloc(dev, desc_bytes + w.bytes, cs, (void**)&ws);
    if (st != GNSS_OK) return st;
    BatchGroup g;
    fill_wave(w, reqs, shape, lay, ws + desc_bytes, ws, hr, hb, g);
    e = cudaMemcpyAsync(ws, hr.data(), sizeof(BatchReq) * hr.size(), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<uint32_t*>(g.fold_base), hb.data(), sizeof(uint32_t) * hb.size(),
                          cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = launch_batch(g, cs);
    cudaError_t ef = cudaFreeAsync(ws, cs);
    if (e != cudaSuccess) return cuda_fail(e, "gnss_acquire_batch");
    if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
  }
  return GNSS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched acquisition captured once into a CUDA graph (the batch mode of
// Section 5 as one replayable launch).
// ---------------------------------------------------------------------------
struct gnss_batch_graph {
  int device;
  size_t n_req;
  void* scratch;  // one region reused by every wave (waves run in order)
  void* desc;     // every wave's device tables
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" {

gnss_status gnss_batch_graph_create(const gnss_request* reqs, size_t n_req, size_t scratch_budget,
                                    gnss_batch_graph** out) {
  if (!out) return fail(GNSS_EINVAL, "NULL argument");
  *out = nullptr;
  if (n_req == 0) return fail(GNSS_EINVAL, "empty batch");
  if (!reqs) return fail(GNSS_EINVAL, "NULL argument");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::vector<AcqShape> shape;
  std::vector<AcqScratch> lay;
  std::vector<Wave> waves;
  gnss_status st = plan_batch(reqs, n_req, scratch_budget, dev, shape, lay, waves);
  if (st != GNSS_OK) return st;
  size_t scratch_bytes = 0, desc_bytes = 0;
  for (const Wave& w : waves) {
    scratch_bytes = std::max(scratch_bytes, w.bytes);
    desc_bytes += wave_desc_bytes(w.idx.size());
  }
  gnss_batch_graph* g = new (std::nothrow) gnss_batch_graph();
  if (!g) return fail(GNSS_ENOMEM, "host allocation failed");
  g->device = dev;
  g->n_req = n_req;
  cudaStream_t cs = nullptr;
  e = cudaMalloc(&g->scratch, scratch_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&g->desc, desc_bytes);
  // device tables are written now; the graph holds only the launches
  std::vector<BatchGroup> groups(waves.size());
  std::vector<BatchReq> hr;
  std::vector<uint32_t> hb;
  size_t off = 0;
  for (size_t k = 0; k < waves.size() && e == cudaSuccess; ++k) {
    char* d = reinterpret_cast<char*>(g->desc) + off;
    fill_wave(waves[k], reqs, shape, lay, reinterpret_cast<char*>(g->scratch), d, hr, hb, groups[k]);
    e = cudaMemcpy(d, hr.data(), sizeof(BatchReq) * hr.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(const_cast<uint32_t*>(groups[k].fold_base), hb.data(), sizeof(uint32_t) * hb.size(),
                     cudaMemcpyHostToDevice);
    off += wave_desc_bytes(waves[k].idx.size());
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t el = cudaSuccess;
    for (size_t k = 0; k < groups.size() && el == cudaSuccess; ++k) el = launch_batch(groups[k], cs);
    e = cudaStreamEndCapture(cs, &g->graph);  // ends the capture even after a failed launch
    if (e == cudaSuccess) e = el;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    gnss_status r = (e == cudaErrorMemoryAllocation) ? fail(GNSS_ENOMEM, "device allocation failed")
                                                      : cuda_fail(e, "gnss_batch_graph_create");
    gnss_batch_graph_destroy(g);
    return r;
  }
  *out = g;
  return GNSS_OK;
}

gnss_status gnss_batch_graph_launch(gnss_batch_graph* g, void* stream) {
  if (!g) return fail(GNSS_EINVAL, "NULL argument");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != g->device) return fail(GNSS_EINVAL, "graph belongs to another device than the current one");
  e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_batch_graph_launch");
  return GNSS_OK;
}

gnss_status gnss_batch_graph_destroy(gnss_batch_graph* g) {
  if (!g) return GNSS_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFree(g->scratch);
  cudaFree(g->desc);
  delete g;
  return GNSS_OK;
}

gnss_status gnss_testing_set_stage_wait_limit(uint32_t iters, void* stream) {
  const cudaError_t e = set_stage_wait_limit(iters, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_testing_set_stage_wait_limit");
  return GNSS_OK;
}

gnss_status gnss_testing_set_buf_wait_limit(uint32_t iters, void* stream) {
  const cudaError_t e = set_buf_wait_limit(iters, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gnss_testing_set_buf_wait_limit");
  return GNSS_OK;
}

}  // extern "C"

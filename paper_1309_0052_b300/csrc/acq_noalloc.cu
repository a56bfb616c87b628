// acq_noalloc.cu -- acquisition entry point that allocates no memory.
//
// gnss_acquire and gnss_acquire_device take their scratch (the Doppler x
// block spectra and the per-row peak statistics) from a stream-ordered
// memory pool.  Some callers cannot allow that: services that must keep a
// fixed device-memory footprint once started, or processes where another
// allocator (a framework's caching allocator, a reserved arena) owns the
// device memory, so a cudaMalloc / cudaMallocAsync at request time is
// forbidden or may fail.  gnss_acquire_noalloc serves them: it runs the
// same kernels with its scratch in the fixed array below, which is part of
// the library's device image.  Every GPU that loads the library holds this
// array until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "internal.h"

// Fixed scratch shared by every gnss_acquire_noalloc call on a device.
// 32 MiB holds the scratch of the 100 ms / 4.096 MHz / 81-bin / 10-block
// workload: 2.6 MB of spectra per class of bins (26.5 MB per bin with code
// Doppler) plus its folded blocks and row statistics.
#define GNSS_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[GNSS_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch per device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current (cudaGetSymbolAddress) and passed to the
// kernels.  The cache lives as long as the device's primary context: like
// the plans, it does not survive cudaDeviceReset (or another teardown of
// that context), after which the process must not call this entry point.
std::mutex g_mu;
void* g_addr[128];

gnss_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= 128) {
    gnss::set_error("gnss_acquire_noalloc: device index out of range");
    return GNSS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      gnss::set_error(std::string("gnss_acquire_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return GNSS_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return GNSS_OK;
}

}  // namespace

extern "C" GNSS_API gnss_status gnss_acquire_noalloc(gnss_plan* plan, const void* samples_dev, size_t n_samples,
                                                    gnss_detection* out_dev, float* surface_dev, void* stream) {
  using namespace gnss;
  if (!plan || !samples_dev || !out_dev) {
    set_error("gnss_acquire_noalloc: NULL argument");
    return GNSS_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("gnss_acquire_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return GNSS_ECUDA;
  }
  if (dev != plan->device) {
    set_error("gnss_acquire_noalloc: plan belongs to another device than the current one");
    return GNSS_EINVAL;
  }
  if ((uintptr_t)samples_dev & 15u) {
    set_error("gnss_acquire_noalloc: device samples must be 16-byte aligned");
    return GNSS_EINVAL;
  }
  const int B = blocks_of(plan, n_samples);
  if (B < 1) {
    set_error("gnss_acquire_noalloc: n_samples is shorter than one coherent block");
    return GNSS_EINVAL;
  }
  if ((plan->desc.flags & GNSS_SECOND_WHOLE) && !surface_dev) {
    set_error("gnss_acquire_noalloc: GNSS_SECOND_WHOLE needs a surface buffer");
    return GNSS_EINVAL;
  }
  // the same shape as gnss_acquire_device builds, so the same launches
  const AcqShape s = shape_of(plan, B);
  const AcqScratch lay = scratch_layout(s);
  if (lay.total > GNSS_NOALLOC_SCRATCH_BYTES) {
    set_error("gnss_acquire_noalloc: this request needs " + std::to_string(lay.total) +
              " bytes of scratch (folded blocks, blocks * N * 8 bytes of spectra per class of bins a whole kHz apart"
              " or per bin with code-Doppler compensation, row statistics),"
              " more than the fixed " + std::to_string((size_t)GNSS_NOALLOC_SCRATCH_BYTES) + " bytes");
    return GNSS_EINVAL;
  }
  void* base = nullptr;
  gnss_status st = scratch_address(dev, &base);
  if (st != GNSS_OK) return st;

  // Every value the kernels read is written earlier in this call (the
  // per-PRN counters are cleared by the first kernel), so the previous
  // call's contents need no clearing.
  unsigned char* sb = reinterpret_cast<unsigned char*>(base);
  cudaStream_t cs = (cudaStream_t)stream;
  e = launch_wipe_fft(s, (const uint8_t*)samples_dev, plan->d_group, plan->d_gkey,
                      reinterpret_cast<float2*>(sb + lay.z), reinterpret_cast<float2*>(sb + lay.y),
                      reinterpret_cast<unsigned*>(sb + lay.counters), cs);
  if (e == cudaSuccess)
    e = launch_xcorr(s, reinterpret_cast<const float2*>(sb + lay.y), plan->d_cspec, plan->d_prns, surface_dev,
                     reinterpret_cast<RowStat*>(sb + lay.rows), reinterpret_cast<unsigned*>(sb + lay.counters),
                     out_dev, cs);
  if (e != cudaSuccess) {
    set_error(std::string("gnss_acquire_noalloc: ") + cudaGetErrorString(e));
    return GNSS_ECUDA;
  }
  return GNSS_OK;
}

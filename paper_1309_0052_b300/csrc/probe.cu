// probe.cu -- FP32 FMA throughput probe used to state the ALU roof that
// bounds the acquisition kernels (not part of the acquisition itself).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace gnss {

// Eight independent FMA chains per thread; 'iters' rounds of 8 FMAs.  The
// result is stored only when it equals a value it never takes, so the
// compiler keeps the chains but nothing is written in practice.
__global__ void k_ffma_probe(int iters, float seed, float* __restrict__ sink) {
  float a0 = seed + threadIdx.x, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
  float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
  const float m = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, m, c);
      a1 = fmaf(a1, m, c);
      a2 = fmaf(a2, m, c);
      a3 = fmaf(a3, m, c);
      a4 = fmaf(a4, m, c);
      a5 = fmaf(a5, m, c);
      a6 = fmaf(a6, m, c);
      a7 = fmaf(a7, m, c);
    }
  }
  const float r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (r == -1.2345f) sink[blockIdx.x] = r;
}

}  // namespace gnss

using namespace gnss;

extern "C" GNSS_API gnss_status gnss_probe_ffma(int iters, double* tflops, double* ms, void* stream) {
  if (!tflops || iters < 1) return GNSS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 512, blocks = sms * 4;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) return GNSS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_ffma_probe<<<blocks, threads, 0, s>>>(iters / 8 + 1, 1.f, sink);  // warm-up
  cudaEventRecord(e0, s);
  k_ffma_probe<<<blocks, threads, 0, s>>>(iters, 1.f, sink);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) {
    set_error(cudaGetErrorString(e));
    return GNSS_ECUDA;
  }
  const double flops = 2.0 * 8 * 16 * (double)iters * threads * blocks;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return GNSS_OK;
}

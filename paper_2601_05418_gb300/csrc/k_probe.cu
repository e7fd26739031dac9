// FP32 FMA throughput probe: the measured denominator of the FP32 ALU
// roofline that the readout kernels (FFTs, pre / post factors, FP32 A_g
// contraction) are reported against.  Not part of the paper's method.
//
// Every thread runs eight independent FMA chains (enough independent work
// to cover the FMA latency at full occupancy) for `iters` iterations; the
// grid is the device's SM count x 8 blocks of 256 threads.  The chains'
// final values are summed into one output word so that no chain can be
// removed by the compiler.
#include <cuda_runtime.h>

#include "gpjc_kernels.h"

namespace gpjc {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(const float* __restrict__ seed, int iters,
                                                            float* __restrict__ out) {
  const float b = seed[0], c = seed[1];
  float a[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) a[j] = seed[2] + 1e-3f * (float)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) s += a[j];
  if (s == 1234.5f) out[0] = s;  // practically never taken; keeps every chain live
}

cudaError_t probe_fma_tflops(int iters, double* tflops) {
  int dev = 0, nsm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  float* buf = nullptr;
  if ((e = cudaMalloc(&buf, 4 * sizeof(float))) != cudaSuccess) return e;
  const float h[4] = {0.999999f, 1e-7f, 0.5f, 0.f};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  const int blocks = nsm * 8;
  if ((e = cudaMemcpy(buf, h, sizeof h, cudaMemcpyHostToDevice)) != cudaSuccess) goto done;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) goto done;
  // warm-up (clocks up, module loaded), then the timed launch
  note_launches(1); k_probe_fma<<<blocks, kProbeThreads>>>(buf, iters, buf + 3);
  cudaEventRecord(e0);
  note_launches(1); k_probe_fma<<<blocks, kProbeThreads>>>(buf, iters, buf + 3);
  cudaEventRecord(e1);
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) goto done;
  if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) goto done;
  *tflops = 2.0 * kProbeChains * (double)iters * blocks * kProbeThreads / (ms * 1e-3) / 1e12;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return e;
}

}  // namespace gpjc

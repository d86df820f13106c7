// apic_probe_fp32_fma: the FP32 CUDA-core throughput of this GPU, measured
// with independent fused multiply-add chains (the ALU ceiling that the push's
// arithmetic is compared with; the push itself is bound by memory traffic and
// instruction issue, far below it).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/apic.h"

namespace {

constexpr int kChains = 8;  // independent chains per thread: enough to cover the FMA latency

__device__ float g_probe_sink;

__global__ void __launch_bounds__(256) k_probe_fma(int reps, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) g_probe_sink = s;  // keeps the chains live; never true for these inputs
}

}  // namespace

extern "C" int apic_probe_fp32_fma(void* stream, int32_t reps, double* tflops) {
  if (!tflops || reps < 1) return APIC_ERR_INVALID_ARG;
  *tflops = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_fma, 256, 0) != cudaSuccess)
    return APIC_ERR_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return APIC_ERR_CUDA;
  // b < 1 and c small keep every chain bounded (a -> c / (1 - b))
  k_probe_fma<<<blocks, 256, 0, s>>>(reps, 0.999f, 1e-3f);  // warm-up
  cudaEventRecord(e0, s);
  k_probe_fma<<<blocks, 256, 0, s>>>(reps, 0.999f, 1e-3f);
  cudaEventRecord(e1, s);
  int rc = APIC_OK;
  float ms = 0.0f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess || !(ms > 0.0f)) {
    rc = APIC_ERR_CUDA;
  } else {
    const double flops = 2.0 * kChains * (double)reps * 256.0 * (double)blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// FMA-pipe throughput probe (measurement tooling for the roofline, built into the
// tooling library, not part of the reweighting ABI).  Every thread runs NCHAIN independent dependent
// chains of fused multiply-adds; the grid covers every SM several times, so the
// issue rate of the FP64 or FP32 FMA pipe is the only limit.
#include <cuda_runtime.h>

#include "../../../include/rex_tooling.h"

namespace {

template <typename T, int NCHAIN>
__global__ void __launch_bounds__(256) fma_chains(T* sink, int iters, T a, T b) {
  T x[NCHAIN];
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < NCHAIN; ++c) s += x[c];
  if (s == T(-1.2345)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the work
}

}  // namespace

extern "C" int rex_probe_fma(int fp64, double* flops_per_second, void* stream) {
  if (!flops_per_second) return REX_TOOLING_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return REX_TOOLING_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return REX_TOOLING_ECUDA;
  const int blocks = sms * 8, threads = 256;
  constexpr int NCHAIN = 8;
  const int iters = fp64 ? 512 : 16384;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, st);
    if (fp64)
      fma_chains<double, NCHAIN><<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999999, 1e-7);
    else
      fma_chains<float, NCHAIN><<<blocks, threads, 0, st>>>(nullptr, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return REX_TOOLING_ECUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * NCHAIN * (double)iters * blocks * threads;
  *flops_per_second = flops / (best * 1e-3);
  return cudaGetLastError() == cudaSuccess ? REX_TOOLING_OK : REX_TOOLING_ECUDA;
}

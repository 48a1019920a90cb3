// Check of the integer-ALU float conversions (fpconv.cuh) that the mixed-precision
// q q~ -> t t~ and q q~ -> t t~ g kernels use in place of FP64-pipe conversions.
// Test tooling, built into the tooling library, not part of the reweighting ABI.
#include <cuda_runtime.h>

#include "../../../include/rex_tooling.h"
#include "../fpconv.cuh"

namespace rex {

__global__ void convert_probe_kernel(const double* __restrict__ in, int64_t n, float* __restrict__ f32,
                                     double* __restrict__ f64, float* __restrict__ f32_finite) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float f = f64_to_f32_alu(in[i]);
  f32[i] = f;
  f64[i] = f32_to_f64_alu(f);
  if (f32_finite) {
    unsigned ahi_max = 0u;
    f32_finite[i] = f64_to_f32_alu_finite(in[i], ahi_max);
  }
}

}  // namespace rex

extern "C" int rex_probe_convert(const double* in, int64_t n, float* f32_out, double* f64_out,
                                 float* f32_finite_out, void* stream) {
  if (n < 0) return REX_TOOLING_EINVAL;
  if (n == 0) return REX_TOOLING_OK;
  if (!in || !f32_out || !f64_out) return REX_TOOLING_EINVAL;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return REX_TOOLING_EINVAL;
  rex::convert_probe_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, n, f32_out,
                                                                                           f64_out, f32_finite_out);
  return cudaGetLastError() == cudaSuccess ? REX_TOOLING_OK : REX_TOOLING_ECUDA;
}

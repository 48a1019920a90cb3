// Standalone launcher of the q q~ -> t t~ reweighting kernel (sm_103a), FP64 and mixed.
#include "../../include/rex.h"
#include "qq_kernel.cuh"

namespace rex {

// resident blocks per SM the register allocator must allow: FP64 4 (<= 128 registers),
// mixed 8 (<= 64 registers)
template <typename R, int MINB, bool EXCL>
__global__ void __launch_bounds__(QQ_BLOCK, MINB)
    qq_ttx_reweight_kernel(const double* __restrict__ mom, const double* __restrict__ w_in, int64_t nev,
                           const __grid_constant__ QcdLaunch lp, double* __restrict__ out,
                           const signed char* __restrict__ hel) {
  __shared__ typename QqTile<R>::Smem sm;
  QqTile<R>::template run<EXCL>(sm, mom, w_in, nev, (int64_t)blockIdx.x, lp, out, hel);
}

int launch_qq_ttx(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                  double* out, void* stream, const signed char* hel) {
  const int64_t blocks = (nev + QQ_BLOCK - 1) / QQ_BLOCK;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned g = (unsigned)blocks;
  if (mixed && hel) qq_ttx_reweight_kernel<float, 8, true><<<g, QQ_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel);
  else if (mixed) qq_ttx_reweight_kernel<float, 8, false><<<g, QQ_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr);
  else if (hel) qq_ttx_reweight_kernel<double, 4, true><<<g, QQ_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel);
  else qq_ttx_reweight_kernel<double, 4, false><<<g, QQ_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr);
  return (int)cudaGetLastError();
}

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
  if (n < 0) return REX_EINVAL;
  if (n == 0) return REX_OK;
  if (!in || !f32_out || !f64_out) return REX_EINVAL;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffffLL) return REX_EINVAL;
  rex::convert_probe_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, n, f32_out,
                                                                                           f64_out, f32_finite_out);
  return cudaGetLastError() == cudaSuccess ? REX_OK : REX_ECUDA;
}

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

}  // namespace rex

// Standalone launcher of the q q~ -> t t~ reweighting kernel (sm_103a), FP64 and mixed.
#include "qq_kernel.cuh"

namespace rex {

template <typename R>
__global__ void __launch_bounds__(QQ_BLOCK)
    qq_ttx_reweight_kernel(const double* __restrict__ mom, const double* __restrict__ w_in, int64_t nev,
                           const __grid_constant__ QcdLaunch lp, double* __restrict__ out) {
  __shared__ typename QqTile<R>::Smem sm;
  QqTile<R>::run(sm, mom, w_in, nev, (int64_t)blockIdx.x, lp, out);
}

int launch_qq_ttx(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                  double* out, void* stream) {
  const int64_t blocks = (nev + QQ_BLOCK - 1) / QQ_BLOCK;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mixed)
    qq_ttx_reweight_kernel<float><<<(unsigned)blocks, QQ_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  else
    qq_ttx_reweight_kernel<double><<<(unsigned)blocks, QQ_BLOCK, 0, st>>>(mom, w_in, nev, lp, out);
  return (int)cudaGetLastError();
}

}  // namespace rex

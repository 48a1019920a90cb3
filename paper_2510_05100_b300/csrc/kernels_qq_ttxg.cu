// Standalone launcher of the q q~ -> t t~ g reweighting kernel (sm_103a), FP64 and mixed.
#include "qqg_kernel.cuh"

namespace rex {

// resident blocks per SM the register allocator must allow: FP64 1, mixed 3 (168
// registers, no spill)
template <typename R, int MINB, bool EXCL, bool TCH = false>
__global__ void __launch_bounds__(QQG_BLOCK, MINB)
    qq_ttxg_reweight_kernel(const double* __restrict__ mom, const double* __restrict__ w_in, int64_t nev,
                            const __grid_constant__ QcdLaunch lp, double* __restrict__ out,
                            const signed char* __restrict__ hel, const __grid_constant__ QqgCrossing cross) {
  __shared__ typename QqgTile<R, TCH>::Smem sm;
  QqgTile<R, TCH>::template run<EXCL>(sm, mom, w_in, nev, (int64_t)blockIdx.x, lp, out, hel, cross);
}

int launch_qq_ttxg(int mixed, const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                   double* out, void* stream, const signed char* hel, const QqgCrossing& cross) {
  constexpr int EPB = QqgTile<float>::EPB;
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned g = (unsigned)blocks;
  // a crossed light line (q g, q~ g): the t-channel tile
  const bool tch = cross.neg[0] != 0 || cross.neg[1] != 0;
  if (mixed && hel) qq_ttxg_reweight_kernel<float, 3, true><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel, cross);
  else if (mixed && tch) qq_ttxg_reweight_kernel<float, 3, false, true><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr, cross);
  else if (mixed) qq_ttxg_reweight_kernel<float, 3, false><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr, cross);
  else if (hel) qq_ttxg_reweight_kernel<double, 1, true><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, hel, cross);
  else if (tch) qq_ttxg_reweight_kernel<double, 1, false, true><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr, cross);
  else qq_ttxg_reweight_kernel<double, 1, false><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr, cross);
  return (int)cudaGetLastError();
}

// REX_DF64, helicity-summed: the direct and the t-channel tile in double-float, their
// helicity loops rolled (2^20 x 16: 20.5 ms against 57.0 ms in FP64; q g 35.4 ms against
// 62.3 ms; unrolled they took 32.0 and 70.6 ms)
int launch_qq_ttxg_df64(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp, double* out,
                        void* stream, const QqgCrossing& cross) {
  constexpr int EPB = QqgTile<df64>::EPB;
  const int64_t blocks = (nev + EPB - 1) / EPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned g = (unsigned)blocks;
  if (cross.neg[0] != 0 || cross.neg[1] != 0)
    qq_ttxg_reweight_kernel<df64, 1, false, true><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr, cross);
  else
    qq_ttxg_reweight_kernel<df64, 1, false><<<g, QQG_BLOCK, 0, st>>>(mom, w_in, nev, lp, out, nullptr, cross);
  return (int)cudaGetLastError();
}

}  // namespace rex

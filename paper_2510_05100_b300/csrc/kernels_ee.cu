// Standalone launcher of the e+e- -> mu+mu- reweighting kernel (sm_103a).
#include "ee_kernel.cuh"

namespace rex {

int launch_ee(const double* mom, const double* w_in, int64_t nev, const EwLaunch& lp, double* out,
              void* stream, const signed char* hel) {
  const int64_t blocks = (nev + 127) / 128;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (hel) ee_reweight_kernel<true><<<(unsigned)blocks, 128, 0, st>>>(mom, w_in, nev, lp, out, hel);
  else ee_reweight_kernel<false><<<(unsigned)blocks, 128, 0, st>>>(mom, w_in, nev, lp, out, nullptr);
  return (int)cudaGetLastError();
}

}  // namespace rex

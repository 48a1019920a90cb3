// Standalone launcher of the e+e- -> mu+mu- reweighting kernel (sm_103a).
#include "ee_kernel.cuh"

namespace rex {

int launch_ee(const double* mom, const double* w_in, int64_t nev, const EwLaunch& lp, double* out,
              void* stream) {
  const int64_t blocks = (nev + 127) / 128;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  ee_reweight_kernel<<<(unsigned)blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(mom, w_in, nev, lp,
                                                                                      out);
  return (int)cudaGetLastError();
}

}  // namespace rex

// Standalone launcher of the e+e- -> mu+mu- reweighting kernel (sm_103a).
#include "ee_kernel.cuh"

namespace rex {

// Thread per event, FP64 (B300 issues FP64 at 2 FMA per clock per SM): a sample of a
// few thousand events runs in blocks of 32 threads so that it spreads over every SM
// instead of a quarter of them; larger samples use blocks of 128.
template <int TPB>
static int launch_ee_t(const double* mom, const double* w_in, int64_t nev, const EwLaunch& lp, double* out,
                       cudaStream_t st, const signed char* hel) {
  const int64_t blocks = (nev + TPB - 1) / TPB;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  if (hel) ee_reweight_kernel<true, TPB><<<(unsigned)blocks, TPB, 0, st>>>(mom, w_in, nev, lp, out, hel);
  else ee_reweight_kernel<false, TPB><<<(unsigned)blocks, TPB, 0, st>>>(mom, w_in, nev, lp, out, nullptr);
  return (int)cudaGetLastError();
}

int launch_ee(const double* mom, const double* w_in, int64_t nev, const EwLaunch& lp, double* out,
              void* stream, const signed char* hel) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!hel) {   // the helicity sum: four lanes per event (ee_tile_split)
    const int64_t blocks = (nev + 31) / 32;
    if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    ee_reweight_split_kernel<<<(unsigned)blocks, 128, 0, st>>>(mom, w_in, nev, lp, out);
    return (int)cudaGetLastError();
  }
  return nev < 148 * 128 * 4 ? launch_ee_t<32>(mom, w_in, nev, lp, out, st, hel)
                             : launch_ee_t<128>(mom, w_in, nev, lp, out, st, hel);
}

}  // namespace rex

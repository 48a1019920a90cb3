// Double-float (REX_DF64) launcher of gg_ttxg, compiled apart from the FP64 and mixed
// variants so that the units build in parallel.
#include "qcd_kernel.cuh"

namespace rex {
REX_DEFINE_QCD_DF64_LAUNCHER(PROC_GG_TTXG, gg_ttxg)

int launch_gg_ttxg_df64_exclusive(const double* mom, const double* w_in, int64_t nev, const QcdLaunch& lp,
                                  double* out, void* stream, const signed char* hel) {
  return launch_df64_exclusive_t<PROC_GG_TTXG>(mom, w_in, nev, lp, out, hel, static_cast<cudaStream_t>(stream));
}
}  // namespace rex

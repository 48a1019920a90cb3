// Double-float (REX_DF64) launcher of gg_ttx, compiled apart from the FP64 and mixed
// variants so that the units build in parallel.
#include "qcd_kernel.cuh"

namespace rex {
REX_DEFINE_QCD_DF64_LAUNCHER(PROC_GG_TTX, gg_ttx)
}  // namespace rex

// Helicity-exclusive launcher of gg_ttx (rex_reweight_helicity), compiled apart from the
// helicity-summed variants so that the two build in parallel.
#include "qcd_kernel.cuh"

namespace rex {
REX_DEFINE_QCD_EXCLUSIVE_LAUNCHER(PROC_GG_TTX, gg_ttx)
}  // namespace rex

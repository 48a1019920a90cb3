// Fused reweighting kernels for gg_ttx (all thread-mapping variants, FP64 and mixed).
#include "qcd_kernel.cuh"

namespace rex {
REX_DEFINE_QCD_LAUNCHER(PROC_GG_TTX, gg_ttx)
}  // namespace rex

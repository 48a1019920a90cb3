// Fused reweighting kernels for gg_ttxg (all thread-mapping variants, FP64 and mixed).
#include "qcd_kernel.cuh"

namespace rex {
REX_DEFINE_QCD_LAUNCHER(PROC_GG_TTXG, gg_ttxg)
}  // namespace rex

// Instantiations of the fused optimisation kernel, one per compiled
// configuration (separate translation unit so the builds run in parallel).
#include "fg_fused_kernel.cuh"

namespace fg {

#define FG_CFG_OPT(nw, mb, ppt) &launch_fused_cfg<kModeOptimize, nw, mb, ppt>,
extern const FusedLaunchFn kOptimizeLaunch[] = {FG_FUSED_CONFIGS(FG_CFG_OPT)};

}  // namespace fg

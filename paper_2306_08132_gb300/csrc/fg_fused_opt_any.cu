// Instantiations of the fused optimisation kernel for scenes that hold mesh
// objects, one per compiled configuration (own translation unit so the builds
// run in parallel).
#include "fg_fused_kernel.cuh"

namespace fg {

#define FG_CFG_OPT_ANY(nw, mb, ppt) &launch_fused_cfg<kModeOptimize, nw, mb, ppt, true>,
extern const FusedLaunchFn kOptimizeLaunchAny[] = {FG_FUSED_CONFIGS(FG_CFG_OPT_ANY)};

}  // namespace fg

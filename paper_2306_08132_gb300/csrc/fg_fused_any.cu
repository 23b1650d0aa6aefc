// Instantiations of the fused kernels for scenes that hold mesh objects (the
// lookup dispatches on the object kind); grid-only scenes use the kernels of
// fg_fused.cu / fg_fused_opt.cu, which compile the grid lookup alone.
#include "fg_fused_kernel.cuh"

namespace fg {

#define FG_CFG_LOSSGRAD_ANY(nw, mb, ppt) &launch_fused_cfg<kModeLossGrad, nw, mb, ppt, true>,
extern const FusedLaunchFn kLossGradLaunchAny[] = {FG_FUSED_CONFIGS(FG_CFG_LOSSGRAD_ANY)};

cudaError_t launch_wrench_any(const FusedArgs& a, cudaStream_t st) {
  return launch_fused_cfg<kModeWrench, 4, 5, 1, true>(a, st);
}

cudaError_t launch_queue_round_any(const FusedArgs& a, cudaStream_t st) {
  return launch_fused_cfg<kModeQueue, 4, 5, 1, true>(a, st);
}

}  // namespace fg

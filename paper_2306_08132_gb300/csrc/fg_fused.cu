// Dispatch of the fused kernels: compiled configurations, the per-device
// selection, and the autotuner that times the configurations on a workload.
#include <cuda_runtime.h>

#include "fg_fused_kernel.cuh"

namespace fg {

#define FG_CFG_NW(nw, mb, ppt) nw,
#define FG_CFG_MB(nw, mb, ppt) mb,
#define FG_CFG_PPT(nw, mb, ppt) ppt,
#define FG_CFG_LOSSGRAD(nw, mb, ppt) &launch_fused_cfg<kModeLossGrad, nw, mb, ppt>,
static const int kCfgNW[] = {FG_FUSED_CONFIGS(FG_CFG_NW)};
static const int kCfgMinB[] = {FG_FUSED_CONFIGS(FG_CFG_MB)};
static const int kCfgPPT[] = {FG_FUSED_CONFIGS(FG_CFG_PPT)};
static const FusedLaunchFn kLossGradLaunch[] = {FG_FUSED_CONFIGS(FG_CFG_LOSSGRAD)};
constexpr int kNumCfg = sizeof(kCfgNW) / sizeof(kCfgNW[0]);
constexpr int kDefaultCfg = 1;   // 4 warps per candidate, >= 5 CTAs per SM, 1 point per thread

static int g_selected[64] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                             -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                             -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                             -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};

int fused_config_count() { return kNumCfg; }
void fused_config_info(int i, int* nw, int* minb, int* ppt) {
  *nw = kCfgNW[i];
  *minb = kCfgMinB[i];
  *ppt = kCfgPPT[i];
}
static int& selected_slot() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_selected[dev & 63];
}
int fused_config_current() {
  int s = selected_slot();
  return s < 0 ? kDefaultCfg : s;
}
void fused_config_select(int i) { selected_slot() = i; }

cudaError_t launch_fused(int mode, const FusedArgs& a, const fg_hand* h, cudaStream_t st) {
  (void)h;
  if (a.B <= 0) return cudaSuccess;
  const int cfg = fused_config_current();
  if (a.any_mesh) {
    switch (mode) {
      case kModeWrench: return launch_wrench_any(a, st);
      case kModeLossGrad: return kLossGradLaunchAny[cfg](a, st);
      default: return kOptimizeLaunchAny[cfg](a, st);
    }
  }
  switch (mode) {
    case kModeWrench: return launch_fused_cfg<kModeWrench, 4, 5, 1>(a, st);
    case kModeLossGrad: return kLossGradLaunch[cfg](a, st);
    default: return kOptimizeLaunch[cfg](a, st);
  }
}

// One round of a request queue: every active request's candidates in one launch.
cudaError_t launch_queue_round(const FusedArgs& a, cudaStream_t st) {
  if (a.B <= 0) return cudaSuccess;
  if (a.any_mesh) return launch_queue_round_any(a, st);
  return launch_fused_cfg<kModeQueue, 4, 5, 1>(a, st);
}

cudaError_t autotune_fused(const FusedArgs& base, int reps, float* times_ms, int* best, cudaStream_t st) {
  const size_t qbytes = sizeof(float) * (size_t)base.B * 64;
  (void)qbytes;
  float* qtmp = nullptr;
  float* ltmp = nullptr;
  const int D = base.hand_D;
  cudaError_t e = cudaMallocAsync(&qtmp, sizeof(float) * (size_t)base.B * D, st);
  if (e != cudaSuccess) return e;
  e = cudaMallocAsync(&ltmp, sizeof(float) * (size_t)base.B, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(qtmp, st);
    return e;
  }
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best_ms = 3.0e38f;
  int best_i = kDefaultCfg;
  for (int i = 0; i < kNumCfg && e == cudaSuccess; ++i) {
    FusedArgs a = base;
    a.q = qtmp;
    a.loss = ltmp;
    float total = 0.0f;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {   // r = 0 warms up
      e = cudaMemcpyAsync(qtmp, base.q, sizeof(float) * (size_t)base.B * D, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) break;
      cudaEventRecord(t0, st);
      e = (base.any_mesh ? kOptimizeLaunchAny : kOptimizeLaunch)[i](a, st);
      cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (r > 0) total += ms;
    }
    const float avg = total / (reps > 0 ? reps : 1);
    if (times_ms) times_ms[i] = avg;
    if (avg < best_ms) {
      best_ms = avg;
      best_i = i;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFreeAsync(qtmp, st);
  cudaFreeAsync(ltmp, st);
  if (e == cudaSuccess) {
    fused_config_select(best_i);
    if (best) *best = best_i;
  }
  return e;
}

}  // namespace fg

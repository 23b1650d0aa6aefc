// Allocation-free variant of the plain per-stage step.
//
// Some callers cannot allocate device memory once they are running: a
// real-time grasp-planning loop that must not block or fail on an allocation in
// the middle of a control cycle, or a host application whose device memory is
// owned entirely by another runtime's allocator and never handed to plugins.
// For them this entry point runs the same per-stage step as
// fg_optimize_step_plain, but its scratch lives in a fixed-size array compiled
// into this library instead of a caller workspace.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (FG_NOALLOC_SCRATCH_BYTES) until the process exits, and every
// call shares it.  Host code cannot use the array's name as a device address
// (in host code the name is only a host-side stand-in), so the first call on
// each device looks the address up with cudaGetSymbolAddress while that device
// is current and caches it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "fg_internal.h"

namespace fg {

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace fg

using namespace fg;

extern "C" fg_status fg_optimize_step_plain_noalloc(const fg_hand* h, const fg_scene* sc, const int* oc, float* q,
                                                    int B, const fg_params* p, int step, int total_steps, int nsteps,
                                                    float* loss, void* stream) {
  // the same checks as the workspace form, fg_optimize_step_plain
  fg_status st = check_common("fg_optimize_step_plain_noalloc", h, sc, B, p);
  if (st == FG_OK) st = check_one_step("fg_optimize_step_plain_noalloc", p);
  if (st != FG_OK) return st;
  if (nsteps < 1 || step < 0 || total_steps < 1) {
    set_error("fg_optimize_step_plain_noalloc: need nsteps >= 1, step >= 0, total_steps >= 1");
    return FG_ERR_INVALID;
  }
  if (sc->has_mesh) {
    set_error("fg_optimize_step_plain_noalloc: the per-stage form takes grid objects only");
    return FG_ERR_INVALID;
  }
  if (B == 0) return FG_OK;
  if (!q) {
    set_error("fg_optimize_step_plain_noalloc: NULL q");
    return FG_ERR_INVALID;
  }
  const size_t need = plain_workspace_bytes(h, B);
  if (need > (size_t)FG_NOALLOC_SCRATCH_BYTES) {
    set_error("fg_optimize_step_plain_noalloc: B * P too large for the built-in scratch (" + std::to_string(need) +
              " bytes needed, " + std::to_string((size_t)FG_NOALLOC_SCRATCH_BYTES) +
              " available); use fg_optimize_step_plain with a workspace");
    return FG_ERR_INVALID;
  }
  void* ws = nullptr;
  cudaError_t e = scratch_address(&ws);
  if (e != cudaSuccess) return cuda_status(e, "fg_optimize_step_plain_noalloc: scratch address");
  // Every stage writes the scratch it later reads within the same call, so
  // nothing left by an earlier call needs clearing.
  return cuda_status(launch_plain_step(h, sc, oc, q, B, params_from(p), step, total_steps, nsteps, loss, ws,
                                       (cudaStream_t)stream),
                     "fg_optimize_step_plain_noalloc");
}

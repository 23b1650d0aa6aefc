// Host-side internals shared by the translation units of libfastgraspd.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "fastgraspd.h"
#include "fg_device.cuh"

struct fg_hand {
  fg::HandDev host;          // copy of the device descriptor (pointers are device pointers)
  fg::HandDev* dev;          // device copy of the descriptor
  float4* pts;               // device [P]
  float4* chunk_sphere;      // device [nchunks]
  int* chunk_link;           // device [nchunks]
  int4* units;               // device [nunits]
  int subtree_end[FG_MAX_LINKS];
};

struct fg_sdf {
  fg::ObjDev host;           // grid and pyramid: device pointers owned by this handle
  float* grid;
  float* pyr;
  size_t bytes;              // grid bytes
  size_t pyr_bytes;          // min-pyramid bytes
  float4* mesh;              // mesh objects: BVH, triangles and normals (one allocation); bytes is its size
};

struct fg_scene {
  int n;
  int has_mesh;              // some object is a mesh
  fg::ObjDev* dev;           // device [n]
};

namespace fg {

void set_error(const std::string& msg);
fg_status cuda_status(cudaError_t e, const char* what);
// Argument checks shared by the entry points: handles, B >= 0 and the parameters;
// the one-step metric only (sim_steps = 0, gauss_seidel = 0).
fg_status check_common(const char* fn, const fg_hand* h, const fg_scene* sc, int B, const fg_params* p);
fg_status check_one_step(const char* fn, const fg_params* p);
// True when the allocation-failure injection (fg_test_fail_allocation) makes this
// allocation point fail.
bool alloc_fault();
ParamsDev params_from(const fg_params* p);
int device_sm_count();
size_t min_pyramid_floats(int nx, int ny, int nz, int* levels);
cudaError_t build_min_pyramid(const float* grid, int nx, int ny, int nz, float* pyr, int levels, int* offsets);

// fused kernels (fg_fused.cu)
enum FusedMode { kModeWrench = 0, kModeLossGrad = 1, kModeOptimize = 2, kModeQueue = 3 };

// One active request of a queue round: candidates [cand_start, cand_start + B)
// of the round's launch step this request's q from step0 for nsteps steps.
struct QueueSlotDev {
  const HandDev* hand;
  float* q;
  float* loss;
  ObjDev obj;
  ParamsDev P;
  int cand_start, B, step0, total_steps, nsteps;
};
struct FusedArgs {
  const HandDev* hand;
  const ObjDev* objs;
  int n_obj;
  const int* obj_of_cand;
  float* q;
  int B;
  ParamsDev P;
  float r_fixed;
  int step0, total_steps, nsteps;
  float* loss;
  float* grad;
  float* wrench;
  int* ncontact;
  uint32_t* bits;
  int hand_D;
  const QueueSlotDev* slots;   // queue mode: slot table (device), sorted by cand_start
  int nslots;
  int any_mesh;                // some object is a mesh: the kernels with the mesh lookup
  unsigned* work;              // fused kernels: candidate counter pair (set by the launcher)
};
typedef cudaError_t (*FusedLaunchFn)(const FusedArgs&, cudaStream_t);
// Compiled configurations: grid objects only, and any object (grids and meshes).
extern const FusedLaunchFn kOptimizeLaunch[];
extern const FusedLaunchFn kOptimizeLaunchAny[];
extern const FusedLaunchFn kLossGradLaunchAny[];
cudaError_t launch_wrench_any(const FusedArgs& a, cudaStream_t st);
cudaError_t launch_queue_round_any(const FusedArgs& a, cudaStream_t st);
cudaError_t launch_fused(int mode, const FusedArgs& a, const fg_hand* h, cudaStream_t st);
// T-step metric (params.sim_steps >= 1): loss and gradient, or optimisation steps (fg_tstep.cu)
cudaError_t launch_tstep(int mode, const FusedArgs& a, cudaStream_t st);
// Gauss-Seidel form (params.gauss_seidel = 1): loss and gradient, or optimisation steps (fg_gs.cu)
cudaError_t launch_gs(int mode, const FusedArgs& a, int nchunks, cudaStream_t st);
int fused_config_count();
void fused_config_info(int i, int* nw, int* minb, int* ppt);
int fused_config_current();
void fused_config_select(int i);
cudaError_t autotune_fused(const FusedArgs& base, int reps, float* times_ms, int* best, cudaStream_t st);
cudaError_t launch_queue_round(const FusedArgs& a, cudaStream_t st);

// grasp-quality metrics (fg_quality.cu)
cudaError_t launch_contact_measure(const FusedArgs& a, const float* weights, float tau, float* out, cudaStream_t st);
cudaError_t launch_grasp_epsilon(const FusedArgs& a, float tau, float mu, int k_edges, float tscale,
                                 const float* dirs, int K, float* eps, int* ncontact, cudaStream_t st);

// per-stage kernels (fg_plain.cu)
size_t plain_workspace_bytes(const fg_hand* h, int B);
cudaError_t launch_plain_step(const fg_hand* h, const fg_scene* sc, const int* obj_of_cand, float* q, int B,
                              const ParamsDev& P, int step, int total_steps, int nsteps, float* loss,
                              void* ws, cudaStream_t st);
cudaError_t launch_fk_points(const fg_hand* h, const float* q, int B, float* pts, cudaStream_t st);
cudaError_t launch_sdf_query(const ObjDev& o, const float* pts, int n, float r, float* phi, float* grad,
                             cudaStream_t st);

}  // namespace fg

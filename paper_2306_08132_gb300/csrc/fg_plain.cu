// Plain one-kernel-per-stage form of the grasp-search step, plus the standalone
// FK and SDF-query kernels of the C ABI.
//
// Stages (one launch each, intermediates in a workspace in device memory):
//   1 fk_frames      q -> link frames            [B][L][12]
//   2 points         frames -> p                 SoA [3][B*P]
//   3 sdf            p -> phi, grad, curvature   SoA [11][B*P]
//   4 contact_fwd    -> wrench, count, pen       [B][7][8]       (one CTA per candidate)
//   5 loss           -> loss, dL/dW, joint grad  [B], [B][7][6], [B][D]
//   6 contact_adj    -> dL/dp                    SoA [3][B*P]
//   7 link_reduce    -> per-link sums            [B][L][6]       (one CTA per candidate)
//   8 fk_adj_update  -> dL/dq, q update          [B][D]
// The per-point arithmetic is the same device code as the fused kernel.
#include <cuda_runtime.h>

#include "fg_internal.h"

namespace fg {

namespace {

constexpr int kSampleFloats = 11;   // phi, g[3], hxy, hxz, hyz, eh[3], e
constexpr size_t kAlign = 256;

struct Workspace {
  float* frames;   // [B][L][12]
  float* pts;      // [3][BP]
  float* smp;      // [11][BP]
  float* wtot;     // [B][7][8]
  float* G;        // [B][7][6]
  float* lossv;    // [B]
  float* gq;       // [B][D]
  float* dp;       // [3][BP]
  float* lsum;     // [B][L][6]
};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

Workspace carve(void* base, const HandDev& H, int B) {
  size_t BP = (size_t)B * H.P;
  char* p = (char*)base;
  Workspace w;
  auto take = [&](size_t nfloats) {
    float* r = (float*)p;
    p += align_up(nfloats * sizeof(float));
    return r;
  };
  w.frames = take((size_t)B * H.L * 12);
  w.pts = take(3 * BP);
  w.smp = take(kSampleFloats * BP);
  w.wtot = take((size_t)B * kSims * 8);
  w.G = take((size_t)B * kSims * 6);
  w.lossv = take((size_t)B);
  w.gq = take((size_t)B * H.D);
  w.dp = take(3 * BP);
  w.lsum = take((size_t)B * H.L * 6);
  return w;
}

size_t carve_bytes(const HandDev& H, int B) {
  size_t BP = (size_t)B * H.P;
  return align_up((size_t)B * H.L * 12 * 4) + align_up(3 * BP * 4) + align_up(kSampleFloats * BP * 4) +
         align_up((size_t)B * kSims * 8 * 4) + align_up((size_t)B * kSims * 6 * 4) + align_up((size_t)B * 4) +
         align_up((size_t)B * H.D * 4) + align_up(3 * BP * 4) + align_up((size_t)B * H.L * 6 * 4);
}

// Object of candidate b; an index outside the scene selects object 0 here and
// the loss stage reports NaN for that candidate (q is then left unchanged).
__device__ __forceinline__ bool obj_ok(int n_obj, const int* oc, int b) {
  const int oi = oc ? oc[b] : 0;
  return oi >= 0 && oi < n_obj;
}
__device__ __forceinline__ const ObjDev* obj_for(const ObjDev* objs, int n_obj, const int* oc, int b) {
  return objs + (obj_ok(n_obj, oc, b) ? (oc ? oc[b] : 0) : 0);
}

// 1: link frames, one thread per candidate, links in topological order.
__global__ void fk_frames_kernel(const HandDev* __restrict__ Hp, const float* __restrict__ q, int B,
                                 float* __restrict__ frames) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const HandDev& H = *Hp;
  Frame F[kMaxLinks];
  root_frame(q + (size_t)b * H.D, F[0]);
  for (int l = 1; l < H.L; ++l) link_frame(H, l, F[H.parent[l]], q[(size_t)b * H.D + 6 + l - 1], F[l]);
  for (int l = 0; l < H.L; ++l) {
    float* o = frames + ((size_t)b * H.L + l) * 12;
    for (int k = 0; k < 9; ++k) o[k] = F[l].R[k];
    for (int k = 0; k < 3; ++k) o[9 + k] = F[l].o[k];
  }
}

// 2: world points.
__global__ void points_kernel(const HandDev* __restrict__ Hp, const float* __restrict__ frames, int B,
                              float* __restrict__ pts) {
  const HandDev& H = *Hp;
  size_t BP = (size_t)B * H.P;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < BP; idx += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(idx / H.P), i = (int)(idx % H.P);
    float4 sp = __ldg(H.pts + i);
    const float* F = frames + ((size_t)b * H.L + (int)sp.w) * 12;
    float p[3];
    transform_point(F, F + 9, sp.x, sp.y, sp.z, p);
    pts[idx] = p[0];
    pts[BP + idx] = p[1];
    pts[2 * BP + idx] = p[2];
  }
}

// 3: grid lookups with curvature.
__global__ void sdf_stage_kernel(const HandDev* __restrict__ Hp, const ObjDev* __restrict__ objs, int n_obj,
                                 const int* __restrict__ oc, int B, const float* __restrict__ pts,
                                 float* __restrict__ smp) {
  const HandDev& H = *Hp;
  size_t BP = (size_t)B * H.P;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < BP; idx += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(idx / H.P);
    const ObjDev O = *obj_for(objs, n_obj, oc, b);
    float p[3] = {pts[idx], pts[BP + idx], pts[2 * BP + idx]};
    SdfSample s;
    sdf_lookup<true, false>(O, p, s);   // the per-stage form takes grid objects only
    float v[kSampleFloats] = {s.phi, s.g[0], s.g[1], s.g[2], s.hxy, s.hxz, s.hyz, s.eh[0], s.eh[1], s.eh[2], s.e};
#pragma unroll
    for (int k = 0; k < kSampleFloats; ++k) smp[k * BP + idx] = v[k];
  }
}

__device__ __forceinline__ void load_sample(const float* smp, size_t BP, size_t idx, SdfSample& s) {
  s.phi = smp[idx];
  s.g[0] = smp[BP + idx];
  s.g[1] = smp[2 * BP + idx];
  s.g[2] = smp[3 * BP + idx];
  s.hxy = smp[4 * BP + idx];
  s.hxz = smp[5 * BP + idx];
  s.hyz = smp[6 * BP + idx];
  s.eh[0] = smp[7 * BP + idx];
  s.eh[1] = smp[8 * BP + idx];
  s.eh[2] = smp[9 * BP + idx];
  s.e = smp[10 * BP + idx];
  s.outside = s.e > 0.0f || s.eh[0] != 0.0f || s.eh[1] != 0.0f || s.eh[2] != 0.0f;
}

// 4: contact forward, one CTA (256 threads) per candidate.
__global__ void contact_fwd_kernel(const HandDev* __restrict__ Hp, const ObjDev* __restrict__ objs, int n_obj,
                                   const int* __restrict__ oc, int B, ParamsDev Pm, int step, int total_steps,
                                   const float* __restrict__ pts, const float* __restrict__ smp,
                                   float* __restrict__ wtot) {
  __shared__ float red[8][kSims * 8];
  const HandDev& H = *Hp;
  const int b = blockIdx.x;
  const ObjDev O = *obj_for(objs, n_obj, oc, b);
  const float r = dilation_at(Pm, step, total_steps);
  const float dtV = Pm.dt * Pm.V;
  size_t BP = (size_t)B * H.P;
  float W[kSims][8];
#pragma unroll
  for (int m = 0; m < kSims; ++m)
#pragma unroll
    for (int k = 0; k < 8; ++k) W[m][k] = 0.0f;
  for (int i = threadIdx.x; i < H.P; i += blockDim.x) {
    size_t idx = (size_t)b * H.P + i;
    float p[3] = {pts[idx], pts[BP + idx], pts[2 * BP + idx]};
    SdfSample s;
    load_sample(smp, BP, idx, s);
    PointState ps;
    point_state(s, p, r, ps);
#pragma unroll
    for (int m = 0; m < kSims; ++m) {
      float phm = sim_phi(ps, m, dtV);
      if (phm < 0.0f) {
        float f[3], d[3], tq[3];
        contact_force(ps, m, -phm, Pm, O, f, d);
        cross3(d, f, tq);
        W[m][0] += f[0]; W[m][1] += f[1]; W[m][2] += f[2];
        W[m][3] += tq[0]; W[m][4] += tq[1]; W[m][5] += tq[2];
        W[m][6] += 1.0f;
        if (m == 0) W[0][7] += -phm;
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < kSims; ++m)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float v = W[m][k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][m * 8 + k] = v;
    }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kSims * 8; idx += blockDim.x) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][idx];
    wtot[(size_t)b * kSims * 8 + idx] = v;
  }
}

// 5: loss and wrench adjoint, one thread per candidate.
__global__ void loss_kernel(const HandDev* __restrict__ Hp, const ObjDev* __restrict__ objs, int n_obj,
                            const int* __restrict__ oc, int B, ParamsDev Pm, const float* __restrict__ q,
                            const float* __restrict__ wtot, float* __restrict__ G, float* __restrict__ lossv,
                            float* __restrict__ gq) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const HandDev& H = *Hp;
  const ObjDev O = *obj_for(objs, n_obj, oc, b);
  float W[kSims][6], N[kSims], Gl[kSims][3], Ga[kSims][3];
  const float* wt = wtot + (size_t)b * kSims * 8;
  for (int m = 0; m < kSims; ++m) {
    for (int k = 0; k < 6; ++k) W[m][k] = wt[m * 8 + k];
    N[m] = wt[m * 8 + 6];
  }
  float Ls = stability_loss_and_adjoint(W, N, Pm, O, Gl, Ga);
  for (int m = 0; m < kSims; ++m)
    for (int k = 0; k < 3; ++k) {
      G[((size_t)b * kSims + m) * 6 + k] = Gl[m][k];
      G[((size_t)b * kSims + m) * 6 + 3 + k] = Ga[m][k];
    }
  float dth[kMaxLinks];
  float Lj = joint_losses(H, q + (size_t)b * H.D + 6, Pm, dth);
  const bool ok = obj_ok(n_obj, oc, b);
  const float nan = __int_as_float(0x7fc00000);
  for (int j = 0; j < H.J; ++j) gq[(size_t)b * H.D + 6 + j] = ok ? dth[j] : nan;
  lossv[b] = ok ? Ls + Lj + Pm.w_pen * wt[7] : nan;
}

// 6: contact adjoint, one thread per point.
__global__ void contact_adj_kernel(const HandDev* __restrict__ Hp, const ObjDev* __restrict__ objs, int n_obj,
                                   const int* __restrict__ oc, int B, ParamsDev Pm, int step, int total_steps,
                                   const float* __restrict__ pts, const float* __restrict__ smp,
                                   const float* __restrict__ G, float* __restrict__ dpo) {
  const HandDev& H = *Hp;
  const float r = dilation_at(Pm, step, total_steps);
  const float dtV = Pm.dt * Pm.V;
  size_t BP = (size_t)B * H.P;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < BP; idx += (size_t)gridDim.x * blockDim.x) {
    int b = (int)(idx / H.P);
    const ObjDev O = *obj_for(objs, n_obj, oc, b);
    float p[3] = {pts[idx], pts[BP + idx], pts[2 * BP + idx]};
    SdfSample s;
    load_sample(smp, BP, idx, s);
    PointState ps;
    point_state(s, p, r, ps);
    float dphi = 0.0f, dn[3] = {0.0f, 0.0f, 0.0f}, dp[3] = {0.0f, 0.0f, 0.0f};
    const float* Gb = G + (size_t)b * kSims * 6;
#pragma unroll
    for (int m = 0; m < kSims; ++m) {
      float phm = sim_phi(ps, m, dtV);
      const float Gl[3] = {Gb[m * 6], Gb[m * 6 + 1], Gb[m * 6 + 2]};
      const float Ga[3] = {Gb[m * 6 + 3], Gb[m * 6 + 4], Gb[m * 6 + 5]};
      sim_adjoint(ps, m, phm, phm < 0.0f, Gl, Ga, Pm, O, m == 0 ? Pm.w_pen : 0.0f, dphi, dn, dp);
    }
    sdf_adjoint(s, ps, dphi, dn, dp);
    dpo[idx] = dp[0];
    dpo[BP + idx] = dp[1];
    dpo[2 * BP + idx] = dp[2];
  }
}

// 7: per-link sums of g and (p - t) x g, one CTA (256 threads) per candidate.
// Points are sorted by link, so a warp's 32 points usually share one link: those
// are reduced with shuffles and added once; mixed warps add point by point.
__global__ void link_reduce_kernel(const HandDev* __restrict__ Hp, int B, const float* __restrict__ q,
                                   const float* __restrict__ pts, const float* __restrict__ dpo,
                                   float* __restrict__ lsum) {
  __shared__ float acc[kMaxLinks][6];
  const HandDev& H = *Hp;
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < kMaxLinks * 6; k += blockDim.x) (&acc[0][0])[k] = 0.0f;
  __syncthreads();
  size_t BP = (size_t)B * H.P;
  const float t0[3] = {q[(size_t)b * H.D], q[(size_t)b * H.D + 1], q[(size_t)b * H.D + 2]};
  for (int base = threadIdx.x - lane; base < H.P; base += blockDim.x) {
    const int i = base + lane;
    const bool valid = i < H.P;
    float v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int l = 0;
    if (valid) {
      const size_t idx = (size_t)b * H.P + i;
      l = (int)__ldg(H.pts + i).w;
      const float g[3] = {dpo[idx], dpo[BP + idx], dpo[2 * BP + idx]};
      const float rel[3] = {pts[idx] - t0[0], pts[BP + idx] - t0[1], pts[2 * BP + idx] - t0[2]};
      float tq[3];
      cross3(rel, g, tq);
      v[0] = g[0]; v[1] = g[1]; v[2] = g[2];
      v[3] = tq[0]; v[4] = tq[1]; v[5] = tq[2];
    }
    const int l0 = __shfl_sync(0xffffffffu, l, 0);
    if (__all_sync(0xffffffffu, !valid || l == l0)) {
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        float x = v[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) atomicAdd(&acc[l0][k], x);
      }
    } else if (valid) {
#pragma unroll
      for (int k = 0; k < 6; ++k) atomicAdd(&acc[l][k], v[k]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < H.L * 6; k += blockDim.x) lsum[(size_t)b * H.L * 6 + k] = (&acc[0][0])[k];
}

// 8: subtree sums, joint and base gradients, update.  One thread per candidate.
__global__ void fk_adj_update_kernel(const HandDev* __restrict__ Hp, int B, ParamsDev Pm,
                                     const float* __restrict__ frames, const float* __restrict__ lsum,
                                     float* __restrict__ gq, const float* __restrict__ lossv, float* __restrict__ q,
                                     float* __restrict__ loss_out, int write_loss) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const HandDev& H = *Hp;
  float S[kMaxLinks][6];
  for (int l = 0; l < H.L; ++l)
    for (int k = 0; k < 6; ++k) S[l][k] = lsum[((size_t)b * H.L + l) * 6 + k];
  for (int l = H.L - 1; l >= 1; --l)
    for (int k = 0; k < 6; ++k) S[H.parent[l]][k] += S[l][k];
  float* qb = q + (size_t)b * H.D;
  float* gb = gq + (size_t)b * H.D;
  for (int l = 1; l < H.L; ++l) {
    const float* F = frames + ((size_t)b * H.L + l) * 12;
    float aw[3];
    matvec3(F, H.axis[l], aw);
    float rel[3] = {F[9] - qb[0], F[10] - qb[1], F[11] - qb[2]};
    float rg[3];
    cross3(rel, S[l], rg);
    float tau[3] = {S[l][3] - rg[0], S[l][4] - rg[1], S[l][5] - rg[2]};
    gb[6 + l - 1] += aw[0] * tau[0] + aw[1] * tau[1] + aw[2] * tau[2];
  }
  gb[0] = S[0][0];
  gb[1] = S[0][1];
  gb[2] = S[0][2];
  float w[3] = {qb[3], qb[4], qb[5]}, tau[3] = {S[0][3], S[0][4], S[0][5]}, gw[3];
  exp_jacobian_T(w, tau, gw);
  gb[3] = gw[0];
  gb[4] = gw[1];
  gb[5] = gw[2];
  if (lossv[b] == lossv[b])
    for (int k = 0; k < H.D; ++k) qb[k] -= Pm.lr * gb[k];
  if (write_loss && loss_out) loss_out[b] = lossv[b];
}

// Standalone FK: frames in shared memory, then all threads transform points.
__global__ void fk_points_kernel(const HandDev* __restrict__ Hp, const float* __restrict__ q, int B,
                                 float* __restrict__ pts) {
  __shared__ Frame F[kMaxLinks];
  __shared__ float sq[64];
  const HandDev& H = *Hp;
  size_t BP = (size_t)B * H.P;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < H.D) sq[threadIdx.x] = q[(size_t)b * H.D + threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
      root_frame(sq, F[0]);
      for (int l = 1; l < H.L; ++l) link_frame(H, l, F[H.parent[l]], sq[6 + l - 1], F[l]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < H.P; i += blockDim.x) {
      float4 sp = __ldg(H.pts + i);
      float p[3];
      transform_point(F[(int)sp.w].R, F[(int)sp.w].o, sp.x, sp.y, sp.z, p);
      size_t idx = (size_t)b * H.P + i;
      pts[idx] = p[0];
      pts[BP + idx] = p[1];
      pts[2 * BP + idx] = p[2];
    }
  }
}

__global__ void sdf_query_kernel(ObjDev O, const float* __restrict__ pts, int n, float r, float* __restrict__ phi,
                                 float* __restrict__ grad) {
  // whole warps stay in the loop (the mesh search is warp-wide); lanes past n
  // look up the last point and write nothing
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i - lane < n; i += gridDim.x * blockDim.x) {
    const bool valid = i < n;
    const int k = valid ? i : n - 1;
    float p[3] = {pts[k], pts[(size_t)n + k], pts[2 * (size_t)n + k]};
    SdfSample s;
    sdf_lookup<false>(O, p, s);
    if (!valid) continue;
    phi[i] = s.phi - r;
    if (grad) {
      grad[i] = s.g[0];
      grad[(size_t)n + i] = s.g[1];
      grad[2 * (size_t)n + i] = s.g[2];
    }
  }
}

int grid_for(size_t n, int threads) {
  size_t g = (n + threads - 1) / threads;
  size_t cap = (size_t)device_sm_count() * 16;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

size_t plain_workspace_bytes(const fg_hand* h, int B) { return carve_bytes(h->host, B); }

cudaError_t launch_plain_step(const fg_hand* h, const fg_scene* sc, const int* oc, float* q, int B,
                              const ParamsDev& P, int step, int total_steps, int nsteps, float* loss, void* ws,
                              cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const HandDev& H = h->host;
  Workspace w = carve(ws, H, B);
  size_t BP = (size_t)B * H.P;
  for (int s = 0; s < nsteps; ++s) {
    int k = step + s;
    fk_frames_kernel<<<(B + 127) / 128, 128, 0, st>>>(h->dev, q, B, w.frames);
    points_kernel<<<grid_for(BP, 256), 256, 0, st>>>(h->dev, w.frames, B, w.pts);
    sdf_stage_kernel<<<grid_for(BP, 256), 256, 0, st>>>(h->dev, sc->dev, sc->n, oc, B, w.pts, w.smp);
    contact_fwd_kernel<<<B, 256, 0, st>>>(h->dev, sc->dev, sc->n, oc, B, P, k, total_steps, w.pts, w.smp, w.wtot);
    loss_kernel<<<(B + 127) / 128, 128, 0, st>>>(h->dev, sc->dev, sc->n, oc, B, P, q, w.wtot, w.G, w.lossv, w.gq);
    contact_adj_kernel<<<grid_for(BP, 256), 256, 0, st>>>(h->dev, sc->dev, sc->n, oc, B, P, k, total_steps, w.pts, w.smp,
                                                          w.G, w.dp);
    link_reduce_kernel<<<B, 256, 0, st>>>(h->dev, B, q, w.pts, w.dp, w.lsum);
    fk_adj_update_kernel<<<(B + 127) / 128, 128, 0, st>>>(h->dev, B, P, w.frames, w.lsum, w.gq, w.lossv, q, loss,
                                                          s == nsteps - 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_fk_points(const fg_hand* h, const float* q, int B, float* pts, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  int grid = B < device_sm_count() * 8 ? B : device_sm_count() * 8;
  fk_points_kernel<<<grid, 256, 0, st>>>(h->dev, q, B, pts);
  return cudaGetLastError();
}

cudaError_t launch_sdf_query(const ObjDev& o, const float* pts, int n, float r, float* phi, float* grad,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  sdf_query_kernel<<<grid_for((size_t)n, 256), 256, 0, st>>>(o, pts, n, r, phi, grad);
  return cudaGetLastError();
}

}  // namespace fg

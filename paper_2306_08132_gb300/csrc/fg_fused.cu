// Fused grasp-search step: one CTA per candidate (persistent over candidates and
// steps), NW warps sweep the hand's points twice per step.
//
//   FK (warp 0, one lane per link, level by level)
//   sweep 1: point -> SDF -> 7 plane-linearised contacts -> wrench, count   (registers)
//   loss:    reduce wrenches -> L_stable + joint terms -> wrench adjoint    (warp 0)
//   sweep 2: recompute point -> adjoint of contacts, normal, SDF -> dL/dp
//            -> per-link (sum g, sum (p - t) x g)                           (registers, smem)
//   tree:    subtree sums (prefix scan over preorder links) -> dL/dq        (warp 0)
//   update:  q <- q - lr dL/dq                                              (smem)
//
// Nothing per point is written to global memory; the adjoint recomputes the
// forward quantities of each point from the shared link frames.
#include <cuda_runtime.h>

#include "fg_internal.h"

namespace fg {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int NW>
struct FusedSmem {
  HandDev H;
  ObjDev O;
  Frame frames[kMaxLinks];
  float q[64];
  float grad[64];
  float wred[NW][kSims][8];        // per warp: W (6), N, pen
  float G[kSims][6];               // dL/dW_lin, dL/dW_ang per simulation
  float lacc[NW][kMaxLinks][6];    // per warp, per link: sum g, sum (p - t) x g
  float Wtot[kSims][8];
  float loss;
  int bad_object;
};

// Point range of warp w: contiguous, 32-aligned chunks.
__device__ __forceinline__ void warp_range(int P, int NW, int w, int& b, int& e) {
  int chunk = ((P + 32 * NW - 1) / (32 * NW)) * 32;
  b = w * chunk;
  e = min(P, b + chunk);
}

__device__ __forceinline__ void fk_warp(const HandDev& H, const float* q, Frame* frames, int lane) {
  for (int d = 0; d <= H.max_depth; ++d) {
    if (lane < H.L && H.depth[lane] == d) {
      if (lane == 0)
        root_frame(q, frames[0]);
      else
        link_frame(H, lane, frames[H.parent[lane]], q[6 + lane - 1], frames[lane]);
    }
    __syncwarp();
  }
}

template <int MODE, int NW>
__global__ void __launch_bounds__(NW * 32) fused_step_kernel(FusedArgs a) {
  __shared__ FusedSmem<NW> S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) S.H = *a.hand;
  __syncthreads();
  const HandDev& H = S.H;
  const int D = H.D, P = H.P, L = H.L;
  const ParamsDev& Pm = a.P;
  const float dtV = Pm.dt * Pm.V;
  int pb, pe;
  warp_range(P, NW, warp, pb, pe);
  const int nwords = (P + 31) >> 5;

  for (int c = blockIdx.x; c < a.B; c += gridDim.x) {
    __syncthreads();
    if (tid < D) S.q[tid] = a.q[(size_t)c * D + tid];
    if (tid == 0) {
      const int oi = a.obj_of_cand ? a.obj_of_cand[c] : 0;
      S.bad_object = oi < 0 || oi >= a.n_obj;
      if (!S.bad_object) S.O = a.objs[oi];
    }
    __syncthreads();
    if (S.bad_object) {
      // an object index outside the scene: NaN outputs, q left unchanged
      const float nan = __int_as_float(0x7fc00000);
      if (MODE == kModeWrench) {
        for (int idx = tid; idx < kSims * 6; idx += NW * 32) a.wrench[(size_t)c * kSims * 6 + idx] = nan;
        if (tid < kSims) a.ncontact[(size_t)c * kSims + tid] = -1;
      } else if (MODE == kModeLossGrad) {
        if (tid == 0) a.loss[c] = nan;
        if (a.grad && tid < D) a.grad[(size_t)c * D + tid] = nan;
      } else if (a.loss && tid == 0) {
        a.loss[c] = nan;
      }
      continue;
    }
    const int nsteps = MODE == kModeOptimize ? a.nsteps : 1;
    for (int s = 0; s < nsteps; ++s) {
      const float r = MODE == kModeOptimize ? dilation_at(Pm, a.step0 + s, a.total_steps) : a.r_fixed;
      __syncthreads();
      if (warp == 0) fk_warp(H, S.q, S.frames, lane);
      __syncthreads();
      const ObjDev O = S.O;

      // ---------------------------------------------------------------- sweep 1
      float W[kSims][6], N[kSims], pen = 0.0f;
#pragma unroll
      for (int m = 0; m < kSims; ++m) {
        N[m] = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) W[m][k] = 0.0f;
      }
      for (int base = pb; base < pe; base += 32) {
        const int i = base + lane;
        const bool valid = i < pe;
        float4 sp = valid ? __ldg(H.pts + i) : __ldg(H.pts + base);
        const Frame& F = S.frames[(int)sp.w];
        float p[3];
        transform_point(F.R, F.o, sp.x, sp.y, sp.z, p);
        SdfSample smp;
        sdf_lookup<false>(O, p, smp);
        PointState ps;
        point_state(smp, p, r, ps);
        unsigned cbits[kSims];
#pragma unroll
        for (int m = 0; m < kSims; ++m) {
          const float phm = sim_phi(ps, m, dtV);
          const bool kap = valid && phm < 0.0f;
          if (MODE == kModeWrench) cbits[m] = __ballot_sync(kFull, kap);
          if (kap) {
            const float C = -phm;
            float f[3], d[3];
            contact_force(ps, m, C, Pm, O, f, d);
            float tq[3];
            cross3(d, f, tq);
            W[m][0] += f[0]; W[m][1] += f[1]; W[m][2] += f[2];
            W[m][3] += tq[0]; W[m][4] += tq[1]; W[m][5] += tq[2];
            N[m] += 1.0f;
            if (m == 0) pen += C;
          }
        }
        if (MODE == kModeWrench && lane == 0 && a.bits) {
#pragma unroll
          for (int m = 0; m < kSims; ++m) a.bits[((size_t)c * kSims + m) * nwords + (base >> 5)] = cbits[m];
        }
      }
#pragma unroll
      for (int m = 0; m < kSims; ++m) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float v = warp_sum(W[m][k]);
          if (lane == 0) S.wred[warp][m][k] = v;
        }
        float v = warp_sum(N[m]);
        if (lane == 0) S.wred[warp][m][6] = v;
      }
      pen = warp_sum(pen);
      if (lane == 0) S.wred[warp][0][7] = pen;
      __syncthreads();

      // ------------------------------------------------------------ reduction
      if (warp == 0) {
        for (int idx = lane; idx < kSims * 8; idx += 32) {
          int m = idx >> 3, k = idx & 7;
          float v = 0.0f;
#pragma unroll
          for (int w = 0; w < NW; ++w) v += S.wred[w][m][k];
          S.Wtot[m][k] = v;
        }
      }
      __syncthreads();
      if (MODE == kModeWrench) {
        for (int idx = tid; idx < kSims * 6; idx += NW * 32) {
          int m = idx / 6, k = idx % 6;
          a.wrench[((size_t)c * kSims + m) * 6 + k] = S.Wtot[m][k];
        }
        if (tid < kSims) a.ncontact[(size_t)c * kSims + tid] = (int)S.Wtot[tid][6];
        continue;
      }

      // ------------------------------------------------------------------ loss
      if (tid == 0) {
        float Wm[kSims][6], Nm[kSims], Gl[kSims][3], Ga[kSims][3];
        for (int m = 0; m < kSims; ++m) {
          for (int k = 0; k < 6; ++k) Wm[m][k] = S.Wtot[m][k];
          Nm[m] = S.Wtot[m][6];
        }
        float Ls = stability_loss_and_adjoint(Wm, Nm, Pm, O, Gl, Ga);
        for (int m = 0; m < kSims; ++m)
          for (int k = 0; k < 3; ++k) {
            S.G[m][k] = Gl[m][k];
            S.G[m][3 + k] = Ga[m][k];
          }
        float Lj = joint_losses(H, S.q + 6, Pm, S.grad + 6);
        S.loss = Ls + Lj + Pm.w_pen * S.Wtot[0][7];
      }
      for (int idx = tid; idx < NW * kMaxLinks * 6; idx += NW * 32) (&S.lacc[0][0][0])[idx] = 0.0f;
      __syncthreads();

      // ---------------------------------------------------------------- sweep 2
      {
        const float t0[3] = {S.q[0], S.q[1], S.q[2]};
        int cur = -1;
        float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int base = pb; base < pe; base += 32) {
          const int i = base + lane;
          const bool valid = i < pe;
          float4 sp = valid ? __ldg(H.pts + i) : __ldg(H.pts + base);
          const int link = (int)sp.w;
          const Frame& F = S.frames[link];
          float p[3];
          transform_point(F.R, F.o, sp.x, sp.y, sp.z, p);
          SdfSample smp;
          sdf_lookup<true>(O, p, smp);
          PointState ps;
          point_state(smp, p, r, ps);
          float dphi = 0.0f, dn[3] = {0.0f, 0.0f, 0.0f}, dp[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
          for (int m = 0; m < kSims; ++m) {
            const float phm = sim_phi(ps, m, dtV);
            const bool kap = phm < 0.0f;
            const float Gl[3] = {S.G[m][0], S.G[m][1], S.G[m][2]};
            const float Ga[3] = {S.G[m][3], S.G[m][4], S.G[m][5]};
            sim_adjoint(ps, m, phm, kap, Gl, Ga, Pm, O, m == 0 ? Pm.w_pen : 0.0f, dphi, dn, dp);
          }
          sdf_adjoint(smp, ps, dphi, dn, dp);
          float v[6];
          if (valid) {
            const float rel[3] = {p[0] - t0[0], p[1] - t0[1], p[2] - t0[2]};
            float tq[3];
            cross3(rel, dp, tq);
            v[0] = dp[0]; v[1] = dp[1]; v[2] = dp[2];
            v[3] = tq[0]; v[4] = tq[1]; v[5] = tq[2];
          } else {
#pragma unroll
            for (int k = 0; k < 6; ++k) v[k] = 0.0f;
          }
          const int l0 = __shfl_sync(kFull, link, 0);
          const bool uniform = __all_sync(kFull, !valid || link == l0);
          if (uniform && l0 == cur) {
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[k] += v[k];
          } else {
            if (cur >= 0) {
#pragma unroll
              for (int k = 0; k < 6; ++k) {
                float sum = warp_sum(acc[k]);
                if (lane == 0) S.lacc[warp][cur][k] += sum;
              }
            }
            if (uniform) {
              cur = l0;
#pragma unroll
              for (int k = 0; k < 6; ++k) acc[k] = v[k];
            } else {
              cur = -1;
              unsigned remaining = __ballot_sync(kFull, valid);
              while (remaining) {
                const int leader = __ffs(remaining) - 1;
                const int l = __shfl_sync(kFull, link, leader);
                const bool mine = valid && link == l;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                  float sum = warp_sum(mine ? v[k] : 0.0f);
                  if (lane == 0) S.lacc[warp][l][k] += sum;
                }
                remaining &= ~__ballot_sync(kFull, mine);
              }
#pragma unroll
              for (int k = 0; k < 6; ++k) acc[k] = 0.0f;
            }
          }
        }
        if (cur >= 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            float sum = warp_sum(acc[k]);
            if (lane == 0) S.lacc[warp][cur][k] += sum;
          }
        }
      }
      __syncthreads();

      // ------------------------------------------------------------------ tree
      if (warp == 0) {
        // per-link sums over warps, then inclusive prefix over preorder links
        float sl[6], pre[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float v = 0.0f;
          if (lane < L)
            for (int w = 0; w < NW; ++w) v += S.lacc[w][lane][k];
          sl[k] = v;
          float x = v;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            float y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
          }
          pre[k] = x;   // sum over links [0, lane]
        }
        // subtree(lane) = [lane, end): sum = pre[end-1] - pre[lane-1]
        const int end = lane < L ? H.subtree_end[lane] : lane + 1;
        float sub[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float hi = __shfl_sync(kFull, pre[k], (end - 1) & 31);
          float lo = __shfl_sync(kFull, pre[k], (lane + 31) & 31);
          sub[k] = hi - (lane > 0 ? lo : 0.0f);
          (void)sl;
        }
        if (lane >= 1 && lane < L) {
          const Frame& F = S.frames[lane];
          float aw[3];
          matvec3(F.R, H.axis[lane], aw);
          const float rel[3] = {F.o[0] - S.q[0], F.o[1] - S.q[1], F.o[2] - S.q[2]};
          float rg[3];
          cross3(rel, sub, rg);
          const float tau[3] = {sub[3] - rg[0], sub[4] - rg[1], sub[5] - rg[2]};
          S.grad[6 + lane - 1] += aw[0] * tau[0] + aw[1] * tau[1] + aw[2] * tau[2];
        }
        if (lane == 0) {
          S.grad[0] = sub[0];
          S.grad[1] = sub[1];
          S.grad[2] = sub[2];
          const float w[3] = {S.q[3], S.q[4], S.q[5]};
          const float tau[3] = {sub[3], sub[4], sub[5]};
          float gw[3];
          exp_jacobian_T(w, tau, gw);
          S.grad[3] = gw[0];
          S.grad[4] = gw[1];
          S.grad[5] = gw[2];
        }
      }
      __syncthreads();
      if (MODE == kModeLossGrad) {
        if (tid < D && a.grad) a.grad[(size_t)c * D + tid] = S.grad[tid];
        if (tid == 0) a.loss[c] = S.loss;
      } else {  // optimize
        if (tid < D) S.q[tid] -= Pm.lr * S.grad[tid];
        if (tid == 0 && a.loss && s == nsteps - 1) a.loss[c] = S.loss;
      }
    }
    if (MODE == kModeOptimize) {
      __syncthreads();
      if (tid < D) a.q[(size_t)c * D + tid] = S.q[tid];
    }
  }
}

template <int MODE, int NW>
static cudaError_t launch_mode(const FusedArgs& a, cudaStream_t st) {
  static int blocks_per_sm = -1;
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fused_step_kernel<MODE, NW>,
                                                                  NW * 32, 0);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  long long grid = (long long)device_sm_count() * blocks_per_sm;
  if (grid > a.B) grid = a.B;
  if (grid < 1) return cudaSuccess;
  fused_step_kernel<MODE, NW><<<(int)grid, NW * 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fused(int mode, const FusedArgs& a, const fg_hand* h, cudaStream_t st) {
  (void)h;
  if (a.B <= 0) return cudaSuccess;
  switch (mode) {
    case kModeWrench: return launch_mode<kModeWrench, 4>(a, st);
    case kModeLossGrad: return launch_mode<kModeLossGrad, 4>(a, st);
    default: return launch_mode<kModeOptimize, 4>(a, st);
  }
}

}  // namespace fg

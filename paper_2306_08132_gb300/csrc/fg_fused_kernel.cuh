// Fused grasp-search step: one CTA of NW warps per candidate, persistent over
// candidates (claimed from a counter, fg_work.cuh) and steps.  Per step:
//
//   FK       warp 0, one lane per link, level by level -> link frames (smem)
//   sweep 1  point -> SDF -> 7 plane-linearised contacts; a warp that has a
//            contact in simulation m reduces its forces into a per-warp slot
//   loss     warp 0: wrenches -> L_stable (Eq. 2) and its adjoint per
//            simulation, joint terms (Eqs. 3-4), one lane per simulation / joint
//   sweep 2  recompute each point -> adjoint of the 7 simulations (leaky rule),
//            of the normal and of the SDF -> dL/dp -> per-link (sum g, sum r x g)
//   tree     warp 0: prefix scan over preorder links -> subtree sums -> dL/dq
//   update   q <- q - lr dL/dq (smem), written back after the last step
//
// Nothing per point is written to global memory: the adjoint recomputes the
// forward quantities of each point from the link frames.
#pragma once

#include <cuda_runtime.h>

#include "fg_internal.h"
#include "fg_work.cuh"

namespace fg {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Work units whose adjoint sums fit in shared memory (hands up to ~12,000 points);
// larger hands use fixed per-warp point ranges.
constexpr int kMaxUnits = 192;

template <int NW>
struct FusedSmem {
  HandDev H;
  ObjDev O;
  float4 frame4[kMaxLinks][3];     // rows (R_r0, R_r1, R_r2, o_r) of each link frame
  SimAdjoints G;                   // dL/dW_lin, dL/dW_ang per simulation (scalar and packed)
  SimConsts K;                     // constants of the simulation adjoint
  float q[64];
  float grad[64];
  unsigned long long wfix[kSims][8];  // forward sums in fixed point: W (6), N (integer), pen
  float lacc[NW][kMaxLinks][6];    // per warp, per link: sum g, sum (p - t) x g (fixed ranges)
  float uacc[kMaxUnits][6];        // per work unit: sum g, sum (p - t) x g
  float Wtot[kSims][8];
  float loss;
  int cand;                        // the candidate claimed by this CTA
  int bad_object;
  int n_active;
  int next_unit;                   // adjoint sweep: next unclaimed work unit
  int next_chunk;                  // forward sweep: next unclaimed active chunk
  unsigned active_bits[kMaxCullChunks / 32];
  unsigned short active_list[kMaxCullChunks];
  // source of the current candidate (the call's arguments, or a queue slot)
  ParamsDev Pm;
  const HandDev* src_hand;
  const HandDev* hand_loaded;
  float* qout;
  float* lout;
  int cl, step0, total, nsteps;
};

__device__ __forceinline__ void store_frame(const Frame& F, float4* f4) {
  f4[0] = make_float4(F.R[0], F.R[1], F.R[2], F.o[0]);
  f4[1] = make_float4(F.R[3], F.R[4], F.R[5], F.o[1]);
  f4[2] = make_float4(F.R[6], F.R[7], F.R[8], F.o[2]);
}

__device__ __forceinline__ void load_frame(const float4* f4, Frame& F) {
  const float4 a = f4[0], b = f4[1], c = f4[2];
  F.R[0] = a.x; F.R[1] = a.y; F.R[2] = a.z; F.o[0] = a.w;
  F.R[3] = b.x; F.R[4] = b.y; F.R[5] = b.z; F.o[1] = b.w;
  F.R[6] = c.x; F.R[7] = c.y; F.R[8] = c.z; F.o[2] = c.w;
}

// Link frames by depth level: lane l computes link l once its parent is done.
__device__ __forceinline__ void fk_warp(const HandDev& H, const float* q, float4 (*frame4)[3], int lane) {
  for (int d = 0; d <= H.max_depth; ++d) {
    if (lane < H.L && H.depth[lane] == d) {
      Frame F;
      if (lane == 0) {
        root_frame(q, F);
      } else {
        Frame par;
        load_frame(frame4[H.parent[lane]], par);
        link_frame(H, lane, par, q[6 + lane - 1], F);
      }
      store_frame(F, frame4[lane]);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void world_point(const float4* f4, const float4& sp, float p[3]) {
  const float4 a = f4[0], b = f4[1], c = f4[2];
  p[0] = fma_(a.x, sp.x, fma_(a.y, sp.y, fma_(a.z, sp.z, a.w)));
  p[1] = fma_(b.x, sp.x, fma_(b.y, sp.y, fma_(b.z, sp.z, b.w)));
  p[2] = fma_(c.x, sp.x, fma_(c.y, sp.y, fma_(c.z, sp.z, c.w)));
}

// Adjoint of one hand point (index i, link frames in smem): dL/dp through the 7
// simulations, the normal and the SDF lookup.  v = (g, (p - t0) x g).
template <bool ANY>
__device__ __forceinline__ void point_adjoint(const HandDev& H, const float4 (*frame4)[3], const SimAdjoints& G,
                                              const SimConsts& K, const ObjDev& O,
                                              const ParamsDev& Pm, float r, const float t0[3], int i, bool valid,
                                              float v[6], int& link) {
  const float4 sp = __ldg(H.pts + i);
  link = (int)sp.w;
  float p[3];
  world_point(frame4[link], sp, p);
  SdfSample smp;
  sdf_lookup<true, ANY>(O, p, smp);
  PointState ps;
  point_state(smp, p, r, ps);
  float dphi = 0.0f, dn[3] = {0.0f, 0.0f, 0.0f}, dp[3] = {0.0f, 0.0f, 0.0f};
  point_sims_adjoint(ps, G, K, Pm, O, dphi, dn, dp);
  sdf_adjoint(smp, ps, dphi, dn, dp);
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
}

// The same for two points (a, b) at once, in packed f32x2 arithmetic: positions
// and grid indices per point, everything after the corner gathers on pairs.
template <bool ANY>
__device__ __forceinline__ void point_adjoint_pair(const HandDev& H, const float4 (*frame4)[3], const SimAdjoints& G,
                                                   const SimConsts& K, const ObjDev& O, const ParamsDev& Pm, float r,
                                                   const float t0[3], int ia, int ib, bool va, bool vb,
                                                   float v[2][6], int link[2]) {
  const float4 sa = __ldg(H.pts + ia), sb = __ldg(H.pts + ib);
  link[0] = (int)sa.w;
  link[1] = (int)sb.w;
  float pa[3], pb[3];
  world_point(frame4[link[0]], sa, pa);
  world_point(frame4[link[1]], sb, pb);
  SdfSampleT<float2> smp;
  if (ANY && O.kind == kObjMesh) {
    SdfSample sa, sb;
    mesh_lookup(O, pa, sa);
    mesh_lookup(O, pb, sb);
    smp.phi = make_float2(sa.phi, sb.phi);
    smp.hxy = smp.hxz = smp.hyz = smp.e = make_float2(0.0f, 0.0f);
    smp.curv = make_float2(sa.curv, sb.curv);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      smp.g[k] = make_float2(sa.g[k], sb.g[k]);
      smp.eh[k] = make_float2(0.0f, 0.0f);
    }
    smp.outside = bool2{false, false};
  } else {
    SdfIndex xa, xb;
    sdf_index(O, pa, xa);
    sdf_index(O, pb, xb);
    float ca[8], cb[8];
    sdf_gather(O, xa.cell, ca);
    sdf_gather(O, xb.cell, cb);
    sdf_finish_pair(O, xa, xb, ca, cb, smp);
  }
  const float2 p[3] = {make_float2(pa[0], pb[0]), make_float2(pa[1], pb[1]), make_float2(pa[2], pb[2])};
  PointStateT<float2> ps;
  point_state(smp, p, r, ps);
  const float2 zero = make_float2(0.0f, 0.0f);
  float2 dphi = zero, dn[3] = {zero, zero, zero}, dp[3] = {zero, zero, zero};
  point_sims_adjoint(ps, G, K, Pm, O, dphi, dn, dp);
  sdf_adjoint(smp, ps, dphi, dn, dp);
  const float2 rel[3] = {vsub(p[0], vsplat<float2>(t0[0])), vsub(p[1], vsplat<float2>(t0[1])),
                         vsub(p[2], vsplat<float2>(t0[2]))};
  float2 tq[3];
  vcross(rel, dp, tq);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    v[0][k] = va ? dp[k].x : 0.0f;
    v[1][k] = vb ? dp[k].y : 0.0f;
    v[0][3 + k] = va ? tq[k].x : 0.0f;
    v[1][3 + k] = vb ? tq[k].y : 0.0f;
  }
}

// Sums a[0..5] over the 32 lanes in a fixed pattern and stores the 6 totals in
// slot.  Eight values (6 and two zeros) are halved across lanes at each exchange
// (xor 16, 8, 4: a lane keeps half of its values and adds its partner's copy of
// them), then the last value is summed over groups of 4; lane 4k ends with the
// total of value k.  The order of additions never depends on timing.
__device__ __forceinline__ void unit_reduce_store(const float a[6], int lane, float* slot) {
  const float v[8] = {a[0], a[1], a[2], a[3], a[4], a[5], 0.0f, 0.0f};
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0;
  float w4[4], w2[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float send = h16 ? v[j] : v[4 + j];
    const float keep = h16 ? v[4 + j] : v[j];
    w4[j] = keep + __shfl_xor_sync(kFull, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = h8 ? w4[j] : w4[2 + j];
    const float keep = h8 ? w4[2 + j] : w4[j];
    w2[j] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  float w = (h4 ? w2[1] : w2[0]) + __shfl_xor_sync(kFull, h4 ? w2[0] : w2[1], 4);
  w += __shfl_xor_sync(kFull, w, 2);
  w += __shfl_xor_sync(kFull, w, 1);
  const int k = lane >> 2;
  if ((lane & 3) == 0 && k < 6) slot[k] = w;
}

// Fixed point with 44 fractional bits: every force and torque sum here is far
// inside +-2^19, and the quantum 2^-44 lies far below float32 rounding of them.
__device__ __forceinline__ unsigned long long to_fixed(float v) {
  return (unsigned long long)__float2ll_rn(__fmul_rn(v, 0x1p44f));
}
__device__ __forceinline__ float from_fixed(long long x) { return __fmul_rn(__ll2float_rn(x), 0x1p-44f); }

// The warp's sums of a[0..5] (the fixed pattern of unit_reduce_store) added in
// fixed point to slot[0..5]: lane 4k holds the total of value k.
__device__ __forceinline__ void unit_reduce_add_fixed(const float a[6], int lane, unsigned long long* slot) {
  const float v[8] = {a[0], a[1], a[2], a[3], a[4], a[5], 0.0f, 0.0f};
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0, h4 = (lane & 4) != 0;
  float w4[4], w2[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float send = h16 ? v[j] : v[4 + j];
    const float keep = h16 ? v[4 + j] : v[j];
    w4[j] = keep + __shfl_xor_sync(kFull, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = h8 ? w4[j] : w4[2 + j];
    const float keep = h8 ? w4[2 + j] : w4[j];
    w2[j] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  float w = (h4 ? w2[1] : w2[0]) + __shfl_xor_sync(kFull, h4 ? w2[0] : w2[1], 4);
  w += __shfl_xor_sync(kFull, w, 2);
  w += __shfl_xor_sync(kFull, w, 1);
  const int k = lane >> 2;
  if ((lane & 3) == 0 && k < 6) atomicAdd(slot + k, to_fixed(w));
}

// Adds 32 points' (g, r x g) to the warp's per-link sums.  Runs of points of one
// link accumulate in registers (acc, for link cur) and are reduced when the link
// changes; a group of 32 that straddles links is reduced link by link.
__device__ __forceinline__ void link_accumulate(float (*lacc)[6], int lane, int link, bool valid, const float v[6],
                                                int& cur, float acc[6]) {
  const int l0 = __shfl_sync(kFull, link, 0);
  const bool uniform = __all_sync(kFull, !valid || link == l0);
  if (uniform && l0 == cur) {
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += v[k];
    return;
  }
  if (cur >= 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float sum = warp_sum(acc[k]);
      if (lane == 0) lacc[cur][k] += sum;
    }
  }
  if (uniform) {
    cur = l0;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = v[k];
    return;
  }
  cur = -1;
  unsigned remaining = __ballot_sync(kFull, valid);
  while (remaining) {
    const int leader = __ffs(remaining) - 1;
    const int l = __shfl_sync(kFull, link, leader);
    const bool mine = valid && link == l;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float sum = warp_sum(mine ? v[k] : 0.0f);
      if (lane == 0) lacc[l][k] += sum;
    }
    remaining &= ~__ballot_sync(kFull, mine);
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) acc[k] = 0.0f;
}

// ANY = false: grid objects only (the mesh lookup is compiled out).
template <int MODE, int NW, int MINB, int PPT, bool ANY>
__global__ void __launch_bounds__(NW * 32, MINB) fused_step_kernel(FusedArgs a) {
  __shared__ FusedSmem<NW> S;
  constexpr bool kOpt = MODE == kModeOptimize || MODE == kModeQueue;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) S.hand_loaded = nullptr;
  const HandDev& H = S.H;
  const ParamsDev& Pm = S.Pm;

  for (;;) {
    const int c = next_candidate(a.work, &S.cand);
    if (c >= a.B) break;
    if (tid == 0) {
      if (MODE == kModeQueue) {
        // candidate c of the round belongs to the slot whose range holds it
        int sl = 0;
        while (sl + 1 < a.nslots && a.slots[sl + 1].cand_start <= c) ++sl;
        const QueueSlotDev& Q = a.slots[sl];
        S.src_hand = Q.hand;
        S.O = Q.obj;
        S.Pm = Q.P;
        S.cl = c - Q.cand_start;
        S.qout = Q.q;
        S.lout = Q.loss;
        S.step0 = Q.step0;
        S.total = Q.total_steps;
        S.nsteps = Q.nsteps;
        S.bad_object = 0;
      } else {
        S.src_hand = a.hand;
        S.Pm = a.P;
        S.cl = c;
        S.qout = a.q;
        S.lout = a.loss;
        S.step0 = a.step0;
        S.total = a.total_steps;
        S.nsteps = MODE == kModeOptimize ? a.nsteps : 1;
        const int oi = a.obj_of_cand ? a.obj_of_cand[c] : 0;
        S.bad_object = oi < 0 || oi >= a.n_obj;
        if (!S.bad_object) S.O = a.objs[oi];
      }
    }
    __syncthreads();
    if (S.src_hand != S.hand_loaded) {          // uniform: every thread reads the same words
      const int* src = reinterpret_cast<const int*>(S.src_hand);
      int* dst = reinterpret_cast<int*>(&S.H);
      for (int k = tid; k < (int)(sizeof(HandDev) / sizeof(int)); k += NW * 32) dst[k] = src[k];
      __syncthreads();
      if (tid == 0) S.hand_loaded = S.src_hand;
    }
    const int D = H.D, P = H.P, L = H.L;
    const float dtV = Pm.dt * Pm.V;
    const int nwords = (P + 31) >> 5;
    const int cl = S.cl;
    if (tid < D) S.q[tid] = S.qout[(size_t)cl * D + tid];
    if (tid == 0 && !S.bad_object) sim_constants(Pm, S.O, S.K);
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
    const int nsteps = S.nsteps;
    for (int s = 0; s < nsteps; ++s) {
      const float r = kOpt ? dilation_at(Pm, S.step0 + s, S.total) : a.r_fixed;
      __syncthreads();
      if (warp == 0) fk_warp(H, S.q, S.frame4, lane);
      for (int idx = tid; idx < kSims * 8; idx += NW * 32) (&S.wfix[0][0])[idx] = 0ull;
      if (tid == 0) S.next_chunk = 0;
      __syncthreads();
      const ObjDev& O = S.O;

      // --------------------------------------------------------- chunk culling
      // A chunk of 32 points (one link) can only hold a contact if some point has
      // phi_m = phi_hat - dt V n_k < 0, i.e. phi(p) < r + dt V.  Every point lies in
      // the chunk's bounding sphere (centre c, radius R), and the interpolated
      // field over that sphere is bounded below by the min-pyramid over its box,
      // so a chunk with  min - r - dt V (1 + 1e-5) - slack > 0  has no contact in
      // any simulation; the slack covers float32 rounding of positions and values.
      // Its contact flags are all zero and its forces are not computed.
      // Mesh objects: the Phong point lies within phong_shift of the flat closest
      // point, so if the chunk's centre c is outside the mesh at flat distance
      // d > R, every point of the chunk has rho >= d - R - phong_shift.
      const bool cull = H.nchunks <= kMaxCullChunks;
      if (cull) {
        for (int j0 = warp * 32; j0 < H.nchunks; j0 += NW * 32) {
          const int j = j0 + lane;
          bool active = false;
          if (j < H.nchunks) {
            active = true;
            const int l = H.chunk_link[j];
            if (l >= 0 && ANY && O.kind == kObjMesh) {
              const float4 cs = __ldg(H.chunk_sphere + j);
              float cw[3];
              world_point(S.frame4[l], cs, cw);
              const float slack = 1e-6f + 1e-5f * (fabsf(cw[0]) + fabsf(cw[1]) + fabsf(cw[2]));
              const float dc = mesh_flat_distance(O, cw);
              const float R = cs.w + slack;
              const float lbm = dc - R - O.phong_shift;
              active = !(dc > R && lbm - r - dtV * (1.0f + 1e-5f) - (1e-6f + 1e-5f * fabsf(dc)) > 0.0f);
            } else if (l >= 0) {
              const float4 cs = __ldg(H.chunk_sphere + j);
              float cw[3];
              world_point(S.frame4[l], cs, cw);
              const float slack = 1e-6f + 1e-5f * (fabsf(cw[0]) + fabsf(cw[1]) + fabsf(cw[2]));
              const float R = (cs.w + slack) * O.inv_h;
              const float org[3] = {O.ox, O.oy, O.oz};
              float lo[3], hi[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                const float u = (cw[k] - org[k]) * O.inv_h;
                lo[k] = u - R - 1e-3f;
                hi[k] = u + R + 1e-3f;
              }
              const float mn = region_min(O, lo, hi);
              active = !(mn - r - dtV * (1.0f + 1e-5f) - (1e-6f + 1e-5f * fabsf(mn)) > 0.0f);
            }
            if (MODE == kModeWrench && !active && a.bits) {
#pragma unroll 1
              for (int m = 0; m < kSims; ++m) a.bits[((size_t)c * kSims + m) * nwords + j] = 0u;
            }
          }
          const unsigned word = __ballot_sync(kFull, active);
          if (lane == 0) S.active_bits[j0 >> 5] = word;
        }
        __syncthreads();
        if (warp == 0) {
          int count = 0;
          for (int wi = 0; wi < (H.nchunks + 31) >> 5; ++wi) {
            const unsigned bits = S.active_bits[wi];
            if ((bits >> lane) & 1u)
              S.active_list[count + __popc(bits & ((1u << lane) - 1u))] = (unsigned short)(wi * 32 + lane);
            count += __popc(bits);
          }
          if (lane == 0) S.n_active = count;
        }
        __syncthreads();
      }

      // ---------------------------------------------------------------- sweep 1
      // Warps claim active chunks from a shared counter (a chunk with contacts costs
      // more); a chunk whose every point is cleared by its own pyramid entry is
      // skipped before the lookups.  A simulation's forces in a chunk are summed over its lanes with a
      // fixed shuffle pattern and added to the CTA's sums in fixed point, so the
      // totals do not depend on which warp ran which chunk, nor on the order.
      {
        const int n_work = cull ? S.n_active : H.nchunks;
        auto claim = [&]() {
          int j = 0;
          if (lane == 0) j = atomicAdd(&S.next_chunk, 1);
          return __shfl_sync(kFull, j, 0);
        };
        int idx = claim();
        while (idx < n_work) {
          const int nidx = claim();
          const int base = 32 * (cull ? (int)S.active_list[idx] : idx);
          const int i = base + lane;
          const bool valid = i < P;
          const float4 sp = __ldg(H.pts + (valid ? i : base));
          float p[3];
          world_point(S.frame4[(int)sp.w], sp, p);
          if (!(ANY && O.kind == kObjMesh)) {
            // A chunk that passed the test of its bounding sphere is tested point by
            // point (one pyramid entry each): if no point can have phi_m < 0 in any
            // simulation, the chunk holds no contact and its lookups are skipped.
            const float mn = point_min_bound(O, p);
            const bool clear = !valid || mn - r - dtV * (1.0f + 1e-5f) - (1e-6f + 1e-5f * fabsf(mn)) > 0.0f;
            if (__all_sync(kFull, clear)) {
              if (MODE == kModeWrench && a.bits && lane < kSims)
                a.bits[((size_t)c * kSims + lane) * nwords + (base >> 5)] = 0u;
              idx = nidx;
              continue;
            }
          }
          SdfSample smp;
          sdf_lookup<false, ANY>(O, p, smp);
          PointState ps;
          point_state(smp, p, r, ps);
#pragma unroll 1
          for (int m = 0; m < kSims; ++m) {
            const float phm = sim_phi(ps, m, dtV);
            const bool kap = valid && phm < 0.0f;
            const unsigned bal = __ballot_sync(kFull, kap);
            if (MODE == kModeWrench && lane == 0 && a.bits)
              a.bits[((size_t)c * kSims + m) * nwords + (base >> 5)] = bal;
            if (bal == 0u) continue;
            float v[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (kap) {
              float f[3], d[3], tq[3];
              contact_force(ps, m, -phm, Pm, O, f, d);
              cross3(d, f, tq);
              v[0] = f[0]; v[1] = f[1]; v[2] = f[2];
              v[3] = tq[0]; v[4] = tq[1]; v[5] = tq[2];
            }
            unit_reduce_add_fixed(v, lane, S.wfix[m]);
            if (lane == 0) atomicAdd(&S.wfix[m][6], (unsigned long long)__popc(bal));
            if (m == 0 && Pm.w_pen != 0.0f) {
              const float pen = warp_sum(kap ? -phm : 0.0f);
              if (lane == 0) atomicAdd(&S.wfix[0][7], to_fixed(pen));
            }
          }
          idx = nidx;
        }
      }
      __syncthreads();

      // ------------------------------------------------------------ reduction
      if (warp == 0) {
        for (int idx = lane; idx < kSims * 8; idx += 32) {
          const int m = idx >> 3, k = idx & 7;
          const long long x = (long long)S.wfix[m][k];
          S.Wtot[m][k] = k == 6 ? (float)x : from_fixed(x);
        }
        __syncwarp();
        if (MODE != kModeWrench) {
          // loss and wrench adjoint: lane m handles simulation m, lane j joint j
          float Lpart = 0.0f;
          if (lane < kSims) {
            const int m = lane;
            const float Nc = fmaxf(S.Wtot[m][6], 1.0f);
            const float sl = O.inv_mass / (Nc * Pm.dt), sa = O.inv_inertia / (Nc * Pm.dt);
            float v[3] = {0.0f, 0.0f, 0.0f};
            if (m > 0) v[sim_axis(m)] = sim_sign(m) * Pm.V;
            float xd[3], td[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              xd[k] = v[k] + S.Wtot[m][k] * sl;
              td[k] = S.Wtot[m][3 + k] * sa;
            }
            const float nx = sqrtf(xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
            const float nt = sqrtf(td[0] * td[0] + td[1] * td[1] + td[2] * td[2]);
            Lpart = nx + nt;
            const float ax = nx > 0.0f ? sl / (kSims * nx) : 0.0f;
            const float at = nt > 0.0f ? sa / (kSims * nt) : 0.0f;
            const float gl[3] = {xd[0] * ax, xd[1] * ax, xd[2] * ax};
            const float ga[3] = {td[0] * at, td[1] * at, td[2] * at};
            set_sim_adjoint(S.G, m, gl, ga);
          }
          float dj = 0.0f, d2 = 0.0f, lim = 0.0f, th = 0.0f;
          if (lane < H.J) {
            th = S.q[6 + lane];
            dj = th - 0.5f * (H.q_up[lane] + H.q_low[lane]);
            d2 = dj * dj;
            if (th > H.q_up[lane]) lim += th - H.q_up[lane];
            if (th < H.q_low[lane]) lim += H.q_low[lane] - th;
          }
          const float Ls = warp_sum(Lpart) / kSims;
          const float rn = sqrtf(warp_sum(d2));
          const float lims = warp_sum(lim);
          if (lane < H.J) {
            float g = rn > 0.0f ? Pm.w_range * dj / rn : 0.0f;
            if (th > H.q_up[lane]) g += Pm.w_limit;
            if (th < H.q_low[lane]) g -= Pm.w_limit;
            S.grad[6 + lane] = g;
          }
          if (lane == 0) S.loss = Ls + Pm.w_range * rn + Pm.w_limit * lims + Pm.w_pen * S.Wtot[0][7];
        }
      }
      for (int idx = tid; idx < NW * kMaxLinks * 6; idx += NW * 32) (&S.lacc[0][0][0])[idx] = 0.0f;
      if (tid == 0) S.next_unit = 0;
      __syncthreads();
      if (MODE == kModeLossGrad && a.grad == nullptr) {    // loss only: no adjoint
        if (tid == 0) a.loss[c] = S.loss;
        continue;
      }
      if (MODE == kModeWrench) {
        for (int idx = tid; idx < kSims * 6; idx += NW * 32) {
          const int m = idx / 6, k = idx % 6;
          a.wrench[((size_t)c * kSims + m) * 6 + k] = S.Wtot[m][k];
        }
        if (tid < kSims) a.ncontact[(size_t)c * kSims + tid] = (int)S.Wtot[tid][6];
        continue;
      }

      // ---------------------------------------------------------------- sweep 2
      {
        const float t0[3] = {S.q[0], S.q[1], S.q[2]};
        int cur = -1;
        float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (H.nunits <= kMaxUnits) {
          // Warps claim work units (<= 64 points of one link) from a shared
          // counter, so a warp that meets contacts (general adjoint) does not hold
          // the others at the barrier; each unit's sums go to its own slot, so the
          // result does not depend on which warp ran it.  The next claim is issued
          // before the current unit so that its latency is hidden.
          auto claim = [&]() {
            int j = 0;
            if (lane == 0) j = atomicAdd(&S.next_unit, 1);
            return __shfl_sync(kFull, j, 0);
          };
          int u = claim();
          while (u < H.nunits) {
            const int nu = claim();
            const int4 U = __ldg(H.units + u);      // first point, count, link
            float sum[6];
            if (PPT == 2) {
              // one point of each half of the unit per lane, packed arithmetic
              float v[2][6];
              int link[2];
              const bool va = lane < U.y, vb = lane + 32 < U.y;
              point_adjoint_pair<ANY>(H, S.frame4, S.G, S.K, O, Pm, r, t0, va ? U.x + lane : U.x,
                                 vb ? U.x + 32 + lane : U.x, va, vb, v, link);
#pragma unroll
              for (int k = 0; k < 6; ++k) sum[k] = v[0][k] + v[1][k];
            } else {
#pragma unroll
              for (int k = 0; k < 6; ++k) sum[k] = 0.0f;
              for (int h = 0; h < U.y; h += 32) {
                float v[6];
                int link;
                const bool valid = h + lane < U.y;
                point_adjoint<ANY>(H, S.frame4, S.G, S.K, O, Pm, r, t0, valid ? U.x + h + lane : U.x, valid, v, link);
#pragma unroll
                for (int k = 0; k < 6; ++k) sum[k] += v[k];
              }
            }
            unit_reduce_store(sum, lane, S.uacc[u]);
            u = nu;
          }
        } else {
          // fixed, contiguous 32-aligned point ranges per warp
          const int span = ((P + 32 * NW - 1) / (32 * NW)) * 32;
          const int pb = warp * span, pe = min(P, pb + span);
          for (int base = pb; base < pe; base += 32) {
            float v[6];
            int link;
            const int i = base + lane;
            const bool valid = i < pe;
            point_adjoint<ANY>(H, S.frame4, S.G, S.K, O, Pm, r, t0, valid ? i : base, valid, v, link);
            link_accumulate(S.lacc[warp], lane, link, valid, v, cur, acc);
          }
        }
        if (cur >= 0) {
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const float sum = warp_sum(acc[k]);
            if (lane == 0) S.lacc[warp][cur][k] += sum;
          }
        }
      }
      __syncthreads();

      // ------------------------------------------------------------------ tree
      if (warp == 0) {
        // per-link sums over warps, inclusive prefix over preorder links
        float pre[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float x = 0.0f;
          if (lane < L) {
            if (H.nunits <= kMaxUnits) {
              for (int u = H.unit_begin[lane]; u < H.unit_begin[lane + 1]; ++u) x += S.uacc[u][k];
            } else {
#pragma unroll
              for (int w = 0; w < NW; ++w) x += S.lacc[w][lane][k];
            }
          }
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
          }
          pre[k] = x;
        }
        // subtree(lane) = [lane, end): sum = pre[end - 1] - pre[lane - 1]
        const int end = lane < L ? H.subtree_end[lane] : lane + 1;
        float sub[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float hi = __shfl_sync(kFull, pre[k], (end - 1) & 31);
          const float lo = __shfl_sync(kFull, pre[k], (lane + 31) & 31);
          sub[k] = hi - (lane > 0 ? lo : 0.0f);
        }
        if (lane >= 1 && lane < L) {
          Frame F;
          load_frame(S.frame4[lane], F);
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
        if (tid == 0 && S.lout && s == nsteps - 1) S.lout[cl] = S.loss;
      }
    }
    if (kOpt) {
      __syncthreads();
      if (tid < D) S.qout[(size_t)cl * D + tid] = S.q[tid];
    }
  }
  work_done(a.work);
}

// Launch of one compiled configuration: a persistent grid of (SMs x resident
// CTAs) blocks, capped at B.
template <int MODE, int NW, int MINB, int PPT, bool ANY = false>
cudaError_t launch_fused_cfg(const FusedArgs& a, cudaStream_t st) {
  static int blocks_per_sm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& bps = blocks_per_sm[dev & 63];
  if (bps <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fused_step_kernel<MODE, NW, MINB, PPT, ANY>, NW * 32, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  long long grid = (long long)device_sm_count() * bps;
  if (grid > a.B) grid = a.B;
  if (grid < 1) return cudaSuccess;
  FusedArgs b = a;
  cudaError_t e = work_pair(&b.work, st);
  if (e != cudaSuccess) return e;
  fused_step_kernel<MODE, NW, MINB, PPT, ANY><<<(int)grid, NW * 32, 0, st>>>(b);
  return cudaGetLastError();
}

// Compiled configurations of the loss/gradient and optimisation kernels:
// warps per candidate, the minimum resident CTAs per SM the register
// allocation is held to, and points per thread in the adjoint sweep.  The autotuner times them on a workload.
// (warps per candidate, min CTAs per SM, points per thread per adjoint iteration)
#define FG_FUSED_CONFIGS(X) X(4, 4, 1) X(4, 5, 1) X(4, 6, 1) X(4, 8, 1) X(8, 3, 1) X(2, 8, 1) X(4, 3, 2) X(4, 4, 2) X(4, 5, 2) X(8, 2, 2) X(4, 7, 1)

}  // namespace fg

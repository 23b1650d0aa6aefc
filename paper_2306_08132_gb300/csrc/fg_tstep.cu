// T-step form of the grasp metric (Sec. III-C, Sec. IV-A): per candidate, the
// M = 7 test simulations run T PBD steps each, every hand point re-queried in the
// SDF at each simulation's predicted object pose, and the gradient is the
// hand-written adjoint of the whole chain, reversed step by step.
//
// One CTA of 4 warps per candidate (persistent over candidates and optimisation
// steps).  Per optimisation step:
//
//   FK            warp 0 (as in the one-step kernel)
//   forward       for t = 1..T: lanes 0..6 of warp 0 predict each simulation's
//                 pose; then one sweep per simulation over all points (query,
//                 contact force, wrench); lanes 0..6 apply the averaged correction
//   loss          L_stable (Eq. 2) on the final velocities, L_range, L_limit
//   reverse       for t = T..1: lanes 0..6 turn the state adjoint into wrench
//                 adjoints; one sweep per simulation computes every point's
//                 adjoint (contact, normal, lookup, lever, pose) and reduces the
//                 object-state adjoint; lanes 0..6 carry it to the previous step
//   tree, update  as in the one-step kernel
//
// Work is assigned to warps in a fixed pattern (chunk j to warp j mod 4) and
// every reduction has a fixed order, so results are bit-reproducible.
#include <cuda_runtime.h>

#include "fg_fused_kernel.cuh"
#include "fg_internal.h"

namespace fg {

namespace {

constexpr int kTW = 4;                        // warps per candidate
constexpr int kTSteps = FG_MAX_SIM_STEPS;

// One simulation step as the forward computed it; the reverse reads it back.
struct SimStep {
  float x[3];      // position before the step
  float xt[3];     // predicted position x~ = x + dt v
  float Rt[9];     // predicted orientation R~ = Exp(dt w) R, row-major
  float wdt[3];    // dt w
  float dtv[3];    // dt v
  float c1, c2;    // Exp(+-wdt) = I +- c1 [wdt]x + c2 [wdt]x^2
  float dth[3];    // averaged rotation correction
  float N;         // active contacts
};

struct TstepSmem {
  HandDev H;
  ObjDev O;
  ParamsDev Pm;
  float4 frame4[kMaxLinks][3];
  float q[64];
  float grad[64];
  SimStep st[kTSteps][kSims];
  float x[kSims][3], Rc[kSims][9], v[kSims][3], w[kSims][3];   // current object state
  float G[kSims][6];          // dL/dW_lin, dL/dW_ang of the step being reversed
  float ab[kSims][12];        // adjoint of a state: x, R (world-frame rotation vector), v, w
  float red[kTW][kSims][12];  // per-warp partial sums
  float lacc[kTW][kMaxLinks][6];
  unsigned act[kSims][kMaxCullChunks / 32];   // forward: chunks that may touch the object, per simulation
  float loss;
  int cand;                        // the candidate claimed by this CTA
  int bad_object;
  const HandDev* hand_loaded;
};

__device__ __forceinline__ void mat_t_vec(const float R[9], const float v[3], float o[3]) {
  o[0] = fma_(R[0], v[0], fma_(R[3], v[1], mul_(R[6], v[2])));
  o[1] = fma_(R[1], v[0], fma_(R[4], v[1], mul_(R[7], v[2])));
  o[2] = fma_(R[2], v[0], fma_(R[5], v[1], mul_(R[8], v[2])));
}

// Coefficients of Exp(w) = I + c1 [w]x + c2 [w]x^2 (series at small angles).
__device__ __forceinline__ void exp_coeffs(const float w[3], float& c1, float& c2) {
  const float a2 = fma_(w[0], w[0], fma_(w[1], w[1], mul_(w[2], w[2])));
  if (a2 < 1e-12f) {
    c1 = sub_(1.0f, mul_(a2, 1.0f / 6.0f));
    c2 = sub_(0.5f, mul_(a2, 1.0f / 24.0f));
  } else {
    const float a = sqrtf(a2);
    float sh, ch;
    sincosf(0.5f * a, &sh, &ch);
    c1 = __fdiv_rn(mul_(2.0f, mul_(sh, ch)), a);
    const float sa = __fdiv_rn(sh, mul_(0.5f, a));
    c2 = mul_(0.5f, mul_(sa, sa));
  }
}

// z + sg c1 (w x z) + c2 (w x (w x z)) = Exp(sg w) z for sg = +-1.
__device__ __forceinline__ void exp_apply(const float w[3], float c1, float c2, float sg, const float z[3],
                                          float o[3]) {
  float a[3], b[3];
  cross3(w, z, a);
  cross3(w, a, b);
#pragma unroll
  for (int k = 0; k < 3; ++k) o[k] = fma_(c2, b[k], fma_(sg * c1, a[k], z[k]));
}

// Point p (world) at the predicted pose of a step: lever d = p - x~ and the
// object-frame query r = R~^T d.
__device__ __forceinline__ void step_query(const SimStep& s, const float p[3], float d[3], float r[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = sub_(p[k], s.xt[k]);
  mat_t_vec(s.Rt, d, r);
}

// Displacement over the step of the object's material point that sits at p at
// the predicted pose: s = p - (x + R r) = dt v + c1 (wdt x d) - c2 (wdt x (wdt x d)),
// written without the cancellation of the definition.
__device__ __forceinline__ void material_displacement(const SimStep& s, const float d[3], float sr[3]) {
  float a[3], b[3];
  cross3(s.wdt, d, a);
  cross3(s.wdt, a, b);
#pragma unroll
  for (int k = 0; k < 3; ++k) sr[k] = fma_(-s.c2, b[k], fma_(s.c1, a[k], s.dtv[k]));
}

// Tangential part of a displacement: s = sr - (sr . n) n, t = s/|s|; returns |s|
// (0 and t = 0 when the displacement is normal to the surface).
__device__ __forceinline__ float tangent_of(const float n[3], const float sr[3], float t[3]) {
  const float sn = dot3(sr, n);
  float s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = fma_(-sn, n[k], sr[k]);
  const float s2 = dot3(s, s);
  if (!(s2 > 0.0f)) {
    t[0] = t[1] = t[2] = 0.0f;
    return 0.0f;
  }
  const float rs = rsqrtf(s2);
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = mul_(s[k], rs);
  return mul_(s2, rs);
}

// Correction of one contact (C > 0) as a generalised force f = -(lambda_n n +
// lambda_t t) with lever d (Eq. 1 and Coulomb friction on the displacement sr).
__device__ __forceinline__ void force_general(const float d[3], const float n[3], const float sr[3], float C,
                                              const ParamsDev& P, const ObjDev& O, float f[3]) {
  float un[3];
  cross3(d, n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  const float lam_n = C / wn;
  float t[3];
  const float sig = tangent_of(n, sr, t);
  float lam_t = 0.0f;
  if (sig > 0.0f) {
    float ut[3];
    cross3(d, t, ut);
    const float wt = fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass);
    const float muC = mul_(P.mu, C);
    lam_t = (sig <= muC ? sig : muC) / wt;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = -(lam_n * n[k] + lam_t * t[k]);
}

// Adjoint of one (point, simulation) term of a step: given the wrench adjoint
// (Gl, Ga), returns dL/dphi_hat (leaky rule), dL/dn, dL/dd (lever) and dL/dsr.
__device__ void contact_adjoint(const float d[3], const float n[3], const float sr[3], float phi_hat, bool kappa,
                                const float Gl[3], const float Ga[3], const ParamsDev& P, const ObjDev& O,
                                float extra_dC, float& dphi, float dn[3], float dd[3], float dsr[3]) {
  const float C = kappa ? -phi_hat : 0.0f;
  float gad[3];
  cross3(Ga, d, gad);
  const float gf[3] = {Gl[0] + gad[0], Gl[1] + gad[1], Gl[2] + gad[2]};
  float un[3];
  cross3(d, n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  const float rwn = __fdividef(1.0f, wn);
  const float dlam_n = -dot3(gf, n);
  float dC = dlam_n * rwn + extra_dC;
  float t[3];
  const float sig = tangent_of(n, sr, t);
  float rwt = 0.0f, dlam_t = 0.0f;
  float ut[3] = {0.0f, 0.0f, 0.0f};
  bool stat = false;
  if (sig > 0.0f) {
    cross3(d, t, ut);
    const float wt = fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass);
    rwt = __fdividef(1.0f, wt);
    dlam_t = -dot3(gf, t);
    stat = sig <= mul_(P.mu, C);
    if (!stat) dC += P.mu * dlam_t * rwt;      // kinetic: lambda_t = mu C / w_t
  }
  float ds[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int k = 0; k < 3; ++k) dn[k] = dd[k] = 0.0f;
  if (C > 0.0f) {
    const float lam_n = C * rwn;
    const float lam_t = sig > 0.0f ? (stat ? sig : P.mu * C) * rwt : 0.0f;
    float f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = -(lam_n * n[k] + lam_t * t[k]);
    cross3(f, Ga, dd);                               // d(Ga . (d x f))/dd
    float dnl[3] = {-lam_n * gf[0], -lam_n * gf[1], -lam_n * gf[2]};
    const float dwn = -dlam_n * lam_n * rwn;
    const float sn = 2.0f * O.inv_inertia * dwn;
    const float dun[3] = {sn * un[0], sn * un[1], sn * un[2]};
    float tmp[3];
    cross3(n, dun, tmp);
    dd[0] += tmp[0]; dd[1] += tmp[1]; dd[2] += tmp[2];
    cross3(dun, d, tmp);
    dnl[0] += tmp[0]; dnl[1] += tmp[1]; dnl[2] += tmp[2];
    if (sig > 0.0f) {
      float dtt[3] = {-lam_t * gf[0], -lam_t * gf[1], -lam_t * gf[2]};
      const float dsig = stat ? dlam_t * rwt : 0.0f;
      const float dwt = -dlam_t * lam_t * rwt;
      const float st = 2.0f * O.inv_inertia * dwt;
      const float dut[3] = {st * ut[0], st * ut[1], st * ut[2]};
      cross3(t, dut, tmp);
      dd[0] += tmp[0]; dd[1] += tmp[1]; dd[2] += tmp[2];
      cross3(dut, d, tmp);
      dtt[0] += tmp[0]; dtt[1] += tmp[1]; dtt[2] += tmp[2];
      // t = s/sigma, sigma = |s|
      const float tdt = dot3(t, dtt);
      const float rs = __fdividef(1.0f, sig);
#pragma unroll
      for (int k = 0; k < 3; ++k) ds[k] = (dtt[k] - tdt * t[k]) * rs + dsig * t[k];
    }
    dn[0] = dnl[0]; dn[1] = dnl[1]; dn[2] = dnl[2];
  }
  // s = sr - (sr . n) n
  const float nds = dot3(n, ds), srn = dot3(sr, n);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dsr[k] = ds[k] - nds * n[k];
    dn[k] -= srn * ds[k] + nds * sr[k];
  }
  dphi = kappa ? -dC : -P.alpha * dC;
}

// Whether a chunk of points can hold a contact at a step's predicted pose: its
// bounding sphere (centre cw in the world, radius R), moved into the object frame,
// lies in a box over which the min-pyramid bounds the interpolated field; with
// that bound above r_dil (plus float32 slack on positions and values) no point of
// the chunk is in contact.  Same test as the one-step kernel's culling, without
// the plane term.
__device__ __forceinline__ bool chunk_may_touch(const ObjDev& O, const SimStep& st, const float cw[3], float R,
                                                float rdil) {
  float d[3], c[3];
  step_query(st, cw, d, c);
  if (O.kind == kObjMesh) {
    // the centre outside the mesh at flat distance dc > R: rho >= dc - R - (Phong shift bound)
    const float slack = 1e-6f + 1e-5f * (fabsf(cw[0]) + fabsf(cw[1]) + fabsf(cw[2]) + fabsf(d[0]) + fabsf(d[1]) +
                                         fabsf(d[2]));
    const float dc = mesh_flat_distance(O, c);
    const float Rs = R + slack;
    return !(dc > Rs && dc - Rs - O.phong_shift - rdil - (1e-6f + 1e-5f * fabsf(dc)) > 0.0f);
  }
  const float slack = 1e-6f + 1e-5f * (fabsf(cw[0]) + fabsf(cw[1]) + fabsf(cw[2]) + fabsf(d[0]) + fabsf(d[1]) +
                                       fabsf(d[2]));
  const float Ru = (R + slack) * O.inv_h;
  const float org[3] = {O.ox, O.oy, O.oz};
  float lo[3], hi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = (c[k] - org[k]) * O.inv_h;
    lo[k] = u - Ru - 1e-3f;
    hi[k] = u + Ru + 1e-3f;
  }
  const float mn = region_min(O, lo, hi);
  return !(mn - rdil - (1e-6f + 1e-5f * fabsf(mn)) > 0.0f);
}

// Contact flag of a query from its cell and corners: the same arithmetic as the
// full lookup's value (sdf_finish), so the decision is the same bit for bit.
__device__ __forceinline__ bool query_in_contact(const ObjDev& O, const SdfIndex& ix, const float c[8], float rdil) {
  SdfSample smp;
  sdf_finish<false>(O, ix, c, smp);
  return sub_(smp.phi, rdil) < 0.0f;
}

// dL/dphi_hat of a point out of contact (C = 0, kinetic friction since
// sigma > mu C = 0): dC = -(gf . n)/w_n - mu (gf . t)/w_t, dphi_hat = -alpha dC.
__device__ __forceinline__ float leaky_adjoint(const float d[3], const float n[3], const float sr[3],
                                               const float Gl[3], const float Ga[3], const ParamsDev& P,
                                               const ObjDev& O, float extra_dC) {
  float gad[3];
  cross3(Ga, d, gad);
  const float gf[3] = {Gl[0] + gad[0], Gl[1] + gad[1], Gl[2] + gad[2]};
  float un[3];
  cross3(d, n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  float dC = -dot3(gf, n) * __fdividef(1.0f, wn) + extra_dC;
  float t[3];
  const float sig = tangent_of(n, sr, t);
  if (sig > 0.0f) {
    float ut[3];
    cross3(d, t, ut);
    const float wt = fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass);
    dC -= P.mu * dot3(gf, t) * __fdividef(1.0f, wt);
  }
  return -P.alpha * dC;
}

// ANY = false: grid objects only; true: grids and meshes (the lookup dispatches on the kind).
template <int MODE, bool ANY>
__global__ void __launch_bounds__(kTW * 32, 4) tstep_kernel(FusedArgs a) {
  __shared__ TstepSmem S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) S.hand_loaded = nullptr;
  const HandDev& H = S.H;
  const ParamsDev& Pm = S.Pm;

  for (;;) {
    const int c = next_candidate(a.work, &S.cand);
    if (c >= a.B) break;
    if (tid == 0) {
      S.Pm = a.P;
      const int oi = a.obj_of_cand ? a.obj_of_cand[c] : 0;
      S.bad_object = oi < 0 || oi >= a.n_obj;
      if (!S.bad_object) S.O = a.objs[oi];
    }
    __syncthreads();
    if (a.hand != S.hand_loaded) {
      const int* src = reinterpret_cast<const int*>(a.hand);
      int* dst = reinterpret_cast<int*>(&S.H);
      for (int k = tid; k < (int)(sizeof(HandDev) / sizeof(int)); k += kTW * 32) dst[k] = src[k];
      __syncthreads();
      if (tid == 0) S.hand_loaded = a.hand;
    }
    const int D = H.D, P = H.P, L = H.L, T = Pm.sim_steps;
    if (tid < D) S.q[tid] = a.q[(size_t)c * D + tid];
    __syncthreads();
    if (S.bad_object) {
      const float nan = __int_as_float(0x7fc00000);
      if (tid == 0 && a.loss) a.loss[c] = nan;
      if (MODE == kModeLossGrad && a.grad && tid < D) a.grad[(size_t)c * D + tid] = nan;
      continue;
    }
    const ObjDev& O = S.O;
    const int nsteps = MODE == kModeOptimize ? a.nsteps : 1;
    for (int s = 0; s < nsteps; ++s) {
      const float rdil = MODE == kModeOptimize ? dilation_at(Pm, a.step0 + s, a.total_steps) : a.r_fixed;
      const float dt = Pm.dt;
      __syncthreads();
      if (warp == 0) fk_warp(H, S.q, S.frame4, lane);
      if (tid < kSims) {
        const int m = tid;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          S.x[m][k] = 0.0f;
          S.w[m][k] = 0.0f;
          S.v[m][k] = (m > 0 && sim_axis(m) == k) ? sim_sign(m) * Pm.V : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) S.Rc[m][k] = (k % 4 == 0) ? 1.0f : 0.0f;
      }
      for (int idx = tid; idx < kTW * kMaxLinks * 6; idx += kTW * 32) (&S.lacc[0][0][0])[idx] = 0.0f;
      __syncthreads();

      // ------------------------------------------------------------- forward
      for (int t = 0; t < T; ++t) {
        if (tid < kSims) {          // predict (symplectic Euler, no external force)
          const int m = tid;
          SimStep& st = S.st[t][m];
          float E[9];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            st.x[k] = S.x[m][k];
            st.wdt[k] = mul_(dt, S.w[m][k]);
            st.dtv[k] = mul_(dt, S.v[m][k]);
            st.xt[k] = add_(S.x[m][k], st.dtv[k]);
          }
          so3_exp(st.wdt, E);
          matmul3(E, S.Rc[m], st.Rt);
          exp_coeffs(st.wdt, st.c1, st.c2);
        }
        __syncthreads();
        const bool cull = H.nchunks <= kMaxCullChunks;
        if (cull) {
          const int span = ((H.nchunks + 31) >> 5) * 32;
          for (int e = tid; e < kSims * span; e += kTW * 32) {      // a warp's 32 entries share m
            const int m = e / span, j = e - m * span;
            bool active = false;
            if (j < H.nchunks) {
              const int l = H.chunk_link[j];
              active = true;
              if (l >= 0) {
                const float4 cs = __ldg(H.chunk_sphere + j);
                float cw[3];
                world_point(S.frame4[l], cs, cw);
                active = chunk_may_touch(O, S.st[t][m], cw, cs.w, rdil);
              }
            }
            const unsigned word = __ballot_sync(kFull, active);
            if (lane == 0) S.act[m][j >> 5] = word;
          }
          __syncthreads();
        }
        for (int m = 0; m < kSims; ++m) {
          const SimStep st = S.st[t][m];          // registers: the sweep also writes shared memory
          float W[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, cnt = 0.0f;
          for (int j = warp; j < H.nchunks; j += kTW) {
            if (cull && !((S.act[m][j >> 5] >> (j & 31)) & 1u)) continue;   // no contact possible
            const int base = 32 * j, i = base + lane;
            const bool valid = i < P;
            const float4 sp = __ldg(H.pts + (valid ? i : base));
            float p[3], d[3], r[3];
            world_point(S.frame4[(int)sp.w], sp, p);
            step_query(st, p, d, r);
            if (!(ANY && O.kind == kObjMesh)) {
              // point by point (one pyramid entry each): phi_hat(r) >= min - rdil
              const float mn = point_min_bound(O, r);
              if (__all_sync(kFull, !valid || mn - rdil - (1e-6f + 1e-5f * fabsf(mn)) > 0.0f)) continue;
            }
            SdfSample smp;
            sdf_lookup<false, ANY>(O, r, smp);
            PointState ps;
            point_state(smp, r, rdil, ps);
            const bool kap = valid && ps.phi_hat < 0.0f;
            cnt += (float)__popc(__ballot_sync(kFull, kap));
            if (kap) {
              float n[3], sr[3], f[3], tq[3];
              matvec3(st.Rt, ps.n, n);
              material_displacement(st, d, sr);
              force_general(d, n, sr, -ps.phi_hat, Pm, O, f);
              cross3(d, f, tq);
              W[0] += f[0]; W[1] += f[1]; W[2] += f[2];
              W[3] += tq[0]; W[4] += tq[1]; W[5] += tq[2];
            }
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const float v = warp_sum(W[k]);
            if (lane == 0) S.red[warp][m][k] = v;
          }
          if (lane == 0) S.red[warp][m][6] = cnt;
        }
        __syncthreads();
        if (tid < kSims) {          // averaged correction, velocities
          const int m = tid;
          SimStep& st = S.st[t][m];
          float Wt[7];
#pragma unroll
          for (int k = 0; k < 7; ++k) {
            float v = 0.0f;
#pragma unroll
            for (int w = 0; w < kTW; ++w) v += S.red[w][m][k];
            Wt[k] = v;
          }
          const float Nc = fmaxf(Wt[6], 1.0f);
          st.N = Wt[6];
          float dx[3], E[9];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            dx[k] = Wt[k] * O.inv_mass / Nc;
            st.dth[k] = Wt[3 + k] * O.inv_inertia / Nc;
            S.x[m][k] = st.xt[k] + dx[k];
            S.v[m][k] += dx[k] / dt;
            S.w[m][k] += st.dth[k] / dt;
          }
          so3_exp(st.dth, E);
          matmul3(E, st.Rt, S.Rc[m]);
        }
        __syncthreads();
      }

      // ---------------------------------------------------------------- loss
      if (warp == 0) {
        float Lpart = 0.0f;
        if (lane < kSims) {
          const int m = lane;
          const float nv = sqrtf(S.v[m][0] * S.v[m][0] + S.v[m][1] * S.v[m][1] + S.v[m][2] * S.v[m][2]);
          const float nw = sqrtf(S.w[m][0] * S.w[m][0] + S.w[m][1] * S.w[m][1] + S.w[m][2] * S.w[m][2]);
          Lpart = nv + nw;
          const float av = nv > 0.0f ? 1.0f / (kSims * nv) : 0.0f;
          const float aw = nw > 0.0f ? 1.0f / (kSims * nw) : 0.0f;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            S.ab[m][k] = 0.0f;                       // x
            S.ab[m][3 + k] = 0.0f;                   // R
            S.ab[m][6 + k] = S.v[m][k] * av;         // v
            S.ab[m][9 + k] = S.w[m][k] * aw;         // w
          }
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
        if (lane < 6) S.grad[lane] = 0.0f;
        if (lane == 0) S.loss = Ls + Pm.w_range * rn + Pm.w_limit * lims;
      }
      __syncthreads();
      if (MODE == kModeLossGrad && a.grad == nullptr) {
        if (tid == 0) a.loss[c] = S.loss;
        continue;
      }

      // ------------------------------------------------------------- reverse
      for (int t = T - 1; t >= 0; --t) {
        if (tid < kSims) {          // wrench adjoint of the step
          const int m = tid;
          const SimStep& st = S.st[t][m];
          const float Nc = fmaxf(st.N, 1.0f);
          float rb[3], jr[3], E[9], er[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) rb[k] = S.ab[m][3 + k];
          exp_jacobian_T(st.dth, rb, jr);              // R+ = Exp(dtheta) R~
          so3_exp(st.dth, E);
          mat_t_vec(E, rb, er);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float dxb = S.ab[m][k] + S.ab[m][6 + k] / dt;     // x+ = x~ + dx, v+ = v + dx/dt
            const float dthb = S.ab[m][9 + k] / dt + jr[k];        // w+ = w + dtheta/dt
            S.G[m][k] = O.inv_mass * dxb / Nc;
            S.G[m][3 + k] = O.inv_inertia * dthb / Nc;
            S.ab[m][3 + k] = er[k];                                 // R~ part of the adjoint so far
          }
        }
        __syncthreads();
        for (int m = 0; m < kSims; ++m) {
          const SimStep st = S.st[t][m];          // registers: the sweep also writes shared memory
          const float Gl[3] = {S.G[m][0], S.G[m][1], S.G[m][2]};
          const float Ga[3] = {S.G[m][3], S.G[m][4], S.G[m][5]};
          const float extra = (m == 0 && t == 0) ? Pm.w_pen : 0.0f;   // L_pen on the first step at rest
          const float t0[3] = {S.q[0], S.q[1], S.q[2]};
          float accS[12];
#pragma unroll
          for (int k = 0; k < 12; ++k) accS[k] = 0.0f;
          int cur = -1;
          float accL[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
          // contiguous chunks per warp: a warp meets each link in one run
          const int span = (H.nchunks + kTW - 1) / kTW, jb = warp * span, je = min(H.nchunks, jb + span);
          for (int j = jb; j < je; ++j) {
            const int base = 32 * j, i = base + lane;
            const bool valid = i < P;
            const float4 sp = __ldg(H.pts + (valid ? i : base));
            const int link = (int)sp.w;
            float p[3], d[3], r[3];
            world_point(S.frame4[link], sp, p);
            step_query(st, p, d, r);
            // A warp with no point in contact in this simulation and step takes the
            // leaky-only adjoint: C = 0 there, so the force direction (normal,
            // tangent) carries no gradient and only dphi_hat = -alpha dC reaches
            // the query, through the gradient of the SDF (no curvature term).
            SdfIndex ix;
            float corner[8];
            SdfSample msmp;              // mesh objects: the whole lookup (value, gradient, curvature) at once
            bool touch;
            if (ANY && O.kind == kObjMesh) {
              mesh_lookup(O, r, msmp);
              touch = sub_(msmp.phi, rdil) < 0.0f;
            } else {
              sdf_index(O, r, ix);
              sdf_gather(O, ix.cell, corner);
              touch = query_in_contact(O, ix, corner, rdil);
            }
            float pb[3];
            if (!__any_sync(kFull, valid && touch)) {
              SdfSample smp;
              if (ANY && O.kind == kObjMesh)
                smp = msmp;
              else
                sdf_finish<false>(O, ix, corner, smp);
              PointState ps;
              point_state(smp, r, rdil, ps);
              float n[3], sr[3];
              matvec3(st.Rt, ps.n, n);
              material_displacement(st, d, sr);
              const float dphi = leaky_adjoint(d, n, sr, Gl, Ga, Pm, O, extra);
              float rb[3], Rrb[3], rtb[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) rb[k] = dphi * smp.g[k];
              matvec3(st.Rt, rb, Rrb);
              cross3(Rrb, d, rtb);
#pragma unroll
              for (int k = 0; k < 3; ++k) pb[k] = Rrb[k];
              if (valid) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                  accS[k] -= Rrb[k];         // x~
                  accS[3 + k] += rtb[k];     // R~
                }
              }
            } else {
              SdfSample smp;
              if (ANY && O.kind == kObjMesh)
                smp = msmp;
              else
                sdf_finish<true>(O, ix, corner, smp);
              PointState ps;
              point_state(smp, r, rdil, ps);
              const bool kap = ps.phi_hat < 0.0f;
              float n[3], sr[3];
              matvec3(st.Rt, ps.n, n);
              material_displacement(st, d, sr);
              float dphi, dn[3], dd[3], dsr[3];
              contact_adjoint(d, n, sr, ps.phi_hat, kap, Gl, Ga, Pm, O, extra, dphi, dn, dd, dsr);
              // sr = p - x - R r: r gets -R^T dsr, with R^T = R~^T Exp(wdt)
              float e[3], rb[3];
              exp_apply(st.wdt, st.c1, st.c2, 1.0f, dsr, e);
              mat_t_vec(st.Rt, e, rb);
              rb[0] = -rb[0]; rb[1] = -rb[1]; rb[2] = -rb[2];
              // n = R~ n_obj
              float dno[3], rtb[3];
              mat_t_vec(st.Rt, dn, dno);
              cross3(n, dn, rtb);
              sdf_adjoint(smp, ps, dphi, dno, rb);          // adds the lookup's adjoint to rb
              // r = R~^T d
              float Rrb[3], tmp[3];
              matvec3(st.Rt, rb, Rrb);
              cross3(Rrb, d, tmp);
              float Rr[3], rRb[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                dd[k] += Rrb[k];
                rtb[k] += tmp[k];
                pb[k] = dd[k] + dsr[k];
                Rr[k] = d[k] + st.dtv[k] - sr[k];           // R r = p - x - sr
              }
              cross3(dsr, Rr, rRb);
              if (valid) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                  accS[k] -= dd[k];          // x~
                  accS[3 + k] += rtb[k];     // R~
                  accS[6 + k] -= dsr[k];     // x (through sr)
                  accS[9 + k] += rRb[k];     // R (through sr)
                }
              }
            }
            float vL[6];
            if (valid) {
              const float rel[3] = {p[0] - t0[0], p[1] - t0[1], p[2] - t0[2]};
              float tq[3];
              cross3(rel, pb, tq);
              vL[0] = pb[0]; vL[1] = pb[1]; vL[2] = pb[2];
              vL[3] = tq[0]; vL[4] = tq[1]; vL[5] = tq[2];
            } else {
#pragma unroll
              for (int k = 0; k < 6; ++k) vL[k] = 0.0f;
            }
            link_accumulate(S.lacc[warp], lane, link, valid, vL, cur, accL);
          }
          if (cur >= 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              const float sum = warp_sum(accL[k]);
              if (lane == 0) S.lacc[warp][cur][k] += sum;
            }
          }
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            const float v = warp_sum(accS[k]);
            if (lane == 0) S.red[warp][m][k] = v;
          }
        }
        __syncthreads();
        if (tid < kSims) {          // carry the adjoint to the state before the step
          const int m = tid;
          const SimStep& st = S.st[t][m];
          float xtb[3], rtb[3], xd[3], rR[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
            for (int w = 0; w < kTW; ++w) {
              s0 += S.red[w][m][k];
              s1 += S.red[w][m][3 + k];
              s2 += S.red[w][m][6 + k];
              s3 += S.red[w][m][9 + k];
            }
            xtb[k] = S.ab[m][k] + s0;        // x+ = x~ + dx gave ab_x
            rtb[k] = S.ab[m][3 + k] + s1;
            xd[k] = s2;
            rR[k] = s3;
          }
          float E[9], er[3], jr[3];
          so3_exp(st.wdt, E);                 // R~ = Exp(dt w) R
          mat_t_vec(E, rtb, er);
          exp_jacobian_T(st.wdt, rtb, jr);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float vb = S.ab[m][6 + k], wb = S.ab[m][9 + k];
            S.ab[m][k] = xtb[k] + xd[k];          // x~ = x + dt v
            S.ab[m][6 + k] = vb + dt * xtb[k];
            S.ab[m][3 + k] = er[k] + rR[k];
            S.ab[m][9 + k] = wb + dt * jr[k];
          }
        }
        __syncthreads();
      }

      // ---------------------------------------------------------------- tree
      if (warp == 0) {
        float pre[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float x = 0.0f;
          if (lane < L) {
#pragma unroll
            for (int w = 0; w < kTW; ++w) x += S.lacc[w][lane][k];
          }
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
          }
          pre[k] = x;
        }
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
      } else {
        if (tid < D) S.q[tid] -= Pm.lr * S.grad[tid];
        if (tid == 0 && a.loss && s == nsteps - 1) a.loss[c] = S.loss;
      }
    }
    if (MODE == kModeOptimize) {
      __syncthreads();
      if (tid < D) a.q[(size_t)c * D + tid] = S.q[tid];
    }
  }
  work_done(a.work);
}

template <int MODE, bool ANY>
cudaError_t launch_tstep_mode(const FusedArgs& a, cudaStream_t st) {
  static int blocks_per_sm[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& bps = blocks_per_sm[dev & 63];
  if (bps <= 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tstep_kernel<MODE, ANY>, kTW * 32, 0);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
  }
  long long grid = (long long)device_sm_count() * bps;
  if (grid > a.B) grid = a.B;
  if (grid < 1) return cudaSuccess;
  FusedArgs b = a;
  cudaError_t e = work_pair(&b.work, st);
  if (e != cudaSuccess) return e;
  tstep_kernel<MODE, ANY><<<(int)grid, kTW * 32, 0, st>>>(b);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tstep(int mode, const FusedArgs& a, cudaStream_t st) {
  if (a.B <= 0) return cudaSuccess;
  if (a.P.sim_steps < 1 || a.P.sim_steps > kTSteps) return cudaErrorInvalidValue;
  if (a.any_mesh)
    return mode == kModeLossGrad ? launch_tstep_mode<kModeLossGrad, true>(a, st)
                                 : launch_tstep_mode<kModeOptimize, true>(a, st);
  return mode == kModeLossGrad ? launch_tstep_mode<kModeLossGrad, false>(a, st)
                               : launch_tstep_mode<kModeOptimize, false>(a, st);
}

}  // namespace fg

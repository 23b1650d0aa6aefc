// Gauss-Seidel form of the one-step grasp metric (Sec. III-C: the update of
// Eq. 1 for each constraint, applied in turn).  Each of the M = 7 simulations
// keeps a correction state s = (dx, dth), zero at the predicted pose
// x~ = dt v_m, and visits the hand points in index order; point i sees the
// object's material point at p_i displaced by D = x~ + dx + dth x d
// (d = p_i - x~), so its constraint is phi = phi_hat - n . D, and its correction
// (normal projection of Eq. 1, Coulomb friction on the tangential part of D) is
// added to s in full.  x_dot+ = v + dx/dt, theta_dot+ = dth/dt, Eqs. (2)-(4).
// Leaky rule: outside contact C = -alpha (phi - phi_0) through the hand point
// only (the state is held constant in it), so a non-contact point neither moves
// the state nor passes gradient along the chain.
//
// One CTA of 7 warps per candidate (persistent over candidates and steps):
//
//   FK, cull   warp 0 frames; per 32-point chunk a lower bound of phi_hat over
//              its bounding sphere (min-pyramid; for a mesh the flat distance of
//              its centre) and, per simulation, a bound on its points' levers
//   forward    warp m runs simulation m over the chunks in order.  A chunk whose
//              bound exceeds the largest displacement the state can give any
//              of its points holds no contact and is skipped.  Otherwise the
//              lanes evaluate their constraints at the current state, the first
//              lane in contact (after the last one projected) projects, the
//              state is broadcast, and the rest re-evaluate; the lanes projected
//              (the chunk's event mask) and the state at the chunk's start are
//              kept in shared memory.
//   loss       L_stable (Eq. 2) from the final states, its adjoint per
//              simulation, the joint terms
//   reverse    warp m carries the state adjoint backwards over the chunks with
//              events (re-running each such chunk from its start state: per lane
//              state and adjoint, the general contact adjoint for the projected
//              lanes, the leaky one for the rest, through the lookup's adjoint
//              into the warp's link sums) and keeps the adjoint at every chunk's start.
//   adjoint    warps take chunks in a fixed pattern; per point one lookup with
//              second derivatives serves the simulations without events in the
//              chunk: the leaky adjoint at the chunk's (state, state adjoint).
//              dL/dp -> per-link sums.
//   tree, update  as in the one-step kernel
//
// The decision arithmetic (constraint value, tangential displacement, friction
// regime, state updates) is spelled with round-to-nearest intrinsics, and the
// re-runs repeat the forward's operations on the same inputs, so they reproduce
// its states bit for bit.  Work and reductions have a fixed order: results are
// bit-reproducible.
#include <cuda_runtime.h>

#include "fg_fused_kernel.cuh"
#include "fg_internal.h"

namespace fg {

namespace {

constexpr int kGW = kSims;                    // one warp per simulation
constexpr int kSnapWords = 14;                // per chunk and simulation: state (6), adjoint (6), event mask, pad

struct GsSmem {
  HandDev H;
  ObjDev O;
  ParamsDev Pm;
  float4 frame4[kMaxLinks][3];
  float q[64];
  float grad[64];
  float lb[kMaxCullChunks];        // lower bound of phi_hat over the chunk (-inf: never culled)
  float reach[kMaxCullChunks][kSims];   // |c - x~_m| + R: lever bound of the chunk's points in simulation m
  float sfin[kSims][6];            // final state per simulation
  __align__(8) float afin[kSims][6];   // dL/d(final state)
  float red[kSims][8];             // per simulation: sum f (3), sum d x f (3), contacts, penetration
  float lacc[kGW][kMaxLinks][6];   // per warp, per link: sum g, sum (p - t) x g
  float loss;
  int cand;                        // the candidate claimed by this CTA
  int bad_object;
  const HandDev* hand_loaded;
};

// Dynamic shared memory, per chunk c and simulation m (word offsets):
//   [0, 6)  state at the chunk's start,  [6, 12) state adjoint at the chunk's start,
//   12      event mask (lanes projected, as float bits), 13 padding (an even stride
//   keeps the state and the adjoint 8-byte aligned: three 8-byte loads each)
__device__ __forceinline__ float* snap(float* dyn, int c, int m) { return dyn + ((size_t)c * kSims + m) * kSnapWords; }

// v[k] for k = lane (0..5), by selects (no local-memory indexing).
__device__ __forceinline__ float pick6(const float v[6], int k) {
  return k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : k == 3 ? v[3] : k == 4 ? v[4] : v[5];
}

__device__ __forceinline__ void sim_pred(int m, float dtV, float xt[3]) {
  float vd[3];
  sim_dir(m, vd);
  xt[0] = mul_(dtV, vd[0]);
  xt[1] = mul_(dtV, vd[1]);
  xt[2] = mul_(dtV, vd[2]);
}

// Lever d = p - x~ and displacement D = x~ + dx + dth x d of the object's
// material point at p; returns phi = phi_hat - n . D.
__device__ __forceinline__ float gs_phi(const PointState& ps, const float xt[3], const float st[6], float d[3],
                                        float D[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = sub_(ps.p[k], xt[k]);
  float c[3];
  cross3(st + 3, d, c);
#pragma unroll
  for (int k = 0; k < 3; ++k) D[k] = add_(add_(xt[k], st[k]), c[k]);
  return sub_(ps.phi_hat, dot3(ps.n, D));
}

// Tangential part of D: s = D - (D . n) n, t = s/|s|; returns |s| (0 and t = 0
// when D is normal to the surface).
__device__ __forceinline__ float gs_tangent(const float n[3], const float D[3], float t[3], float& sn) {
  sn = dot3(D, n);
  float s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) s[k] = fma_(-sn, n[k], D[k]);
  const float s2 = dot3(s, s);
  if (!(s2 > 0.0f)) {
    t[0] = t[1] = t[2] = 0.0f;
    return 0.0f;
  }
  const float rs = rsqrtf(s2);
  const float sig = mul_(s2, rs);
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = mul_(s[k], rs);
  return sig;
}

// Correction of one projected point (C = -phi > 0): force f = -(lambda_n n +
// lambda_t t) with lambda_n = C / w_n (Eq. 1) and Coulomb friction on the
// tangential displacement (static when sigma <= mu C), torque d x f.
__device__ __forceinline__ void gs_force(const PointState& ps, const float d[3], const float D[3], float C,
                                         const ParamsDev& P, const ObjDev& O, float f[3], float tq[3]) {
  float un[3];
  cross3(d, ps.n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  const float lam_n = mul_(C, rcp_fast(wn));
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = -mul_(lam_n, ps.n[k]);
  float t[3], sn;
  const float sig = gs_tangent(ps.n, D, t, sn);
  if (sig > 0.0f) {
    float ut[3];
    cross3(d, t, ut);
    const float wt = fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass);
    const float muC = mul_(P.mu, C);
    const float lam_t = mul_(sig <= muC ? sig : muC, rcp_fast(wt));
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = fma_(-lam_t, t[k], f[k]);
  }
  cross3(d, f, tq);
}

// s += (f / m, (d x f) / I), the correction of lane j broadcast to the warp.
__device__ __forceinline__ void gs_apply(float st[6], const float f[3], const float tq[3], const ObjDev& O, int j) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    st[k] = fma_(O.inv_mass, __shfl_sync(kFull, f[k], j), st[k]);
    st[3 + k] = fma_(O.inv_inertia, __shfl_sync(kFull, tq[k], j), st[3 + k]);
  }
}

// Leaky adjoint of a point out of contact, given the state st before it and the
// adjoint a of the state after it (equal to the one before: the point changes
// nothing).  With g = n / w_n + mu t / w_t (kinetic friction at C = 0), the
// correction's adjoint is -c dC, c = (a_x . g)/m + (a_th . (d x g))/I, and
// dphi = -alpha dC on phi = phi_hat - n . (x~ + dx + dth x d), the state held.
__device__ __forceinline__ void gs_leaky(const PointState& ps, const float xt[3], const float st[6], const float a[6],
                                         float extra_dC, const ParamsDev& P, const ObjDev& O, float& dphi,
                                         float dn[3], float dp[3]) {
  float d[3], D[3];
  gs_phi(ps, xt, st, d, D);
  float un[3];
  cross3(d, ps.n, un);
  const float rwn = rcp_fast(fma_(O.inv_inertia, dot3(un, un), O.inv_mass));
  // tangential direction of D (no branch depends on its rounding: only s2 > 0 does)
  const float sn = dot3(D, ps.n);
  float t[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = fmaf(-sn, ps.n[k], D[k]);
  const float s2 = dot3(t, t);
  float c = rwn * (O.inv_mass * dot3(a, ps.n) + O.inv_inertia * dot3(a + 3, un));
  if (s2 > 0.0f) {
    const float rs = rsqrtf(s2);
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] *= rs;
    float ut[3];
    cross3(d, t, ut);
    const float rwt = rcp_fast(fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass));
    c += P.mu * rwt * (O.inv_mass * dot3(a, t) + O.inv_inertia * dot3(a + 3, ut));
  }
  const float phibar = P.alpha * (c - extra_dC);      // -alpha (-c + extra)
  dphi += phibar;
  float wn_[3];
  cross3(st + 3, ps.n, wn_);                            // dphi/dd = -(n x dth) = dth x n
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dn[k] -= phibar * D[k];
    dp[k] += phibar * wn_[k];
  }
}

// The record a chunk without events of simulation m keeps for the adjoint of its
// points, in place of its state and state adjoint: e = x~ + dx - dth x x~ (then
// D = e + dth x p for every point of the chunk), dth, and the state adjoint scaled
// by the inverse mass and inertia.  The state and its adjoint are constant across
// such a chunk, so these are shared by its 32 points.
__device__ __forceinline__ void gs_segment_record(float* sc, const float a[6], const float xt[3], const ObjDev& O) {
  const float dth[3] = {sc[3], sc[4], sc[5]};
  float c[3];
  cross3(dth, xt, c);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sc[k] = sc[k] + xt[k] - c[k];
    sc[6 + k] = O.inv_mass * a[k];
    sc[9 + k] = O.inv_inertia * a[3 + k];
  }
}

// gs_leaky from a chunk's record (gs_segment_record): the same leaky adjoint, with
// U = p x n shared by the simulations and the outputs that are linear in phibar
// accumulated per point (sd = sum phibar dth, se = sum phibar e; afterwards
// dn -= se + sd x p and dp += sd x n).
__device__ __forceinline__ void gs_leaky_rec(const PointState& ps, const float U[3], const float xt[3],
                                             const float e[3], const float dth[3], const float ax[3],
                                             const float ath[3], float extra_dC, const ParamsDev& P,
                                             const ObjDev& O, float& dphi, float sd[3], float se[3]) {
  float c3[3], xn[3], D[3], un[3];
  cross3(dth, ps.p, c3);
  cross3(xt, ps.n, xn);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    D[k] = e[k] + c3[k];
    un[k] = U[k] - xn[k];
  }
  const float rwn = rcp_fast(fma_(O.inv_inertia, dot3(un, un), O.inv_mass));
  const float sn = dot3(D, ps.n);
  float t[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = fmaf(-sn, ps.n[k], D[k]);
  const float s2 = dot3(t, t);
  float c = rwn * (dot3(ax, ps.n) + dot3(ath, un));
  if (s2 > 0.0f) {
    const float rs = rsqrtf(s2);
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] *= rs;
    const float d[3] = {ps.p[0] - xt[0], ps.p[1] - xt[1], ps.p[2] - xt[2]};
    float ut[3];
    cross3(d, t, ut);
    const float rwt = rcp_fast(fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass));
    c += P.mu * rwt * (dot3(ax, t) + dot3(ath, ut));
  }
  const float phibar = P.alpha * (c - extra_dC);
  dphi += phibar;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sd[k] = fmaf(phibar, dth[k], sd[k]);
    se[k] = fmaf(phibar, e[k], se[k]);
  }
}

// General adjoint of a projected point: a is the adjoint of the state after
// it, st the state before it.  Adds dL/dphi_hat, dL/dn, dL/dp and returns the
// adjoint of the state before it minus a in ds (the correction's dependence on
// the state through D).
__device__ __forceinline__ void gs_contact_adjoint(const PointState& ps, const float xt[3], const float st[6],
                                                   const float a[6], float extra_dC, const ParamsDev& P,
                                                   const ObjDev& O, float& dphi, float dn[3], float dp[3],
                                                   float ds[6]) {
  float d[3], D[3];
  const float phi = gs_phi(ps, xt, st, d, D);
  const float C = -phi;
  const float* n = ps.n;
  // forward values
  float un[3];
  cross3(d, n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  const float rwn = rcp_fast(wn);
  const float lam_n = C * rwn;
  float t[3], sn;
  const float sig = gs_tangent(n, D, t, sn);
  float ut[3] = {0.0f, 0.0f, 0.0f}, rwt = 0.0f, lam_t = 0.0f;
  bool stat = false;
  if (sig > 0.0f) {
    cross3(d, t, ut);
    rwt = rcp_fast(fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass));
    stat = sig <= mul_(P.mu, C);
    lam_t = (stat ? sig : P.mu * C) * rwt;
  }
  float f[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = -(lam_n * n[k] + lam_t * t[k]);
  // reverse: ds_after = (f/m, (d x f)/I) against a
  float gf[3], tmp[3];
  cross3(a + 3, d, tmp);                                 // a_th . (d x f) = f . (a_th x d)
#pragma unroll
  for (int k = 0; k < 3; ++k) gf[k] = O.inv_mass * a[k] + O.inv_inertia * tmp[k];
  float dd[3];
  cross3(f, a + 3, dd);                                  // d(a_th . (d x f))/dd = f x a_th
#pragma unroll
  for (int k = 0; k < 3; ++k) dd[k] *= O.inv_inertia;
  const float lbn = -dot3(gf, n), lbt = -dot3(gf, t);
  float nb[3], tb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nb[k] = -lam_n * gf[k];
    tb[k] = -lam_t * gf[k];
  }
  float Cb = lbn * rwn + extra_dC;
  {  // w_n = 1/m + |d x n|^2 / I
    const float s = 2.0f * O.inv_inertia * (-lbn * lam_n * rwn);
    const float ub[3] = {s * un[0], s * un[1], s * un[2]};
    cross3(n, ub, tmp);
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] += tmp[k];
    cross3(ub, d, tmp);
#pragma unroll
    for (int k = 0; k < 3; ++k) nb[k] += tmp[k];
  }
  float Db[3] = {0.0f, 0.0f, 0.0f};
  if (sig > 0.0f) {
    float sigb = 0.0f;
    if (stat)
      sigb = lbt * rwt;
    else
      Cb += P.mu * lbt * rwt;
    const float s = 2.0f * O.inv_inertia * (-lbt * lam_t * rwt);
    const float ub[3] = {s * ut[0], s * ut[1], s * ut[2]};
    cross3(t, ub, tmp);
#pragma unroll
    for (int k = 0; k < 3; ++k) dd[k] += tmp[k];
    cross3(ub, d, tmp);
#pragma unroll
    for (int k = 0; k < 3; ++k) tb[k] += tmp[k];
    // t = s/sigma, sigma = |s|, s = D - (D . n) n
    const float ttb = dot3(t, tb);
    const float rs = __fdividef(1.0f, sig);
    float sb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sb[k] = (tb[k] - ttb * t[k]) * rs + sigb * t[k];
    const float nsb = dot3(n, sb);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Db[k] = sb[k] - nsb * n[k];
      nb[k] -= sn * sb[k] + nsb * D[k];
    }
  }
  // C = -phi (in contact), phi = phi_hat - n . D
  const float phib = -Cb;
  dphi += phib;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    nb[k] -= phib * D[k];
    Db[k] -= phib * n[k];
    dn[k] += nb[k];
  }
  // D = x~ + dx + dth x d
  float dthb[3], ddb[3];
  cross3(d, Db, dthb);                                   // d(Db . (dth x d))/ddth = d x Db
  cross3(Db, st + 3, ddb);                               // ... /dd = Db x dth
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ds[k] = Db[k];
    ds[3 + k] = dthb[k];
    dp[k] += dd[k] + ddb[k];
  }
}

// One chunk of simulation m in reverse: from the state st0 at its start, the
// adjoint a at its end and its event mask, gives each lane the state before it
// (smine) and the adjoint after it (amine), computes the general adjoint of the
// projected lanes (into dphi, dn, dp) and returns in a the adjoint at the
// chunk's start.
__device__ __forceinline__ void gs_chunk_reverse(const PointState& ps, const float xt[3], const float st0[6],
                                                 float a[6], unsigned mask, int m, int lane, const ParamsDev& P,
                                                 const ObjDev& O, float smine[6], float amine[6], float& dphi,
                                                 float dn[3], float dp[3]) {
  float st[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) st[k] = smine[k] = st0[k];
  for (unsigned rest = mask; rest; rest &= rest - 1u) {   // forward re-run, lanes in order
    const int j = __ffs(rest) - 1;
    float f[3] = {0.0f, 0.0f, 0.0f}, tq[3] = {0.0f, 0.0f, 0.0f};
    if (lane == j) {
      float d[3], D[3];
      const float phi = gs_phi(ps, xt, st, d, D);
      gs_force(ps, d, D, -phi, P, O, f, tq);
    }
    gs_apply(st, f, tq, O, j);
    if (lane > j) {
#pragma unroll
      for (int k = 0; k < 6; ++k) smine[k] = st[k];
    }
  }
  int hi = 32;
  for (unsigned rest = mask; rest;) {                     // events in reverse
    const int j = 31 - __clz(rest);
    rest &= ~(1u << j);
    if (lane >= j && lane < hi) {
#pragma unroll
      for (int k = 0; k < 6; ++k) amine[k] = a[k];
    }
    float ds[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (lane == j) gs_contact_adjoint(ps, xt, smine, a, m == 0 ? P.w_pen : 0.0f, P, O, dphi, dn, dp, ds);
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] += __shfl_sync(kFull, ds[k], j);
    hi = j;
  }
  if (lane < hi) {
#pragma unroll
    for (int k = 0; k < 6; ++k) amine[k] = a[k];
  }
}

// ANY = false: grid objects only; true: grids and meshes (the lookup dispatches on the kind).
template <int MODE, bool ANY>
__global__ void __launch_bounds__(kGW * 32, 3) gs_kernel(FusedArgs a) {
  __shared__ GsSmem S;
  extern __shared__ float dyn[];
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
    if (a.hand != S.hand_loaded) {              // uniform: every thread reads the same words
      const int* src = reinterpret_cast<const int*>(a.hand);
      int* dst = reinterpret_cast<int*>(&S.H);
      for (int k = tid; k < (int)(sizeof(HandDev) / sizeof(int)); k += kGW * 32) dst[k] = src[k];
    }
    __syncthreads();
    if (tid == 0) S.hand_loaded = a.hand;
    const int D = H.D, P = H.P, L = H.L, nch = H.nchunks;
    if (tid < D) S.q[tid] = a.q[(size_t)c * D + tid];
    __syncthreads();
    if (S.bad_object) {
      const float nan = __int_as_float(0x7fc00000);
      if (MODE == kModeWrench) {
        for (int idx = tid; idx < kSims * 6; idx += kGW * 32) a.wrench[(size_t)c * kSims * 6 + idx] = nan;
        if (tid < kSims) a.ncontact[(size_t)c * kSims + tid] = -1;
      } else if (MODE == kModeLossGrad) {
        if (tid == 0) a.loss[c] = nan;
        if (a.grad && tid < D) a.grad[(size_t)c * D + tid] = nan;
      } else if (a.loss && tid == 0) {
        a.loss[c] = nan;
      }
      continue;
    }
    const ObjDev& O = S.O;
    const float dtV = Pm.dt * Pm.V;
    const int nsteps = MODE == kModeOptimize ? a.nsteps : 1;
    for (int s = 0; s < nsteps; ++s) {
      const float r = MODE == kModeOptimize ? dilation_at(Pm, a.step0 + s, a.total_steps) : a.r_fixed;
      __syncthreads();
      if (warp == 0) fk_warp(H, S.q, S.frame4, lane);
      for (int idx = tid; idx < kGW * kMaxLinks * 6; idx += kGW * 32) (&S.lacc[0][0][0])[idx] = 0.0f;
      __syncthreads();

      // ------------------------------------------------- chunk bounds (culling)
      // Every point of chunk j lies in its bounding sphere (centre cw, radius R);
      // the interpolated field over the sphere's box is bounded below by the
      // min-pyramid, so phi_hat >= lb = min - r over the chunk.  For a mesh: if the
      // centre is outside at flat distance d > R, rho >= d - R - (the Phong shift bound).
      for (int j = tid; j < nch; j += kGW * 32) {
        const int l = H.chunk_link[j];
        float lbj = -3.0e38f;
        float4 cwj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (ANY && O.kind == kObjMesh) {
          if (l >= 0) {
            const float4 cs = __ldg(H.chunk_sphere + j);
            float cw[3];
            world_point(S.frame4[l], cs, cw);
            const float slack = 1e-6f + 1e-5f * (fabsf(cw[0]) + fabsf(cw[1]) + fabsf(cw[2]));
            const float R = cs.w + slack;
            const float dc = mesh_flat_distance(O, cw);
            if (dc > R) lbj = dc - R - O.phong_shift - r - 1e-5f * fabsf(dc);
            cwj = make_float4(cw[0], cw[1], cw[2], R);
          }
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
          lbj = region_min(O, lo, hi) - r;
          cwj = make_float4(cw[0], cw[1], cw[2], cs.w + slack);
        }
        S.lb[j] = lbj;
#pragma unroll
        for (int m = 0; m < kSims; ++m) {
          float xt[3];
          sim_pred(m, dtV, xt);
          const float rel[3] = {cwj.x - xt[0], cwj.y - xt[1], cwj.z - xt[2]};
          S.reach[j][m] = sqrtf(rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2]) + cwj.w;
        }
      }
      __syncthreads();

      // ------------------------------------------------------------- forward
      {
        const int m = warp;
        float xt[3];
        sim_pred(m, dtV, xt);
        float st[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float Wl[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, pen = 0.0f;
        int cnt = 0;
        // |x~ + dx| and |dth| of the current state (recomputed when a projection changes it)
        float ex = sqrtf(xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2]), en = 0.0f;
        // The chunks are visited in windows of 32: lane l tests chunk j + l at the
        // current state, and the chunks before the first one that can hold a contact
        // get their snapshot (the current state, no events) in parallel.  The state
        // changes only at projections, so every chunk is tested at the same state
        // as in a walk that visits the chunks one by one.
        int j = 0;
        while (j < nch) {
          const int jj = j + lane;
          bool open_ = false;
          if (jj < nch) {
            // largest |n . D| over the chunk: |x~ + dx| + |dth| (|c - x~| + R)
            const float bound = fmaf(en, S.reach[jj][m], ex);
            const float lbj = S.lb[jj];
            open_ = !(lbj - bound * (1.0f + 1e-5f) - (1e-6f + 1e-5f * fabsf(lbj)) > 0.0f);
          }
          const unsigned ob = __ballot_sync(kFull, open_);
          const int jn = ob ? j + __ffs(ob) - 1 : min(j + 32, nch);
          if (jj < jn) {                                  // culled chunks: state, no events
            float* sc = snap(dyn, jj, m);
#pragma unroll
            for (int k = 0; k < 6; ++k) sc[k] = st[k];
            sc[12] = __uint_as_float(0u);
          }
          if (!ob) {
            j = jn;
            continue;
          }
          float* sn = snap(dyn, jn, m);
          if (lane < 6) sn[lane] = pick6(st, lane);
          unsigned mask = 0u;
          const int i = 32 * jn + lane;
          const bool valid = i < P;
          const float4 sp = __ldg(H.pts + (valid ? i : 32 * jn));
          float p[3];
          world_point(S.frame4[(int)sp.w], sp, p);
          bool clear = !valid;
          if (!(ANY && O.kind == kObjMesh) && valid) {
            // point by point (one pyramid entry each): phi = phi_hat - n . D with
            // phi_hat >= min - r and |n . D| <= |x~ + dx| + |dth| |p - x~|
            const float mn = point_min_bound(O, p);
            const float dl[3] = {p[0] - xt[0], p[1] - xt[1], p[2] - xt[2]};
            const float bnd = fmaf(en, sqrtf(dl[0] * dl[0] + dl[1] * dl[1] + dl[2] * dl[2]), ex);
            clear = mn - r - bnd * (1.0f + 1e-5f) - (1e-6f + 1e-5f * fabsf(mn)) > 0.0f;
          }
          if (!__all_sync(kFull, clear)) {
            SdfSample smp;
            sdf_lookup<false, ANY>(O, p, smp);
            PointState ps;
            point_state(smp, p, r, ps);
            int last = -1;
            for (;;) {
              float d[3], Dd[3];
              const float phi = gs_phi(ps, xt, st, d, Dd);
              const unsigned cand = __ballot_sync(kFull, valid && lane > last && phi < 0.0f);
              if (!cand) break;
              const int jl = __ffs(cand) - 1;
              float f[3] = {0.0f, 0.0f, 0.0f}, tq[3] = {0.0f, 0.0f, 0.0f};
              if (lane == jl) {
                gs_force(ps, d, Dd, -phi, Pm, O, f, tq);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                  Wl[k] += f[k];
                  Wl[3 + k] += tq[k];
                }
                if (m == 0) pen -= phi;
              }
              gs_apply(st, f, tq, O, jl);
              mask |= 1u << jl;
              last = jl;
            }
          }
          if (lane == 0) sn[12] = __uint_as_float(mask);
          cnt += __popc(mask);
          if (mask) {
            const float e[3] = {xt[0] + st[0], xt[1] + st[1], xt[2] + st[2]};
            ex = sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            en = sqrtf(st[3] * st[3] + st[4] * st[4] + st[5] * st[5]);
          }
          j = jn + 1;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const float v = warp_sum(Wl[k]);
          if (lane == 0) {
            S.red[m][k] = v;
            S.sfin[m][k] = st[k];
          }
        }
        pen = warp_sum(pen);
        if (lane == 0) {
          S.red[m][6] = (float)cnt;
          S.red[m][7] = pen;
        }
      }
      __syncthreads();
      if (MODE == kModeWrench) {
        // the sums of the corrections applied, the points projected, and their lanes per chunk
        for (int idx = tid; idx < kSims * 6; idx += kGW * 32)
          a.wrench[(size_t)c * kSims * 6 + idx] = S.red[idx / 6][idx % 6];
        if (tid < kSims) a.ncontact[(size_t)c * kSims + tid] = (int)S.red[tid][6];
        if (a.bits)
          for (int idx = tid; idx < kSims * nch; idx += kGW * 32) {
            const int m = idx / nch, j = idx - m * nch;
            a.bits[((size_t)c * kSims + m) * nch + j] = __float_as_uint(snap(dyn, j, m)[12]);
          }
        continue;
      }

      // ---------------------------------------------------------------- loss
      if (warp == 0) {
        float Lpart = 0.0f;
        if (lane < kSims) {
          const int m = lane;
          float v[3] = {0.0f, 0.0f, 0.0f};
          if (m > 0) v[sim_axis(m)] = sim_sign(m) * Pm.V;
          const float rdt = 1.0f / Pm.dt;
          float xd[3], td[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            xd[k] = v[k] + S.sfin[m][k] * rdt;
            td[k] = S.sfin[m][3 + k] * rdt;
          }
          const float nx = sqrtf(xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2]);
          const float nt = sqrtf(td[0] * td[0] + td[1] * td[1] + td[2] * td[2]);
          Lpart = nx + nt;
          const float ax = nx > 0.0f ? rdt / (kSims * nx) : 0.0f;
          const float at = nt > 0.0f ? rdt / (kSims * nt) : 0.0f;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            S.afin[m][k] = xd[k] * ax;
            S.afin[m][3 + k] = td[k] * at;
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
        float pen = 0.0f;
        if (lane == 0) pen = S.red[0][7];
        if (lane == 0) S.loss = Ls + Pm.w_range * rn + Pm.w_limit * lims + Pm.w_pen * pen;
      }
      __syncthreads();
      if (MODE == kModeLossGrad && a.grad == nullptr) {    // loss only: no adjoint
        if (tid == 0) a.loss[c] = S.loss;
        continue;
      }

      // ------------------------------------- reverse: state adjoint per chunk
      // A chunk with events of simulation m is finished here: its lanes' states
      // and adjoints come out of the re-run, so their contribution of simulation m
      // goes through the lookup's adjoint and into the warp's link sums now, and
      // the sweep over all points below leaves simulation m of that chunk out.
      int cur = -1;
      float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      const float t0[3] = {S.q[0], S.q[1], S.q[2]};
      {
        const int m = warp;
        float xt[3];
        sim_pred(m, dtV, xt);
        float av[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) av[k] = S.afin[m][k];
        // Windows of 32 chunks from the end: lane l reads the event mask of chunk
        // j - l; the chunks after the last one with events get the adjoint (unchanged
        // across them) in parallel, then that chunk is reversed.
        int j = nch - 1;
        while (j >= 0) {
          const int jj = j - lane;
          const bool ev = jj >= 0 && __float_as_uint(snap(dyn, jj, m)[12]) != 0u;
          const unsigned eb = __ballot_sync(kFull, ev);
          const int je = eb ? j - (__ffs(eb) - 1) : max(j - 32, -1);
          if (jj > je && jj >= 0)                        // chunks without events: the adjoint passes through
            gs_segment_record(snap(dyn, jj, m), av, xt, O);
          if (!eb) {
            j = je;
            continue;
          }
          float* sn = snap(dyn, je, m);
          const unsigned mask = __float_as_uint(sn[12]);
          {
            const int i = 32 * je + lane;
            const bool valid = i < P;
            const float4 sp = __ldg(H.pts + (valid ? i : 32 * je));
            const int link = (int)sp.w;
            float p[3];
            world_point(S.frame4[link], sp, p);
            SdfSample smp;
            sdf_lookup<true, ANY>(O, p, smp);
            PointState ps;
            point_state(smp, p, r, ps);
            float st0[6], smine[6], amine[6], dphi = 0.0f, dn[3] = {0.0f, 0.0f, 0.0f}, dp[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < 6; ++k) st0[k] = sn[k];
            gs_chunk_reverse(ps, xt, st0, av, mask, m, lane, Pm, O, smine, amine, dphi, dn, dp);
            if (!((mask >> lane) & 1u)) gs_leaky(ps, xt, smine, amine, m == 0 ? Pm.w_pen : 0.0f, Pm, O, dphi, dn, dp);
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
            link_accumulate(S.lacc[warp], lane, link, valid, v, cur, acc);
          }
          if (lane < 6) sn[6 + lane] = pick6(av, lane);
          j = je - 1;
        }
      }
      __syncthreads();

      // ----------------------------------------------- adjoint of every point
      {
        for (int j = warp; j < nch; j += kGW) {
          const int i = 32 * j + lane;
          const bool valid = i < P;
          const float4 sp = __ldg(H.pts + (valid ? i : 32 * j));
          const int link = (int)sp.w;
          float p[3];
          world_point(S.frame4[link], sp, p);
          SdfSample smp;
          sdf_lookup<true, ANY>(O, p, smp);
          PointState ps;
          point_state(smp, p, r, ps);
          float dphi = 0.0f, dn[3] = {0.0f, 0.0f, 0.0f}, dp[3] = {0.0f, 0.0f, 0.0f};
          float U[3], sd[3] = {0.0f, 0.0f, 0.0f}, se[3] = {0.0f, 0.0f, 0.0f};
          cross3(ps.p, ps.n, U);
#pragma unroll 1
          for (int m = 0; m < kSims; ++m) {
            const float* sn = snap(dyn, j, m);
            if (__float_as_uint(sn[12]) != 0u) continue;    // reversed with its events above
            float xt[3];
            sim_pred(m, dtV, xt);
            const float2* r2 = reinterpret_cast<const float2*>(sn);
            float rec[12];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              const float2 x = r2[k];
              rec[2 * k] = x.x;
              rec[2 * k + 1] = x.y;
            }
            gs_leaky_rec(ps, U, xt, rec, rec + 3, rec + 6, rec + 9, m == 0 ? Pm.w_pen : 0.0f, Pm, O, dphi, sd, se);
          }
          {
            float sp_[3], sn_[3];
            cross3(sd, ps.p, sp_);
            cross3(sd, ps.n, sn_);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              dn[k] -= se[k] + sp_[k];
              dp[k] += sn_[k];
            }
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
          link_accumulate(S.lacc[warp], lane, link, valid, v, cur, acc);
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
        float pre[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float x = 0.0f;
          if (lane < L) {
#pragma unroll
            for (int w = 0; w < kGW; ++w) x += S.lacc[w][lane][k];
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
cudaError_t launch_gs_mode(const FusedArgs& a, int nchunks, cudaStream_t st) {
  const size_t dyn = sizeof(float) * (size_t)nchunks * kSims * kSnapWords;
  static size_t attr_set[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dyn > attr_set[dev & 63]) {
    cudaError_t e = cudaFuncSetAttribute(gs_kernel<MODE, ANY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    attr_set[dev & 63] = dyn;
  }
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, gs_kernel<MODE, ANY>, kGW * 32, dyn);
  if (e != cudaSuccess) return e;
  if (bps < 1) bps = 1;
  long long grid = (long long)device_sm_count() * bps;
  if (grid > a.B) grid = a.B;
  if (grid < 1) return cudaSuccess;
  FusedArgs b = a;
  e = work_pair(&b.work, st);
  if (e != cudaSuccess) return e;
  gs_kernel<MODE, ANY><<<(int)grid, kGW * 32, dyn, st>>>(b);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gs(int mode, const FusedArgs& a, int nchunks, cudaStream_t st) {
  if (a.B <= 0) return cudaSuccess;
  if (nchunks < 1 || nchunks > kMaxCullChunks) return cudaErrorInvalidValue;
  if (a.any_mesh) {
    if (mode == kModeWrench) return launch_gs_mode<kModeWrench, true>(a, nchunks, st);
    return mode == kModeLossGrad ? launch_gs_mode<kModeLossGrad, true>(a, nchunks, st)
                                 : launch_gs_mode<kModeOptimize, true>(a, nchunks, st);
  }
  if (mode == kModeWrench) return launch_gs_mode<kModeWrench, false>(a, nchunks, st);
  return mode == kModeLossGrad ? launch_gs_mode<kModeLossGrad, false>(a, nchunks, st)
                               : launch_gs_mode<kModeOptimize, false>(a, nchunks, st);
}

}  // namespace fg

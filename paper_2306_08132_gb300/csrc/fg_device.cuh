// Device-side data layouts and per-point arithmetic of the grasp-search step.
//
// Everything a kernel needs about one step of one candidate lives here, written
// once and used by the fused kernel (fg_fused.cu) and the per-stage kernels
// (fg_plain.cu).  The arithmetic that decides a branch (point position, grid
// cell, interpolated value and normal, contact flag, friction regime) is spelled
// with explicit round-to-nearest intrinsics so that every call site rounds
// identically and the forward sweep, the adjoint sweep and the per-stage form
// agree bit for bit on every decision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fastgraspd.h"
#include "fg_vec.cuh"

namespace fg {

constexpr int kSims = FG_NUM_SIMS;
constexpr int kMaxLinks = FG_MAX_LINKS;

struct HandDev {
  int L, J, D, P;
  int max_depth;
  int aligned32;                 // every link starts at a multiple of 32 points
  int parent[kMaxLinks];
  int depth[kMaxLinks];
  float T_fix[kMaxLinks][12];    // row-major [R | t]
  float axis[kMaxLinks][3];
  float q_low[kMaxLinks];        // per joint j = l - 1
  float q_up[kMaxLinks];
  int subtree_end[kMaxLinks];    // links are in depth-first preorder: subtree(l) = [l, subtree_end[l])
  int nchunks;                   // ceil(P / 32) chunks of 32 consecutive points
  const float4* pts;             // [P] (x, y, z, link index as float)
  const float4* chunk_sphere;    // [nchunks] bounding sphere in the link frame (centre, radius)
  const int* chunk_link;         // [nchunks] link of the chunk, -1 when it spans two links
  // work units of the adjoint sweep: runs of at most kUnitPoints points of one link
  int nunits;
  int unit_begin[kMaxLinks + 1]; // units of link l: [unit_begin[l], unit_begin[l + 1])
  const int4* units;             // [nunits] (first point, point count, link, 0)
};

constexpr int kUnitPoints = 64;

// Chunks a fused CTA can cull in shared memory (hands up to 8,192 points).
constexpr int kMaxCullChunks = 256;

constexpr int kMaxPyrLevels = 12;

struct ObjDev {
  const float* grid;             // [nz][ny][nx]
  int nx, ny, nz;
  int pyr_levels;                // levels 1..pyr_levels of the min-pyramid
  float ox, oy, oz;              // origin
  float inv_h, h;                // 1/pitch, pitch
  float inv_mass, inv_inertia;
  float uo[3];                   // -origin / pitch: index coordinate u = p / pitch + uo
  const float* pyr;              // min-pyramid, level k at pyr + pyr_off[k - 1]
  int pyr_off[kMaxPyrLevels];
  // kind 1: a watertight triangle mesh queried directly (Phong SDF); the grid
  // fields above are unused and the min-pyramid is absent.
  int kind;                      // 0 grid, 1 mesh
  int n_faces;
  float phong_alpha;
  float phong_shift;             // bound on |r*_rho - r*| (the Phong point's distance from the flat closest point)
  const float4* bvh;             // 2 per node: (min, right child | first face), (max, face count; 0 = inner)
  // Per face, in BVH order; the w components hold ints (as bits) for the
  // certified local search (mesh_local).
  const float4* tri;             // 3: vertex k of (a, b, c); w: the face across edge (k, k+1)
  const float4* face_nrm;        // 7: vertex normals of a, b, c (w: first edge of the vertex's
                                 // ring); face normal (w: 1 for a face on the convex hull); edge
                                 // pseudonormals of (a,b), (b,c), (c,a) (w: ring length of vertex
                                 // k, bit 30 set when all its faces are hull faces)
  const float4* wing;            // 3: vertex of the face across edge k opposite it (w: 1 when both
                                 // faces of the edge are hull faces)
  const float4* ring;            // per directed edge v -> u, grouped by v: u (w: the face holding it)
  const int* start_face;         // [nz][ny][nx]: closest face at the nodes of a coarse grid
  float start_org[3];            // its first node
  float start_inv_h;             // 1 / node spacing
  int start_n[3];                // nodes per axis
};

constexpr int kObjGrid = 0;
constexpr int kObjMesh = 1;

struct ParamsDev {
  float alpha, dt, V, mu, lr, r0, w_range, w_limit, w_pen;
  int schedule;
  int sim_steps;                 // 0: one plane-linearised step; T >= 1: T re-queried steps
  int gauss_seidel;              // 1: constraints projected one after another in point order
};

// -------------------------------------------------------------------- rounding
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }

struct Frame {                   // rotation (row-major) and origin of a link
  float R[9];
  float o[3];
};

// ------------------------------------------------------------------ kinematics

// Rotation by angle |w| about w (Rodrigues).  (1 - cos a)/a^2 is evaluated as
// (sin(a/2)/(a/2))^2 / 2, which has no cancellation at small angles.
__device__ inline void so3_exp(const float w[3], float R[9]) {
  float a2 = fma_(w[0], w[0], fma_(w[1], w[1], mul_(w[2], w[2])));
  float c1, c2;
  if (a2 < 1e-12f) {
    c1 = sub_(1.0f, mul_(a2, 1.0f / 6.0f));
    c2 = sub_(0.5f, mul_(a2, 1.0f / 24.0f));
  } else {
    float a = sqrtf(a2);
    float sh, ch, s, c;
    sincosf(0.5f * a, &sh, &ch);
    s = mul_(2.0f, mul_(sh, ch));             // sin a
    c1 = __fdiv_rn(s, a);
    float sa = __fdiv_rn(sh, mul_(0.5f, a));
    c2 = mul_(0.5f, mul_(sa, sa));
    (void)c;
  }
  // R = I + c1 K + c2 K^2, K = [w]x, K^2 = w w^T - a2 I
  float x = w[0], y = w[1], z = w[2];
  R[0] = fma_(c2, sub_(mul_(x, x), a2), 1.0f);
  R[4] = fma_(c2, sub_(mul_(y, y), a2), 1.0f);
  R[8] = fma_(c2, sub_(mul_(z, z), a2), 1.0f);
  float xy = mul_(c2, mul_(x, y)), xz = mul_(c2, mul_(x, z)), yz = mul_(c2, mul_(y, z));
  float cx = mul_(c1, x), cy = mul_(c1, y), cz = mul_(c1, z);
  R[1] = sub_(xy, cz); R[3] = add_(xy, cz);
  R[2] = add_(xz, cy); R[6] = sub_(xz, cy);
  R[5] = sub_(yz, cx); R[7] = add_(yz, cx);
}

// Rotation by theta about a unit axis.
__device__ inline void axis_rot(const float a[3], float theta, float R[9]) {
  float sh, ch;
  sincosf(0.5f * theta, &sh, &ch);
  float s = mul_(2.0f, mul_(sh, ch));
  float v = mul_(2.0f, mul_(sh, sh));        // 1 - cos theta
  float x = a[0], y = a[1], z = a[2];
  R[0] = fma_(v, sub_(mul_(x, x), 1.0f), 1.0f);
  R[4] = fma_(v, sub_(mul_(y, y), 1.0f), 1.0f);
  R[8] = fma_(v, sub_(mul_(z, z), 1.0f), 1.0f);
  float xy = mul_(v, mul_(x, y)), xz = mul_(v, mul_(x, z)), yz = mul_(v, mul_(y, z));
  float sx = mul_(s, x), sy = mul_(s, y), sz = mul_(s, z);
  R[1] = sub_(xy, sz); R[3] = add_(xy, sz);
  R[2] = add_(xz, sy); R[6] = sub_(xz, sy);
  R[5] = sub_(yz, sx); R[7] = add_(yz, sx);
}

__device__ inline void matmul3(const float A[9], const float B[9], float C[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = fma_(A[3 * i], B[j], fma_(A[3 * i + 1], B[3 + j], mul_(A[3 * i + 2], B[6 + j])));
}

__device__ inline void matvec3(const float A[9], const float v[3], float out[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = fma_(A[3 * i], v[0], fma_(A[3 * i + 1], v[1], mul_(A[3 * i + 2], v[2])));
}

// Frame of link l >= 1 from its parent's frame: T_l = T_par * T_fix_l * Rot(axis_l, theta).
__device__ inline void link_frame(const HandDev& H, int l, const Frame& par, float theta, Frame& out) {
  float Rf[9], Rj[9], tmp[9], tf[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Rf[3 * i] = H.T_fix[l][4 * i];
    Rf[3 * i + 1] = H.T_fix[l][4 * i + 1];
    Rf[3 * i + 2] = H.T_fix[l][4 * i + 2];
    tf[i] = H.T_fix[l][4 * i + 3];
  }
  axis_rot(H.axis[l], theta, Rj);
  matmul3(par.R, Rf, tmp);
  matmul3(tmp, Rj, out.R);
  float d[3];
  matvec3(par.R, tf, d);
  out.o[0] = add_(par.o[0], d[0]);
  out.o[1] = add_(par.o[1], d[1]);
  out.o[2] = add_(par.o[2], d[2]);
}

__device__ inline void root_frame(const float* q, Frame& out) {
  float w[3] = {q[3], q[4], q[5]};
  so3_exp(w, out.R);
  out.o[0] = q[0];
  out.o[1] = q[1];
  out.o[2] = q[2];
}

// Point in world coordinates: p = R s + o.
__device__ __forceinline__ void transform_point(const float* R, const float* o, float sx, float sy, float sz,
                                                float p[3]) {
  p[0] = fma_(R[0], sx, fma_(R[1], sy, fma_(R[2], sz, o[0])));
  p[1] = fma_(R[3], sx, fma_(R[4], sy, fma_(R[5], sz, o[1])));
  p[2] = fma_(R[6], sx, fma_(R[7], sy, fma_(R[8], sz, o[2])));
}

// ------------------------------------------------------------------------- SDF

// Result of one grid lookup (V = float: one point; float2: two points).  g is
// the gradient of the undilated SDF; hxy, hxz, hyz the mixed second derivatives
// of the trilinear part (zero on clamped axes); when the point lies outside the
// grid, eh = (u - u_c)/|u - u_c| and e the excess distance.
template <class V>
struct SdfSampleT {
  V phi;
  V g[3];
  V hxy, hxz, hyz;
  V eh[3];
  V e;
  V curv;          // mesh objects: s / |p - r*_rho| (curvature of the Phong SDF about r*_rho); 0 for grids
  mask_t<V> outside;
};
using SdfSample = SdfSampleT<float>;

// The lookup in three parts, so that a sweep can issue the next point's corner
// loads before it computes the current point: sdf_index (cell and fractions),
// sdf_gather (the 8 corner values), sdf_finish (value, gradient, curvature).
struct SdfIndex {
  float f[3], du[3];
  bool clamped[3];
  const float* cell;   // corner (i0, j0, k0)
};

__device__ __forceinline__ void sdf_index(const ObjDev& O, const float p[3], SdfIndex& ix) {
  const float n_max[3] = {(float)(O.nx - 1), (float)(O.ny - 1), (float)(O.nz - 1)};
  int i0[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = fma_(p[k], O.inv_h, O.uo[k]);
    const float uc = fminf(fmaxf(u, 0.0f), n_max[k]);     // NaN -> 0
    ix.clamped[k] = uc != u;
    ix.du[k] = sub_(u, uc);                               // 0 unless clamped
    const int ii = __float2int_rd(uc);                   // floor (uc >= 0)
    const int cap = (int)n_max[k] - 1;
    i0[k] = ii < cap ? ii : cap;
    ix.f[k] = sub_(uc, (float)i0[k]);
  }
  // fewer than 2^31 nodes per grid (checked at creation): the index fits 32 bits
  ix.cell = O.grid + (unsigned)((i0[2] * O.ny + i0[1]) * O.nx + i0[0]);
}

__device__ __forceinline__ void sdf_gather(const ObjDev& O, const float* G, float c[8]) {
  const int sy = O.nx, sz = O.nx * O.ny;
  c[0] = __ldg(G);
  c[1] = __ldg(G + 1);
  c[2] = __ldg(G + sy);
  c[3] = __ldg(G + sy + 1);
  c[4] = __ldg(G + sz);
  c[5] = __ldg(G + sz + 1);
  c[6] = __ldg(G + sz + sy);
  c[7] = __ldg(G + sz + sy + 1);
}

__device__ __forceinline__ float rsqrt_or_zero(float x) { return x > 0.0f ? rsqrtf(x) : 0.0f; }
__device__ __forceinline__ float rcp_or_zero(float x) { return x > 0.0f ? __fdividef(1.0f, x) : 0.0f; }
// Reciprocal of a positive, normal float (the effective inverse masses w_n, w_t
// >= 1/m of the simulation adjoint): the hardware approximation, one instruction.
__device__ __forceinline__ float rcp_fast(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Value, gradient and (kHess) mixed second derivatives from the fractions f, the
// excess du = u - u_c, the clamp flags and the corners
// c = (c000, c100, c010, c110, c001, c101, c011, c111).
template <bool kHess, class V>
__device__ __forceinline__ void sdf_finish_v(const ObjDev& O, const V f[3], const V du[3], const mask_t<V> cl[3],
                                             const V c[8], SdfSampleT<V>& s) {
  // trilinear in differences: x first, then y, then z
  const V dx00 = vsub(c[1], c[0]), dx10 = vsub(c[3], c[2]), dx01 = vsub(c[5], c[4]), dx11 = vsub(c[7], c[6]);
  const V x00 = vfma(f[0], dx00, c[0]), x10 = vfma(f[0], dx10, c[2]);
  const V x01 = vfma(f[0], dx01, c[4]), x11 = vfma(f[0], dx11, c[6]);
  const V dy0 = vsub(x10, x00), dy1 = vsub(x11, x01);
  const V y0 = vfma(f[1], dy0, x00), y1 = vfma(f[1], dy1, x01);
  const V dz = vsub(y1, y0);
  const V val = vfma(f[2], dz, y0);
  const V ey0 = vsub(dx10, dx00), ey1 = vsub(dx11, dx01);
  const V a0 = vfma(f[1], ey0, dx00), a1 = vfma(f[1], ey1, dx01);
  const V dax = vsub(a1, a0);
  const V gx = vfma(f[2], dax, a0);             // d/dfx
  const V ddy = vsub(dy1, dy0);
  const V gy = vfma(f[2], ddy, dy0);            // d/dfy
  const V gz = dz;                              // d/dfz
  const V zero = vsplat<V>(0.0f), ih = vsplat<V>(O.inv_h);
  s.g[0] = vsel(cl[0], zero, vmul(gx, ih));
  s.g[1] = vsel(cl[1], zero, vmul(gy, ih));
  s.g[2] = vsel(cl[2], zero, vmul(gz, ih));
  if (kHess) {
    const V ih2 = vsplat<V>(mul_(O.inv_h, O.inv_h));
    const V hxy = vfma(f[2], vsub(ey1, ey0), ey0);
    s.hxy = vsel(mor(cl[0], cl[1]), zero, vmul(hxy, ih2));
    s.hxz = vsel(mor(cl[0], cl[2]), zero, vmul(dax, ih2));
    s.hyz = vsel(mor(cl[1], cl[2]), zero, vmul(ddy, ih2));
  }
  s.outside = mor(mor(cl[0], cl[1]), cl[2]);
  s.curv = zero;
  s.e = zero;
  s.eh[0] = s.eh[1] = s.eh[2] = zero;
  if (many(s.outside)) {
    // du is exactly 0 on unclamped axes, so points inside the grid get eh = 0, e = 0
    const V dn2 = vfma(du[0], du[0], vfma(du[1], du[1], vmul(du[2], du[2])));
    const V r = vmap(dn2, rsqrt_or_zero);
    const V dn = vmul(dn2, r);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      s.eh[k] = vmul(du[k], r);
      s.g[k] = vsel(s.outside, vadd(s.g[k], s.eh[k]), s.g[k]);
    }
    s.e = vmul(vsplat<V>(O.h), dn);
  }
  s.phi = vadd(val, s.e);
}

template <bool kHess>
__device__ __forceinline__ void sdf_finish(const ObjDev& O, const SdfIndex& ix, const float c[8], SdfSample& s) {
  sdf_finish_v<kHess, float>(O, ix.f, ix.du, ix.clamped, c, s);
}

// Two lookups in packed form (points a and b).
__device__ __forceinline__ void sdf_finish_pair(const ObjDev& O, const SdfIndex& ia, const SdfIndex& ib,
                                                const float ca[8], const float cb[8], SdfSampleT<float2>& s) {
  float2 f[3], du[3], c[8];
  bool2 cl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    f[k] = make_float2(ia.f[k], ib.f[k]);
    du[k] = make_float2(ia.du[k], ib.du[k]);
    cl[k] = bool2{ia.clamped[k], ib.clamped[k]};
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k] = make_float2(ca[k], cb[k]);
  sdf_finish_v<true, float2>(O, f, du, cl, c, s);
}


// Lower bound of the interpolated SDF at p from one entry of the min-pyramid: the
// block of 2^lev cells (level 2 when the grid has it) holding p's cell, the cell
// sdf_index picks.  The interpolant in a cell is a convex combination of its
// corners and the excess distance outside the grid is non-negative, so
// phi(p) >= the block's minimum.
__device__ __forceinline__ float point_min_bound(const ObjDev& O, const float p[3]) {
  const int lev = O.pyr_levels >= 2 ? 2 : 1;
  const float n_max[3] = {(float)(O.nx - 1), (float)(O.ny - 1), (float)(O.nz - 1)};
  const int n[3] = {O.nx, O.ny, O.nz};
  int b[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = fma_(p[k], O.inv_h, O.uo[k]);
    const float uc = fminf(fmaxf(u, 0.0f), n_max[k]);      // NaN -> 0
    const int ii = __float2int_rd(uc);
    const int cap = n[k] - 2;
    b[k] = (ii < cap ? ii : cap) >> lev;
  }
  const int bx = ((n[0] - 1) + (1 << lev) - 1) >> lev, by = ((n[1] - 1) + (1 << lev) - 1) >> lev;
  return __ldg(O.pyr + O.pyr_off[lev - 1] + (unsigned)((b[2] * by + b[1]) * bx + b[0]));
}

// Lower bound of the interpolated SDF over every point whose index coordinates
// lie in the box [lo, hi] (any values; clamped to the grid, which also covers
// points outside it since the excess distance is non-negative).  Uses the finest
// pyramid level at which the box spans at most 3 blocks per axis.
__device__ inline float region_min(const ObjDev& O, const float lo[3], const float hi[3]) {
  const int n[3] = {O.nx, O.ny, O.nz};
  int c0[3], c1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float cap = (float)(n[k] - 2);
    const float a = fminf(fmaxf(lo[k], 0.0f), cap), b = fminf(fmaxf(hi[k], 0.0f), cap);
    c0[k] = (int)floorf(a);
    c1[k] = (int)floorf(b);
  }
  int lev = 1;
  for (; lev < O.pyr_levels; ++lev) {
    if ((c1[0] >> lev) - (c0[0] >> lev) <= 2 && (c1[1] >> lev) - (c0[1] >> lev) <= 2 &&
        (c1[2] >> lev) - (c0[2] >> lev) <= 2)
      break;
  }
  const int bx = ((n[0] - 1) + (1 << lev) - 1) >> lev, by = ((n[1] - 1) + (1 << lev) - 1) >> lev;
  const float* L = O.pyr + O.pyr_off[lev - 1];
  int b0[3], b1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b0[k] = c0[k] >> lev;
    b1[k] = c1[k] >> lev;   // b1 - b0 <= 2 except at the coarsest level of a huge grid
  }
  // 27 independent loads; a block index past b1 repeats b1 (same minimum)
  float m = 3.0e38f;
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int x = min(b0[0] + dx, b1[0]), y = min(b0[1] + dy, b1[1]), z = min(b0[2] + dz, b1[2]);
        m = fminf(m, __ldg(L + ((size_t)z * by + y) * bx + x));
      }
  // a grid larger than 2^kMaxPyrLevels cells per axis can leave more than 3 blocks
  if (b1[0] - b0[0] > 2 || b1[1] - b0[1] > 2 || b1[2] - b0[2] > 2) {
    for (int z = b0[2]; z <= b1[2]; ++z)
      for (int y = b0[1]; y <= b1[1]; ++y)
        for (int x = b0[0]; x <= b1[0]; ++x) m = fminf(m, __ldg(L + ((size_t)z * by + y) * bx + x));
  }
  return m;
}

// ------------------------------------------------------------------ contact sims
//
// Simulation m has test velocity v_m = sgn_m * V * e_{ax_m} (m = 0: v = 0).
__device__ __forceinline__ int sim_axis(int m) { return (m - 1) >> 1; }
__device__ __forceinline__ float sim_sign(int m) { return (m & 1) ? 1.0f : -1.0f; }

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
  c[0] = fma_(a[1], b[2], -mul_(a[2], b[1]));
  c[1] = fma_(a[2], b[0], -mul_(a[0], b[2]));
  c[2] = fma_(a[0], b[1], -mul_(a[1], b[0]));
}
__device__ __forceinline__ float dot3(const float a[3], const float b[3]) {
  return fma_(a[0], b[0], fma_(a[1], b[1], mul_(a[2], b[2])));
}

// ----------------------------------------------------------------- mesh SDF
//
// Sec. III-B: phi(r) = s |r - r*| with r* the closest point on the mesh and s the
// inside/outside sign; the Phong SDF rho(r) = s |r - r*_rho| replaces r* by the
// point of the Phong-tessellated surface, r*_rho = (1 - a) r* + a sum_x b_x psi_x(r*),
// psi_x(q) = q - ((q - v_x) . n_x) n_x, with (b_a, b_b, b_c) the barycentric
// coordinates of r* on its face and n_x the vertex normals; grad rho =
// s (r - r*_rho)/|r - r*_rho| (r*_rho held fixed, as the paper gives it).  The sign is
// that of (r - r*) . N with N the angle-weighted pseudonormal of the closest
// feature (face, edge or vertex), which on a watertight mesh matches the ray
// test without a second search.

// Closest point of p on triangle (a, b, c) by the Voronoi regions of its
// vertices, edges and face: barycentric coordinates and the feature
// (0 face, 1 edge ab, 2 edge bc, 3 edge ca, 4/5/6 vertex a/b/c).
__device__ __forceinline__ float closest_on_triangle(const float p[3], const float a[3], const float b[3],
                                                     const float c[3], float bary[3], int& feature) {
  float ab[3], ac[3], ap[3], bp[3], cp[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ab[k] = b[k] - a[k];
    ac[k] = c[k] - a[k];
    ap[k] = p[k] - a[k];
    bp[k] = p[k] - b[k];
    cp[k] = p[k] - c[k];
  }
  const float d1 = dot3(ab, ap), d2 = dot3(ac, ap), d3 = dot3(ab, bp), d4 = dot3(ac, bp);
  const float d5 = dot3(ab, cp), d6 = dot3(ac, cp);
  const float vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
  float u, v, w;
  if (d1 <= 0.0f && d2 <= 0.0f) {
    u = 1.0f; v = 0.0f; w = 0.0f; feature = 4;
  } else if (d3 >= 0.0f && d4 <= d3) {
    u = 0.0f; v = 1.0f; w = 0.0f; feature = 5;
  } else if (vc <= 0.0f && d1 >= 0.0f && d3 <= 0.0f) {
    v = d1 / (d1 - d3); u = 1.0f - v; w = 0.0f; feature = 1;
  } else if (d6 >= 0.0f && d5 <= d6) {
    u = 0.0f; v = 0.0f; w = 1.0f; feature = 6;
  } else if (vb <= 0.0f && d2 >= 0.0f && d6 <= 0.0f) {
    w = d2 / (d2 - d6); u = 1.0f - w; v = 0.0f; feature = 3;
  } else if (va <= 0.0f && (d4 - d3) >= 0.0f && (d5 - d6) >= 0.0f) {
    w = (d4 - d3) / ((d4 - d3) + (d5 - d6)); v = 1.0f - w; u = 0.0f; feature = 2;
  } else {
    const float den = 1.0f / (va + vb + vc);
    v = vb * den; w = vc * den; u = 1.0f - v - w; feature = 0;
  }
  bary[0] = u; bary[1] = v; bary[2] = w;
  float d2sum = 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float q = u * a[k] + v * b[k] + w * c[k];
    d2sum += (p[k] - q) * (p[k] - q);
  }
  return d2sum;
}

__device__ __forceinline__ float box_dist2(const float p[3], const float4& lo, const float4& hi) {
  const float dx = fmaxf(fmaxf(lo.x - p[0], p[0] - hi.x), 0.0f);
  const float dy = fmaxf(fmaxf(lo.y - p[1], p[1] - hi.y), 0.0f);
  const float dz = fmaxf(fmaxf(lo.z - p[2], p[2] - hi.z), 0.0f);
  return dx * dx + dy * dy + dz * dz;
}

constexpr int kBvhStack = 64;

// The mesh searches below are called out of line (one copy per kernel): inlined
// at every lookup site of the fused kernel they overflowed the instruction cache
// (ncu: 42% of the stall samples waiting for an instruction fetch).

// Closest face of the mesh to p: depth-first over the BVH, nearer child first,
// subtrees farther than the best distance found so far skipped.  A face known to
// be at squared distance init_d2 (init >= 0, with bary and feature set for it)
// bounds the search from the start.
static __device__ __noinline__ int mesh_closest(const ObjDev& O, const float p[3], float bary[3], int& feature, int init = -1,
                                   float init_d2 = 3.0e38f) {
  int stack[kBvhStack];
  int sp = 0, node = 0, best = init;
  float best_d2 = init >= 0 ? init_d2 : 3.0e38f;
  for (;;) {
    const float4 lo = __ldg(O.bvh + 2 * node), hi = __ldg(O.bvh + 2 * node + 1);
    const int count = __float_as_int(hi.w);
    if (count > 0) {
      const int first = __float_as_int(lo.w);
      for (int f = first; f < first + count; ++f) {
        const float4 A = __ldg(O.tri + 3 * f), B = __ldg(O.tri + 3 * f + 1), C = __ldg(O.tri + 3 * f + 2);
        const float a[3] = {A.x, A.y, A.z}, b[3] = {B.x, B.y, B.z}, c[3] = {C.x, C.y, C.z};
        float bb[3];
        int ft;
        const float d2 = closest_on_triangle(p, a, b, c, bb, ft);
        if (d2 < best_d2) {
          best_d2 = d2;
          best = f;
          bary[0] = bb[0]; bary[1] = bb[1]; bary[2] = bb[2];
          feature = ft;
        }
      }
    } else {
      const int l = node + 1, r = __float_as_int(lo.w);
      const float dl = box_dist2(p, __ldg(O.bvh + 2 * l), __ldg(O.bvh + 2 * l + 1));
      const float dr = box_dist2(p, __ldg(O.bvh + 2 * r), __ldg(O.bvh + 2 * r + 1));
      const int nearc = dl <= dr ? l : r, farc = dl <= dr ? r : l;
      const float dn = fminf(dl, dr), df = fmaxf(dl, dr);
      if (df < best_d2 && sp < kBvhStack) stack[sp++] = farc;
      if (dn < best_d2) {
        node = nearc;
        continue;
      }
    }
    // next subtree still worth visiting
    bool found = false;
    while (sp > 0) {
      const int cand = stack[--sp];
      if (box_dist2(p, __ldg(O.bvh + 2 * cand), __ldg(O.bvh + 2 * cand + 1)) < best_d2) {
        node = cand;
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  return best;
}

// The same search for the 32 points of a warp at once (every lane must call it):
// the warp walks one path through the BVH, descending into a node while some
// lane's box distance is below that lane's best, and every lane tests every
// triangle of a visited leaf against its own point.  The points of a warp lie
// close together, so the union of the lanes' paths is short, and the walk does
// not diverge.  The result per lane is the closest face, as in mesh_closest
// (up to the choice among faces at exactly equal distance, which share the
// closest edge or vertex).
// Lanes with done set take part without searching (their result is -1); init
// and init_d2 bound a lane's search as in mesh_closest.
static __device__ __noinline__ int mesh_closest_warp(const ObjDev& O, const float p[3], float bary[3], int& feature,
                                        bool done = false, int init = -1, float init_d2 = 3.0e38f) {
  int stack[kBvhStack];
  int sp = 0, node = 0, best = done ? -1 : init;
  float best_d2 = done ? -1.0f : (init >= 0 ? init_d2 : 3.0e38f);
  for (;;) {
    const float4 lo = __ldg(O.bvh + 2 * node), hi = __ldg(O.bvh + 2 * node + 1);
    const int count = __float_as_int(hi.w);
    if (count > 0) {
      const int first = __float_as_int(lo.w);
      for (int f = first; f < first + count; ++f) {
        const float4 A = __ldg(O.tri + 3 * f), B = __ldg(O.tri + 3 * f + 1), C = __ldg(O.tri + 3 * f + 2);
        const float a[3] = {A.x, A.y, A.z}, b[3] = {B.x, B.y, B.z}, c[3] = {C.x, C.y, C.z};
        float bb[3];
        int ft;
        const float d2 = closest_on_triangle(p, a, b, c, bb, ft);
        if (d2 < best_d2) {
          best_d2 = d2;
          best = f;
          bary[0] = bb[0]; bary[1] = bb[1]; bary[2] = bb[2];
          feature = ft;
        }
      }
    } else {
      const int l = node + 1, r = __float_as_int(lo.w);
      const float dl = box_dist2(p, __ldg(O.bvh + 2 * l), __ldg(O.bvh + 2 * l + 1));
      const float dr = box_dist2(p, __ldg(O.bvh + 2 * r), __ldg(O.bvh + 2 * r + 1));
      const bool need_l = __any_sync(0xffffffffu, dl < best_d2);
      const bool need_r = __any_sync(0xffffffffu, dr < best_d2);
      // nearer child first: the one nearer for most lanes
      const bool left_first = __popc(__ballot_sync(0xffffffffu, dl <= dr)) >= 16;
      const int nearc = left_first ? l : r, farc = left_first ? r : l;
      const bool need_near = left_first ? need_l : need_r, need_far = left_first ? need_r : need_l;
      if (need_near && need_far && sp < kBvhStack) stack[sp++] = farc;
      if (need_near) {
        node = nearc;
        continue;
      }
      if (need_far) {
        node = farc;
        continue;
      }
    }
    bool found = false;
    while (sp > 0) {
      const int cand = stack[--sp];
      if (__any_sync(0xffffffffu, box_dist2(p, __ldg(O.bvh + 2 * cand), __ldg(O.bvh + 2 * cand + 1)) < best_d2)) {
        node = cand;
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  return best;
}

// ------------------------------------------------- certified local search
//
// The mesh solid lies inside the half-space of every face on its convex hull.  At
// a point q of the surface whose incident faces are all hull faces, the hull's
// tangent cone is the cone of the incident edges, so if p - q lies in its normal
// cone ((p - q) . e <= 0 for every edge direction e out of q) q is the closest point
// of the hull to p, and, being on the mesh, the closest point of the mesh.  The
// search starts from the closest face at the nearest node of a coarse grid and
// moves to a neighbouring face while one is strictly closer: across the edge
// holding the closest point, or, from a vertex, to the closer of the two faces on
// the edge along which the distance falls fastest.  A point inside the mesh, a
// feature off the hull, or a walk that stops without a certificate is left to the
// BVH walk.  Edge directions within 1e-6 (relative) of the cone's boundary pass
// (cone_violated); moves are taken by the gain in squared distance computed from
// the difference of the two points (closer_by).

constexpr int kLocalHops = 16;

// Index of the start face for p (-1 when p is not finite).
__device__ __forceinline__ int mesh_start(const ObjDev& O, const float p[3]) {
  if (!(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]))) return -1;
  int idx[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = (p[k] - O.start_org[k]) * O.start_inv_h;
    idx[k] = __float2int_rn(fminf(fmaxf(u, 0.0f), (float)(O.start_n[k] - 1)));
  }
  return __ldg(O.start_face + (idx[2] * O.start_n[1] + idx[1]) * O.start_n[0] + idx[0]);
}

// Closest point of face f to p: squared distance, barycentric coordinates,
// feature, the point, and the faces across the three edges.
static __device__ __noinline__ float face_closest(const ObjDev& O, int f, const float p[3], float bary[3], int& feature,
                                              float q[3], int nb[3]) {
  const float4 A = __ldg(O.tri + 3 * f), B = __ldg(O.tri + 3 * f + 1), C = __ldg(O.tri + 3 * f + 2);
  const float a[3] = {A.x, A.y, A.z}, b[3] = {B.x, B.y, B.z}, c[3] = {C.x, C.y, C.z};
  nb[0] = __float_as_int(A.w);
  nb[1] = __float_as_int(B.w);
  nb[2] = __float_as_int(C.w);
  const float d2 = closest_on_triangle(p, a, b, c, bary, feature);
#pragma unroll
  for (int k = 0; k < 3; ++k) q[k] = bary[0] * a[k] + bary[1] * b[k] + bary[2] * c[k];
  return d2;
}

// (p - q) . e > 0 beyond 1e-6 of |p - q| |e|: moving along e from q gets closer.
// Below that the closest point along e is within 1e-6 |p - q| of q.
__device__ __forceinline__ bool cone_violated(const float r[3], const float e[3]) {
  const float re = dot3(r, e);
  return re > 0.0f && re * re > 1e-12f * dot3(r, r) * dot3(e, e);
}

// |p - q|^2 - |p - q'|^2 = (q' - q) . (r + r'), r = p - q, r' = p - q': the gain of
// moving from q to q', from the difference of the points (no cancellation between
// two nearly equal squared distances, so float32 resolves gains far below |p - q|^2).
__device__ __forceinline__ float closer_by(const float q[3], const float r[3], const float q2[3], const float p[3]) {
  return (q2[0] - q[0]) * (r[0] + p[0] - q2[0]) + (q2[1] - q[1]) * (r[1] + p[1] - q2[1]) +
         (q2[2] - q[2]) * (r[2] + p[2] - q2[2]);
}

// The local search from face f: true when certified.  face, bary, feature and d2
// describe the last face reached (face = -1 when p is too far for the test), the
// closest one when certified.
static __device__ __noinline__ bool mesh_local(const ObjDev& O, const float p[3], int f, float bary[3], int& feature, float& d2,
                                  int& face) {
  float q[3];
  int nb[3];
  face = -1;
  d2 = face_closest(O, f, p, bary, feature, q, nb);
  if (!(d2 < 1e30f)) return false;
  for (int hop = 0; hop < kLocalHops; ++hop) {
    face = f;
    const float r[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
    int g = -1;
    if (feature == 0) {
      const float4 N = __ldg(O.face_nrm + 7 * f + 3);
      return (__float_as_int(N.w) & 1) && r[0] * N.x + r[1] * N.y + r[2] * N.z >= 0.0f;
    } else if (feature <= 3) {
      const int k = feature - 1;
      const float4 W = __ldg(O.wing + 3 * f + k);
      const float e[3] = {W.x - q[0], W.y - q[1], W.z - q[2]};
      if (!cone_violated(r, e)) return __float_as_int(W.w) & 1;
      g = nb[k];
      float gb[3], gq[3];
      int gf, gn[3];
      const float gd2 = face_closest(O, g, p, gb, gf, gq, gn);
      if (!(closer_by(q, r, gq, p) > 0.0f)) return false;
      d2 = gd2;
      feature = gf;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        bary[t] = gb[t];
        q[t] = gq[t];
        nb[t] = gn[t];
      }
      f = g;
    } else {
      const int k = feature - 4;
      const int b0 = __float_as_int(__ldg(O.face_nrm + 7 * f + k).w);
      const int info = __float_as_int(__ldg(O.face_nrm + 7 * f + 4 + k).w);
      const int m = info & ((1 << 29) - 1);
      // the edge out of the vertex along which the distance falls fastest
      int bi = -1;
      float bre = 0.0f, be2 = 1.0f;
#pragma unroll 2
      for (int i = 0; i < m; ++i) {
        const float4 U = __ldg(O.ring + b0 + i);
        const float e[3] = {U.x - q[0], U.y - q[1], U.z - q[2]};
        if (cone_violated(r, e)) {
          const float re = dot3(r, e), e2 = dot3(e, e);
          if (bi < 0 || re * re * be2 > bre * bre * e2) {
            bi = i;
            bre = re;
            be2 = e2;
          }
        }
      }
      if (bi < 0) return (info >> 30) & 1;
      if (!((info >> 29) & 1)) return false;
      // the two faces on that edge: ring entries bi and bi - 1 (fan order)
      const int h0 = __float_as_int(__ldg(O.ring + b0 + bi).w);
      const int h1 = __float_as_int(__ldg(O.ring + b0 + (bi > 0 ? bi - 1 : m - 1)).w);
      float bd2 = d2, gain = 0.0f, bq[3] = {q[0], q[1], q[2]};
#pragma unroll 1
      for (int t2 = 0; t2 < 2; ++t2) {
        const int h = t2 == 0 ? h0 : h1;
        if (h == f) continue;
        float hb[3], hq[3];
        int hf, hn[3];
        const float hd2 = face_closest(O, h, p, hb, hf, hq, hn);
        const float gh = closer_by(q, r, hq, p);
        if (gh > gain) {
          gain = gh;
          bd2 = hd2;
          g = h;
          feature = hf;
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            bary[t] = hb[t];
            bq[t] = hq[t];
            nb[t] = hn[t];
          }
        }
      }
      if (g < 0) return false;
#pragma unroll
      for (int t = 0; t < 3; ++t) q[t] = bq[t];
      d2 = bd2;
      f = g;
    }
  }
  face = f;
  return false;
}

// Signed distance from p to the flat mesh (sign by the closest feature's
// pseudonormal, as in mesh_lookup); +inf when p is not finite.
__device__ inline float mesh_flat_distance(const ObjDev& O, const float p[3]) {
  float bary[3], d2 = 3.0e38f;
  int feature = 0, f = -1;
  const int f0 = mesh_start(O, p);
  if (!(f0 >= 0 && mesh_local(O, p, f0, bary, feature, d2, f))) f = mesh_closest(O, p, bary, feature, f, d2);
  if (f < 0) return 3.0e38f;
  const float4 A = __ldg(O.tri + 3 * f), B = __ldg(O.tri + 3 * f + 1), C = __ldg(O.tri + 3 * f + 2);
  const float q[3] = {bary[0] * A.x + bary[1] * B.x + bary[2] * C.x, bary[0] * A.y + bary[1] * B.y + bary[2] * C.y,
                      bary[0] * A.z + bary[1] * B.z + bary[2] * C.z};
  const int slot = feature == 0 ? 3 : (feature <= 3 ? 3 + feature : feature - 4);
  const float4 N = __ldg(O.face_nrm + 7 * f + slot);
  const float dq[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
  const float dist = sqrtf(dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2]);
  return dq[0] * N.x + dq[1] * N.y + dq[2] * N.z < 0.0f ? -dist : dist;
}

// Phong SDF at p for the 32 points of a warp (every lane must call it): the
// certified local search per lane, the warp's BVH walk for the lanes it leaves.
static __device__ __noinline__ void mesh_lookup(const ObjDev& O, const float p[3], SdfSample& s) {
  float bary[3], fd2 = 3.0e38f;
  int feature = 0, f = -1;
  const int f0 = mesh_start(O, p);
  const bool done = f0 >= 0 && mesh_local(O, p, f0, bary, feature, fd2, f);
  if (!__all_sync(0xffffffffu, done)) {
    // the lanes left search the BVH, bounded by the face their local search reached
    const int wf = mesh_closest_warp(O, p, bary, feature, done, f, fd2);
    if (!done) f = wf;
  }
  if (f < 0) {                                  // p not finite: no face compares closer
    const float nan = __int_as_float(0x7fc00000);
    s.phi = s.curv = s.e = nan;
    s.g[0] = s.g[1] = s.g[2] = nan;
    s.eh[0] = s.eh[1] = s.eh[2] = 0.0f;
    s.hxy = s.hxz = s.hyz = 0.0f;
    s.outside = false;
    return;
  }
  const float4 A = __ldg(O.tri + 3 * f), B = __ldg(O.tri + 3 * f + 1), C = __ldg(O.tri + 3 * f + 2);
  const float4* X = O.face_nrm + 7 * f;
  const float4 na = __ldg(X), nb = __ldg(X + 1), nc = __ldg(X + 2);
  const float v[3][3] = {{A.x, A.y, A.z}, {B.x, B.y, B.z}, {C.x, C.y, C.z}};
  const float n[3][3] = {{na.x, na.y, na.z}, {nb.x, nb.y, nb.z}, {nc.x, nc.y, nc.z}};
  float q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) q[k] = bary[0] * v[0][k] + bary[1] * v[1][k] + bary[2] * v[2][k];
  // pseudonormal of the closest feature: face 3, edges 4..6, vertices 0..2
  const int slot = feature == 0 ? 3 : (feature <= 3 ? 3 + feature : feature - 4);
  const float4 N = __ldg(X + slot);
  const float side = (p[0] - q[0]) * N.x + (p[1] - q[1]) * N.y + (p[2] - q[2]) * N.z;
  const float sgn = side < 0.0f ? -1.0f : 1.0f;
  // Phong point
  float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float t = (q[0] - v[j][0]) * n[j][0] + (q[1] - v[j][1]) * n[j][1] + (q[2] - v[j][2]) * n[j][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += bary[j] * (q[k] - t * n[j][k]);
  }
  const float al = O.phong_alpha;
  float diff[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) diff[k] = p[k] - ((1.0f - al) * q[k] + al * acc[k]);
  const float d2 = dot3(diff, diff);
  const float inv = d2 > 0.0f ? rsqrtf(d2) : 0.0f;
  s.phi = sgn * d2 * inv;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.g[k] = sgn * diff[k] * inv;
    s.eh[k] = 0.0f;
  }
  s.hxy = s.hxz = s.hyz = 0.0f;
  s.e = 0.0f;
  s.curv = sgn * inv;
  s.outside = false;
}

// kAnyObj = false compiles the grid lookup alone (callers that only see grids).
// With kAnyObj every lane of the warp must call it (the mesh search is warp-wide).
template <bool kHess, bool kAnyObj = true>
__device__ __forceinline__ void sdf_lookup(const ObjDev& O, const float p[3], SdfSample& s) {
  if constexpr (kAnyObj) {
    if (O.kind == kObjMesh) {
      mesh_lookup(O, p, s);
      return;
    }
  }
  SdfIndex ix;
  sdf_index(O, p, ix);
  float c[8];
  sdf_gather(O, ix.cell, c);
  sdf_finish<kHess>(O, ix, c, s);
}

// Per-point quantities shared by the 7 simulations.
template <class V>
struct PointStateT {
  V p[3];       // world position (= object frame: canonical object pose)
  V n[3];       // unit normal grad/|grad|
  V rg;         // 1/|grad|
  V phi_hat;    // dilated SDF
};
using PointState = PointStateT<float>;

template <class V>
__device__ __forceinline__ void point_state(const SdfSampleT<V>& s, const V p[3], float r_dil, PointStateT<V>& ps) {
  const V g2 = vfma(s.g[0], s.g[0], vfma(s.g[1], s.g[1], vmul(s.g[2], s.g[2])));
  const V rg = vmap(g2, rsqrt_or_zero);
  ps.rg = rg;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ps.p[k] = p[k];
    ps.n[k] = vmul(s.g[k], rg);
  }
  ps.phi_hat = vsub(s.phi, vsplat<V>(r_dil));
}

// Lane l of a packed point state.
__device__ __forceinline__ PointState point_lane(const PointStateT<float2>& ps, int l) {
  PointState o;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    o.p[k] = vlane(ps.p[k], l);
    o.n[k] = vlane(ps.n[k], l);
  }
  o.rg = vlane(ps.rg, l);
  o.phi_hat = vlane(ps.phi_hat, l);
  return o;
}

// Constraint value on the plane through the query for simulation m:
// phi_m = phi_hat - dt n . v_m.
template <class V>
__device__ __forceinline__ V sim_phi(const PointStateT<V>& ps, int m, float dtV) {
  if (m == 0) return ps.phi_hat;
  const int ax = sim_axis(m);
  const V nk = ax == 0 ? ps.n[0] : (ax == 1 ? ps.n[1] : ps.n[2]);
  return vfma(vsplat<V>(-sim_sign(m) * dtV), nk, ps.phi_hat);
}

// Unit direction of test velocity m (zero for m = 0), by selects so that a
// runtime m indexes no local array.
__device__ __forceinline__ void sim_dir(int m, float vd[3]) {
  const int k = (m - 1) >> 1;
  const float sg = sim_sign(m);
  vd[0] = (m > 0 && k == 0) ? sg : 0.0f;
  vd[1] = (m > 0 && k == 1) ? sg : 0.0f;
  vd[2] = (m > 0 && k == 2) ? sg : 0.0f;
}

// Tangential unit vector t = (v - (v.n) n)/|v - (v.n) n| of a moving simulation
// and rho = |e_k - n_k n| = sin(angle(n, v_m)).  rho^2 is the sum of the squares
// of the two other components of n (no cancellation of 1 - n_k^2).  Returns 0
// (and t = 0) when m = 0 or n is parallel to the velocity.
__device__ __forceinline__ float sim_tangent(const float n[3], int m, float t[3]) {
  t[0] = t[1] = t[2] = 0.0f;
  if (m == 0) return 0.0f;
  const int k = (m - 1) >> 1;
  const float sg = sim_sign(m);
  const bool k0 = k == 0, k1 = k == 1, k2 = k == 2;
  const float nk = k0 ? n[0] : (k2 ? n[2] : n[1]);
  const float ea = k0 ? n[1] : n[0];
  const float eb = k2 ? n[1] : n[2];
  const float rho2 = fma_(ea, ea, mul_(eb, eb));
  if (!(rho2 > 0.0f)) return 0.0f;
  const float rr = rsqrtf(rho2);
  const float rho = mul_(rho2, rr);
  const float cc = -sg * nk * rr;
  t[0] = k0 ? sg * rho : cc * n[0];
  t[1] = k1 ? sg * rho : cc * n[1];
  t[2] = k2 ? sg * rho : cc * n[2];
  return rho;
}

// Forward of one contact in simulation m (C > 0): the correction of Eq. (1) as
// a generalised force f = -(lambda_n n + lambda_t t) with lever d = p - x_pred.
// Static friction when sigma <= mu C (sigma = dt V rho, the tangential
// displacement), kinetic otherwise.
__device__ __forceinline__ void contact_force(const PointState& ps, int m, float C, const ParamsDev& P,
                                              const ObjDev& O, float f[3], float d[3]) {
  const float dtV = P.dt * P.V;
  float vd[3];
  sim_dir(m, vd);
  d[0] = fma_(-dtV, vd[0], ps.p[0]);
  d[1] = fma_(-dtV, vd[1], ps.p[1]);
  d[2] = fma_(-dtV, vd[2], ps.p[2]);
  float un[3];
  cross3(d, ps.n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  const float lam_n = C * rcp_fast(wn);       // w_n >= 1/m: a normal float
  f[0] = -lam_n * ps.n[0];
  f[1] = -lam_n * ps.n[1];
  f[2] = -lam_n * ps.n[2];
  float t[3];
  const float rho = sim_tangent(ps.n, m, t);
  if (rho > 0.0f) {
    const float sigma = mul_(dtV, rho);
    float ut[3];
    cross3(d, t, ut);
    const float wt = fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass);
    const float muC = mul_(P.mu, C);
    const float lam_t = (sigma <= muC ? sigma : muC) * rcp_fast(wt);
    f[0] -= lam_t * t[0];
    f[1] -= lam_t * t[1];
    f[2] -= lam_t * t[2];
  }
}

// Adjoint of one simulation at one point (general path, any C).  Inputs: the
// wrench adjoint of the simulation (Gl = dL/dW_lin, Ga = dL/dW_ang), the
// constraint value phi_m and flag kappa.  Accumulates dL/dphi_hat, dL/dn and
// dL/dp (through the lever).  C = max(0, -phi_m) with the leaky rule:
// dC/dphi = -1 in contact, -alpha otherwise (Sec. III-C).
__device__ __forceinline__ void sim_adjoint(const PointState& ps, int m, float phi_m, bool kappa,
                                            const float Gl[3], const float Ga[3], const ParamsDev& P,
                                            const ObjDev& O, float extra_dC, float& d_phi_hat, float dn[3],
                                            float dp[3]) {
  const float dtV = P.dt * P.V;
  float vd[3];
  sim_dir(m, vd);
  const float d[3] = {fma_(-dtV, vd[0], ps.p[0]), fma_(-dtV, vd[1], ps.p[1]), fma_(-dtV, vd[2], ps.p[2])};
  const float C = kappa ? -phi_m : 0.0f;
  // gf = dL/df = Gl + Ga x d
  float gad[3];
  cross3(Ga, d, gad);
  const float gf[3] = {Gl[0] + gad[0], Gl[1] + gad[1], Gl[2] + gad[2]};
  float un[3];
  cross3(d, ps.n, un);
  const float wn = fma_(O.inv_inertia, dot3(un, un), O.inv_mass);
  const float rwn = __fdividef(1.0f, wn);
  const float dlam_n = -dot3(gf, ps.n);
  float dC = dlam_n * rwn + extra_dC;
  float t[3];
  const float rho = sim_tangent(ps.n, m, t);
  float sigma = 0.0f, rwt = 0.0f, dlam_t = 0.0f;
  float ut[3] = {0.0f, 0.0f, 0.0f};
  bool stat = false;
  if (rho > 0.0f) {
    sigma = mul_(dtV, rho);
    cross3(d, t, ut);
    const float wt = fma_(O.inv_inertia, dot3(ut, ut), O.inv_mass);
    rwt = __fdividef(1.0f, wt);
    dlam_t = -dot3(gf, t);
    stat = sigma <= mul_(P.mu, C);
    if (!stat) dC += P.mu * dlam_t * rwt;      // kinetic: lambda_t = mu C / w_t
  }
  if (C > 0.0f) {
    // terms that carry lambda (zero when the point is not in contact)
    const float lam_n = C * rwn;
    const float lam_t = rho > 0.0f ? (stat ? sigma : P.mu * C) * rwt : 0.0f;
    float f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) f[k] = -(lam_n * ps.n[k] + lam_t * t[k]);
    float dd[3];
    cross3(f, Ga, dd);                               // d(d x f).Ga/dd = f x Ga
    float dnl[3] = {-lam_n * gf[0], -lam_n * gf[1], -lam_n * gf[2]};   // f = -lam_n n
    // lam_n = C / w_n, w_n = 1/m + |u_n|^2 / I, u_n = d x n
    const float dwn = -dlam_n * lam_n * rwn;
    const float sn = 2.0f * O.inv_inertia * dwn;
    const float dun[3] = {sn * un[0], sn * un[1], sn * un[2]};
    float tmp[3];
    cross3(ps.n, dun, tmp);                          // d(d x n).dun/dd = n x dun
    dd[0] += tmp[0]; dd[1] += tmp[1]; dd[2] += tmp[2];
    cross3(dun, d, tmp);                             // d(d x n).dun/dn = dun x d
    dnl[0] += tmp[0]; dnl[1] += tmp[1]; dnl[2] += tmp[2];
    if (rho > 0.0f) {
      float dtt[3] = {-lam_t * gf[0], -lam_t * gf[1], -lam_t * gf[2]};   // f = -lam_t t
      const float dsig = stat ? dlam_t * rwt : 0.0f;
      const float dwt = -dlam_t * lam_t * rwt;
      const float st = 2.0f * O.inv_inertia * dwt;
      const float dut[3] = {st * ut[0], st * ut[1], st * ut[2]};
      cross3(t, dut, tmp);
      dd[0] += tmp[0]; dd[1] += tmp[1]; dd[2] += tmp[2];
      cross3(dut, d, tmp);
      dtt[0] += tmp[0]; dtt[1] += tmp[1]; dtt[2] += tmp[2];
      // t = s/sigma, sigma = |s|: ds = (dt - (t.dt) t)/sigma + dsig t
      const float tdt = dot3(t, dtt);
      const float rs = __fdividef(1.0f, sigma);
      float ds[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) ds[k] = (dtt[k] - tdt * t[k]) * rs + dsig * t[k];
      // s = dt V (vd - (vd.n) n): dn += -dt V ((vd.n) ds + (n.ds) vd)
      const float vn = dot3(vd, ps.n), nds = dot3(ps.n, ds);
#pragma unroll
      for (int k = 0; k < 3; ++k) dnl[k] -= dtV * (vn * ds[k] + nds * vd[k]);
    }
    dn[0] += dnl[0]; dn[1] += dnl[1]; dn[2] += dnl[2];
    dp[0] += dd[0]; dp[1] += dd[1]; dp[2] += dd[2];
  }
  // C = max(0, -phi_m), leaky: dphi_m = -dC (contact) or -alpha dC
  const float dphi = kappa ? -dC : -P.alpha * dC;
  d_phi_hat += dphi;
  // phi_m = phi_hat - dt n . v_m
#pragma unroll
  for (int k = 0; k < 3; ++k) dn[k] -= dtV * vd[k] * dphi;
}

// Constants of the simulation adjoint for one candidate step, in shared memory.
// Scalar table (float index):  0 1/m, 1 1/I, 2 c = dt V, 3 c^2, 4 2c/I, 5 mu,
// 6 alpha, 7 alpha c, 8 -c, 9 -mu, 10 -alpha c, 11 -w_pen, 12 w_pen.  The packed
// table holds each entry twice (a float2 per entry), so that a packed operand is
// one shared-memory load.
enum SimConst { kcA = 0, kcB, kcC, kcCC, kcTBC, kcMu, kcAlpha, kcAlphaC, kcMC, kcMMu, kcMAlphaC, kcMWpen, kcWpen,
                kcCount };
struct SimConsts {
  float s[16];
  float2 p[16];
};
__device__ __forceinline__ void sim_constants(const ParamsDev& P, const ObjDev& O, SimConsts& K) {
  const float c = P.dt * P.V;
  const float v[kcCount] = {O.inv_mass, O.inv_inertia, c, c * c, 2.0f * c * O.inv_inertia, P.mu, P.alpha,
                            P.alpha * c, -c, -P.mu, -P.alpha * c, -P.w_pen, P.w_pen};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float x = k < kcCount ? v[k] : 0.0f;
    K.s[k] = x;
    K.p[k] = make_float2(x, x);
  }
}
__device__ __forceinline__ float simk(const SimConsts& K, float, int k) { return K.s[k]; }
__device__ __forceinline__ float2 simk(const SimConsts& K, float2, int k) { return K.p[k]; }

// Wrench adjoint of simulation m, (dL/dW_lin, dL/dW_ang), in shared memory:
// scalar as (Gl, 0), (Ga, 0); packed with every component twice.
struct SimAdjoints {
  float4 s[kSims][2];
  float4 p[kSims][3];
};
__device__ __forceinline__ void set_sim_adjoint(SimAdjoints& G, int m, const float gl[3], const float ga[3]) {
  G.s[m][0] = make_float4(gl[0], gl[1], gl[2], 0.0f);
  G.s[m][1] = make_float4(ga[0], ga[1], ga[2], 0.0f);
  G.p[m][0] = make_float4(gl[0], gl[0], gl[1], gl[1]);
  G.p[m][1] = make_float4(gl[2], gl[2], ga[0], ga[0]);
  G.p[m][2] = make_float4(ga[1], ga[1], ga[2], ga[2]);
}
__device__ __forceinline__ void get_sim_adjoint(const SimAdjoints& G, int m, float gl[3], float ga[3]) {
  const float4 a = G.s[m][0], b = G.s[m][1];
  gl[0] = a.x; gl[1] = a.y; gl[2] = a.z;
  ga[0] = b.x; ga[1] = b.y; ga[2] = b.z;
}
__device__ __forceinline__ void get_sim_adjoint(const SimAdjoints& G, int m, float2 gl[3], float2 ga[3]) {
  const float4 a = G.p[m][0], b = G.p[m][1], c = G.p[m][2];
  gl[0] = make_float2(a.x, a.y); gl[1] = make_float2(a.z, a.w);
  gl[2] = make_float2(b.x, b.y); ga[0] = make_float2(b.z, b.w);
  ga[1] = make_float2(c.x, c.y); ga[2] = make_float2(c.z, c.w);
}

// gl . a + ga . b, as two independent 3-term chains (shorter dependency path)
template <class V>
__device__ __forceinline__ V dot6(const V gl[3], const V a[3], const V ga[3], const V b[3]) {
  return vadd(vfma(gl[0], a[0], vfma(gl[1], a[1], vmul(gl[2], a[2]))),
              vfma(ga[0], b[0], vfma(ga[1], b[1], vmul(ga[2], b[2]))));
}

// Adjoint of all 7 simulations at one point (V = float) or two points (float2).
// A simulation whose constraint is active (phi_m < 0) takes the general path
// (sim_adjoint, per point).  An inactive one has C = 0, so only the leaky slope
// survives:
//   dC = -(gf.n)/w_n - mu (gf.t)/w_t   (kinetic branch, sigma > mu C = 0),
//   dphi_m = -alpha dC,
// with gf = Gl_m + Ga_m x d_m, d_m = p - s c e_k, t = s tau_k.  Every term is
// expanded around quantities shared by the simulations of the point:
//   d x n   = U - s c E_k,      U = p x n,     E_k = e_k x n,  |E_k|^2 = n_i^2 + n_j^2
//   d x tau = T_k - s c F_k,    T_k = p x tau_k, F_k = e_k x tau_k
// so that each inactive simulation costs a few dot products.
template <class V>
__device__ __forceinline__ void point_sims_adjoint(const PointStateT<V>& ps, const SimAdjoints& G,
                                                   const SimConsts& K, const ParamsDev& P, const ObjDev& O,
                                                   V& dphi, V dn[3], V dp[3]) {
  constexpr int W = VecTraits<V>::width;
  const V tag{};
  const V zero = vsplat<V>(0.0f);
  const V* n = ps.n;
  V U[3];
  vcross(ps.p, n, U);
  const V Uu = vdot(U, U);
  unsigned cmask[W];
#pragma unroll
  for (int l = 0; l < W; ++l) cmask[l] = 0u;
  {  // m = 0: v = 0, d = p, no tangential displacement
    const mask_t<V> kap = vlt(ps.phi_hat, zero);
#pragma unroll
    for (int l = 0; l < W; ++l) cmask[l] |= mlane(kap, l) ? 1u : 0u;
    V gl[3], ga[3];
    get_sim_adjoint(G, 0, gl, ga);
    const V gfn = dot6(gl, n, ga, U);
    const V rw = vmap(vfma(simk(K, tag, kcB), Uu, simk(K, tag, kcA)), rcp_fast);
    const V q = vfma(gfn, rw, simk(K, tag, kcMWpen));
    dphi = vfma(simk(K, tag, kcAlpha), vsel(kap, zero, q), dphi);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    const V ni = n[i], nj = n[j], nk = n[k];
    const V rho2 = vfma(ni, ni, vmul(nj, nj));
    const V rr = vmap(rho2, rsqrt_or_zero);          // tau = 0 when n is parallel to e_k
    V tau[3];
    tau[k] = vmul(rho2, rr);
    const V nkr = vnmul(nk, rr);
    tau[i] = vmul(nkr, ni);
    tau[j] = vmul(nkr, nj);
    V T[3];
    vcross(ps.p, tau, T);
    const V UE = vdiff(U[j], ni, U[i], nj);            // U . E_k
    const V TF = vdiff(T[j], tau[i], T[i], tau[j]);    // T_k . F_k
    const V Fsq = vfma(tau[i], tau[i], vmul(tau[j], tau[j]));
    const V a = simk(K, tag, kcA), b = simk(K, tag, kcB), cc = simk(K, tag, kcCC), tbc = simk(K, tag, kcTBC);
    const V wn0 = vfma(b, vfma(cc, rho2, Uu), a), wn1 = vmul(tbc, UE);
    const V wt0 = vfma(b, vfma(cc, Fsq, vdot(T, T)), a), wt1 = vmul(tbc, TF);
    // per-axis parts of the dot products shared by the two signs
    V gdn[2], gdt[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = 1 + 2 * k + h;
      V gl[3], ga[3];
      get_sim_adjoint(G, m, gl, ga);
      const V msc = simk(K, tag, h == 0 ? kcMC : kcC);               // -s c
      const V gaE = vdiff(ga[j], ni, ga[i], nj);
      const V gaF = vdiff(ga[j], tau[i], ga[i], tau[j]);
      gdn[h] = vfma(msc, gaE, dot6(gl, n, ga, U));
      gdt[h] = vfma(msc, gaF, dot6(gl, tau, ga, T));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = 1 + 2 * k + h;
      const mask_t<V> kap = vlt(sim_phi(ps, m, P.dt * P.V), zero);
#pragma unroll
      for (int l = 0; l < W; ++l) cmask[l] |= mlane(kap, l) ? (1u << m) : 0u;
      // dph = -alpha dC,  dC = -(gf.n)/w_n - mu s (gf.tau)/w_t,  w = w0 - s w1
      const V rwn = vmap(h == 0 ? vsub(wn0, wn1) : vadd(wn0, wn1), rcp_fast);
      const V rwt = vmap(h == 0 ? vsub(wt0, wt1) : vadd(wt0, wt1), rcp_fast);
      const V q = vfma(simk(K, tag, h == 0 ? kcMu : kcMMu), vmul(gdt[h], rwt), vmul(gdn[h], rwn));
      const V qa = vsel(kap, zero, q);
      dphi = vfma(simk(K, tag, kcAlpha), qa, dphi);
      dn[k] = vfma(simk(K, tag, h == 0 ? kcMAlphaC : kcAlphaC), qa, dn[k]);
    }
  }
  // simulations in which some lane of the warp is in contact: general adjoint,
  // one instance per point, visiting only those simulations
  unsigned any = 0u;
#pragma unroll
  for (int l = 0; l < W; ++l) any |= cmask[l];
  unsigned wmask = __reduce_or_sync(0xffffffffu, any);
  const float c = P.dt * P.V;
  while (wmask) {
    const int m = __ffs(wmask) - 1;
    wmask &= wmask - 1u;
    float Gl[3], Ga[3];
    get_sim_adjoint(G, m, Gl, Ga);
    if constexpr (W == 1) {
      if ((cmask[0] >> m) & 1u)
        sim_adjoint(ps, m, sim_phi(ps, m, c), true, Gl, Ga, P, O, m == 0 ? P.w_pen : 0.0f, dphi, dn, dp);
    } else {
#pragma unroll 1
      for (int l = 0; l < W; ++l) {
        if ((cmask[l] >> m) & 1u) {
          const PointState s1 = point_lane(ps, l);
          float dph1 = 0.0f, dn1[3] = {0.0f, 0.0f, 0.0f}, dp1[3] = {0.0f, 0.0f, 0.0f};
          sim_adjoint(s1, m, sim_phi(s1, m, c), true, Gl, Ga, P, O, m == 0 ? P.w_pen : 0.0f, dph1, dn1, dp1);
          vlane_add(dphi, l, dph1);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            vlane_add(dn[k], l, dn1[k]);
            vlane_add(dp[k], l, dp1[k]);
          }
        }
      }
    }
  }
}

// Adjoint of the SDF lookup and normalisation: given dL/dphi_hat, dL/dn and the
// direct dL/dp, returns the total dL/dp.  n = g/|g|, g = grad phi(p), and the
// Hessian of phi is the trilinear mixed part plus, outside the grid, the
// curvature (I - eh eh^T)/e of the excess distance on the clamped axes.
template <class V>
__device__ __forceinline__ void sdf_adjoint(const SdfSampleT<V>& s, const PointStateT<V>& ps, V d_phi_hat,
                                            const V dn[3], V dp[3]) {
  const V ndn = vdot(ps.n, dn);
  V dg[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) dg[k] = vmul(vfnma(ndn, ps.n[k], dn[k]), ps.rg);
  dp[0] = vadd(dp[0], vfma(d_phi_hat, s.g[0], vfma(s.hxy, dg[1], vfma(s.hxz, dg[2], vmul(s.curv, dg[0])))));
  dp[1] = vadd(dp[1], vfma(d_phi_hat, s.g[1], vfma(s.hxy, dg[0], vfma(s.hyz, dg[2], vmul(s.curv, dg[1])))));
  dp[2] = vadd(dp[2], vfma(d_phi_hat, s.g[2], vfma(s.hxz, dg[0], vfma(s.hyz, dg[1], vmul(s.curv, dg[2])))));
  if (many(s.outside)) {
    // eh is zero on unclamped axes (and for points inside the grid, where e = 0
    // and the term vanishes), so (I - eh eh^T) restricted to clamped axes is
    // D_c - eh eh^T with D_c the mask of axes where eh != 0.
    const V zero = vsplat<V>(0.0f), one = vsplat<V>(1.0f);
    const V re = vmap(s.e, rcp_or_zero);
    const V ehdg = vdot(s.eh, dg);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const V ck = vsel(vne(s.eh[k], zero), one, zero);
      dp[k] = vfma(vfnma(s.eh[k], ehdg, vmul(ck, dg[k])), re, dp[k]);
    }
  }
}

// Wrench adjoint per simulation and the loss, from the reduced wrenches.
// xdot_m = v_m + W_lin inv_m / (N dt), thdot_m = W_ang inv_I / (N dt),
// L_stable = (1/7) sum_m (|xdot_m| + |thdot_m|)  (Eq. 2).
__device__ inline float stability_loss_and_adjoint(const float W[kSims][6], const float N[kSims],
                                                   const ParamsDev& P, const ObjDev& O,
                                                   float Gl[kSims][3], float Ga[kSims][3]) {
  float L = 0.0f;
  for (int m = 0; m < kSims; ++m) {
    float Nc = N[m] > 1.0f ? N[m] : 1.0f;
    float sl = O.inv_mass / (Nc * P.dt), sa = O.inv_inertia / (Nc * P.dt);
    float v[3] = {0.0f, 0.0f, 0.0f};
    if (m > 0) v[sim_axis(m)] = sim_sign(m) * P.V;
    float xd[3], td[3];
    for (int k = 0; k < 3; ++k) {
      xd[k] = v[k] + W[m][k] * sl;
      td[k] = W[m][3 + k] * sa;
    }
    float nx2 = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
    float nt2 = td[0] * td[0] + td[1] * td[1] + td[2] * td[2];
    float nx = sqrtf(nx2), nt = sqrtf(nt2);
    L += nx + nt;
    float ax = nx > 0.0f ? sl / (kSims * nx) : 0.0f;
    float at = nt > 0.0f ? sa / (kSims * nt) : 0.0f;
    for (int k = 0; k < 3; ++k) {
      Gl[m][k] = xd[k] * ax;
      Ga[m][k] = td[k] * at;
    }
  }
  return L / kSims;
}

// Joint terms L_range (Eq. 3) and L_limit (Eq. 4) with their gradient into dth.
__device__ inline float joint_losses(const HandDev& H, const float* th, const ParamsDev& P, float* dth) {
  float s2 = 0.0f, lim = 0.0f;
  for (int j = 0; j < H.J; ++j) {
    float mid = 0.5f * (H.q_up[j] + H.q_low[j]);
    float d = th[j] - mid;
    s2 += d * d;
    if (th[j] > H.q_up[j]) lim += th[j] - H.q_up[j];
    if (th[j] < H.q_low[j]) lim += H.q_low[j] - th[j];
  }
  float rn = sqrtf(s2);
  float inv = rn > 0.0f ? P.w_range / rn : 0.0f;
  for (int j = 0; j < H.J; ++j) {
    float mid = 0.5f * (H.q_up[j] + H.q_low[j]);
    float g = (th[j] - mid) * inv;
    if (th[j] > H.q_up[j]) g += P.w_limit;
    if (th[j] < H.q_low[j]) g -= P.w_limit;
    dth[j] = g;
  }
  return P.w_range * rn + P.w_limit * lim;
}

// Transpose of the left Jacobian of Exp applied to tau:
// J_l(w)^T tau = tau - b (w x tau) + c (w x (w x tau)),
// b = (1 - cos a)/a^2, c = (a - sin a)/a^3 (Taylor series below a = 0.5, where
// a - sin a loses float32 digits).
__device__ inline void exp_jacobian_T(const float w[3], const float tau[3], float out[3]) {
  float a2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  float b, c;
  if (a2 < 0.25f) {
    b = 0.5f + a2 * (-1.0f / 24.0f + a2 * (1.0f / 720.0f + a2 * (-1.0f / 40320.0f)));
    c = 1.0f / 6.0f + a2 * (-1.0f / 120.0f + a2 * (1.0f / 5040.0f + a2 * (-1.0f / 362880.0f)));
  } else {
    float a = sqrtf(a2);
    float s, co;
    sincosf(a, &s, &co);
    float sh = sinf(0.5f * a);
    b = 2.0f * sh * sh / a2;
    c = (a - s) / (a2 * a);
  }
  float wt[3], wwt[3];
  cross3(w, tau, wt);
  cross3(w, wt, wwt);
  for (int k = 0; k < 3; ++k) out[k] = tau[k] - b * wt[k] + c * wwt[k];
}

__device__ __forceinline__ float dilation_at(const ParamsDev& P, int k, int total_steps) {
  if (P.schedule == 0) return P.r0;
  int den = total_steps - 1 > 1 ? total_steps - 1 : 1;
  float r = P.r0 * (1.0f - (float)k / (float)den);
  return r > 0.0f ? r : 0.0f;
}

}  // namespace fg

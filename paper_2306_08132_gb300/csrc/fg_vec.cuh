// Lane vectors for the per-point arithmetic.
//
// V = float   one hand point per thread;
// V = float2  two hand points per thread, one in each half of a packed f32x2
//             register pair.  sm_100-class GPUs issue an f32x2 add, multiply or
//             fused multiply-add as one instruction, so two points' arithmetic
//             takes the issue slots of one.
//
// Every operation rounds to nearest per component (the _rn forms), so a point's
// results are bit-identical whichever form computed them; decisions (contact
// flags, clamping, friction regime) therefore agree between the scalar forward
// sweep and the packed adjoint sweep.
#pragma once

#include <cuda_runtime.h>

namespace fg {

struct bool2 {
  bool x, y;
};

template <class V>
struct VecTraits;
template <>
struct VecTraits<float> {
  using mask = bool;
  static constexpr int width = 1;
};
template <>
struct VecTraits<float2> {
  using mask = bool2;
  static constexpr int width = 2;
};
template <class V>
using mask_t = typename VecTraits<V>::mask;

// ---------------------------------------------------------------- arithmetic
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }

__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one rounding of a + (-1) b: the same bits as a subtraction
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// c - a b (scalar: one fused multiply-add with a negated operand)
__device__ __forceinline__ float vfnma(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
__device__ __forceinline__ float2 vfnma(float2 a, float2 b, float2 c) { return vsub(c, vmul(a, b)); }
// a b - c d (not used for decisions)
__device__ __forceinline__ float vdiff(float a, float b, float c, float d) { return __fmaf_rn(a, b, -__fmul_rn(c, d)); }
__device__ __forceinline__ float2 vdiff(float2 a, float2 b, float2 c, float2 d) { return vsub(vmul(a, b), vmul(c, d)); }
// -(a b)
__device__ __forceinline__ float vnmul(float a, float b) { return -__fmul_rn(a, b); }
__device__ __forceinline__ float2 vnmul(float2 a, float2 b) { return vmul(vmul(a, b), make_float2(-1.0f, -1.0f)); }

template <class V>
__device__ __forceinline__ V vsplat(float x);
template <>
__device__ __forceinline__ float vsplat<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 vsplat<float2>(float x) { return make_float2(x, x); }

// component k (0 or 1) of a lane vector
__device__ __forceinline__ float vlane(float v, int) { return v; }
__device__ __forceinline__ float vlane(float2 v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ void vlane_add(float& v, int, float x) { v = __fadd_rn(v, x); }
__device__ __forceinline__ void vlane_add(float2& v, int k, float x) {
  if (k == 0)
    v.x = __fadd_rn(v.x, x);
  else
    v.y = __fadd_rn(v.y, x);
}

// per-component function (reciprocals, square roots, comparisons that pick a branch)
template <class F>
__device__ __forceinline__ float vmap(float a, F f) {
  return f(a);
}
template <class F>
__device__ __forceinline__ float2 vmap(float2 a, F f) {
  return make_float2(f(a.x), f(a.y));
}

// --------------------------------------------------------------------- masks
__device__ __forceinline__ bool vlt(float a, float b) { return a < b; }
__device__ __forceinline__ bool2 vlt(float2 a, float2 b) { return {a.x < b.x, a.y < b.y}; }
__device__ __forceinline__ bool vgt(float a, float b) { return a > b; }
__device__ __forceinline__ bool2 vgt(float2 a, float2 b) { return {a.x > b.x, a.y > b.y}; }
__device__ __forceinline__ bool vne(float a, float b) { return a != b; }
__device__ __forceinline__ bool2 vne(float2 a, float2 b) { return {a.x != b.x, a.y != b.y}; }

__device__ __forceinline__ bool mor(bool a, bool b) { return a || b; }
__device__ __forceinline__ bool2 mor(bool2 a, bool2 b) { return {a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ bool many(bool m) { return m; }
__device__ __forceinline__ bool many(bool2 m) { return m.x || m.y; }
__device__ __forceinline__ bool mlane(bool m, int) { return m; }
__device__ __forceinline__ bool mlane(bool2 m, int k) { return k == 0 ? m.x : m.y; }

__device__ __forceinline__ float vsel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ float2 vsel(bool2 m, float2 a, float2 b) {
  return make_float2(m.x ? a.x : b.x, m.y ? a.y : b.y);
}

// ------------------------------------------------------------ 3-vector forms
// (not used for decisions: the packed form rounds both products)
__device__ __forceinline__ void vcross(const float a[3], const float b[3], float c[3]) {
  c[0] = __fmaf_rn(a[1], b[2], -__fmul_rn(a[2], b[1]));
  c[1] = __fmaf_rn(a[2], b[0], -__fmul_rn(a[0], b[2]));
  c[2] = __fmaf_rn(a[0], b[1], -__fmul_rn(a[1], b[0]));
}
__device__ __forceinline__ void vcross(const float2 a[3], const float2 b[3], float2 c[3]) {
  c[0] = vdiff(a[1], b[2], a[2], b[1]);
  c[1] = vdiff(a[2], b[0], a[0], b[2]);
  c[2] = vdiff(a[0], b[1], a[1], b[0]);
}
template <class V>
__device__ __forceinline__ V vdot(const V a[3], const V b[3]) {
  return vfma(a[0], b[0], vfma(a[1], b[1], vmul(a[2], b[2])));
}

}  // namespace fg

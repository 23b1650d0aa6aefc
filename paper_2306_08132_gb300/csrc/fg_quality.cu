// Grasp-quality metrics of the paper's evaluation (Sec. V, "Metrics") for batches
// of candidates: the weighted contact measure (contact area CA with surface
// samples and area weights, intersection volume IV with interior samples and
// volume weights) and epsilon over a set of wrench-space directions.
//
// Contacts are the hand points with phi(p) < tau (undilated SDF, object at its
// canonical pose).  A contact with outward normal n contributes the k edges of
// its Coulomb cone, f_e = -n + mu (cos(2 pi e/k) t1 + sin(2 pi e/k) t2) with the
// tangent basis (t1, t2) of Duff et al. (2017), as wrenches
// w = (f, s (p - c) x f), s the torque scale and c the object's origin.  For a
// unit direction u = (u_f, u_t), u . w = a . f with a = u_f + s (u_t x p), so
//   max_e u . w_e = -a . n + mu max_e (cos_e a . t1 + sin_e a . t2),
// and eps_U = min over the directions of the maximum over all contacts.
//
// Both kernels: one CTA per candidate (persistent, candidates claimed from a
// counter), FK by warp 0, warps over 32-point chunks.  Epsilon collects the contacts of 32 chunks at a time in
// shared memory (point, normal, tangent basis) and every thread folds them into
// the running maxima of its directions; max and min do not depend on order, so
// the result is exact with respect to the order of the contacts.
#include <cuda_runtime.h>

#include <math.h>

#include "fg_fused_kernel.cuh"
#include "fg_internal.h"

namespace fg {

namespace {

constexpr int kQW = 8;                       // warps per candidate
constexpr int kQBatchChunks = 32;            // chunks per contact batch (<= 1024 contacts)
constexpr int kQBatch = 32 * kQBatchChunks;
constexpr int kQD = 4;                       // directions per thread per pass over the contacts

struct QualitySmem {
  HandDev H;
  float4 frame4[kMaxLinks][3];
  float q[64];
  float red[kQW];
  float ce[32], se[32];                      // cone edge angles
  int count;
  int total;
  ObjDev O;
  int bad_object;
  int cand;                                  // the candidate claimed by this CTA
  const HandDev* hand_loaded;
};

// Loads the hand descriptor (if it changed) and the candidate's object and q,
// then computes the link frames.  Returns false for an object index outside the scene.
__device__ bool quality_setup(QualitySmem& S, const FusedArgs& a, int c, int tid, int nthreads) {
  __syncthreads();
  if (tid == 0) {
    const int oi = a.obj_of_cand ? a.obj_of_cand[c] : 0;
    S.bad_object = oi < 0 || oi >= a.n_obj;
    if (!S.bad_object) S.O = a.objs[oi];
  }
  if (a.hand != S.hand_loaded) {
    const int* src = reinterpret_cast<const int*>(a.hand);
    int* dst = reinterpret_cast<int*>(&S.H);
    for (int k = tid; k < (int)(sizeof(HandDev) / sizeof(int)); k += nthreads) dst[k] = src[k];
  }
  __syncthreads();
  if (tid == 0) S.hand_loaded = a.hand;
  if (tid < S.H.D) S.q[tid] = a.q[(size_t)c * S.H.D + tid];
  __syncthreads();
  if (S.bad_object) return false;
  if (tid < 32) fk_warp(S.H, S.q, S.frame4, tid);
  __syncthreads();
  return true;
}

template <bool ANY>
__global__ void __launch_bounds__(kQW * 32) measure_kernel(FusedArgs a, const float* __restrict__ weights, float tau,
                                                        float* __restrict__ out) {
  __shared__ QualitySmem S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) S.hand_loaded = nullptr;
  for (;;) {
    const int c = next_candidate(a.work, &S.cand);
    if (c >= a.B) break;
    if (!quality_setup(S, a, c, tid, kQW * 32)) {
      if (tid == 0) out[c] = __int_as_float(0x7fc00000);
      continue;
    }
    const HandDev& H = S.H;
    float acc = 0.0f;
    for (int j = warp; j < H.nchunks; j += kQW) {
      const int i = 32 * j + lane;
      const bool valid = i < H.P;
      const float4 sp = __ldg(H.pts + (valid ? i : 32 * j));
      float p[3];
      world_point(S.frame4[(int)sp.w], sp, p);
      SdfSample smp;
      sdf_lookup<false, ANY>(S.O, p, smp);
      if (valid && smp.phi < tau) acc += __ldg(weights + i);
    }
    acc = warp_sum(acc);
    if (lane == 0) S.red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      float t = 0.0f;
#pragma unroll
      for (int w = 0; w < kQW; ++w) t += S.red[w];
      out[c] = t;
    }
  }
  work_done(a.work);
}

// Contact record in the batch: point p, outward normal n, tangent basis t1, t2.
struct ContactRec {
  float4 a;   // p.x p.y p.z n.x
  float4 b;   // n.y n.z t1.x t1.y
  float4 c;   // t1.z t2.x t2.y t2.z
};

template <bool ANY>
__global__ void __launch_bounds__(kQW * 32) epsilon_kernel(FusedArgs a, float tau, float mu, int k_edges,
                                                        float tscale, const float* __restrict__ dirs, int K,
                                                        float* __restrict__ eps, int* __restrict__ ncontact) {
  __shared__ QualitySmem S;
  extern __shared__ float4 dyn4[];
  ContactRec* rec = reinterpret_cast<ContactRec*>(dyn4);        // [kQBatch]
  float* hmax = reinterpret_cast<float*>(rec + kQBatch);       // [K]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NT = kQW * 32;
  if (tid == 0) S.hand_loaded = nullptr;
  if (tid < k_edges) {
    float s, co;
    sincospif(2.0f * (float)tid / (float)k_edges, &s, &co);
    S.ce[tid] = co;
    S.se[tid] = s;
  }
  for (;;) {
    const int c = next_candidate(a.work, &S.cand);
    if (c >= a.B) break;
    if (!quality_setup(S, a, c, tid, NT)) {
      if (tid == 0) {
        eps[c] = __int_as_float(0x7fc00000);
        if (ncontact) ncontact[c] = -1;
      }
      continue;
    }
    const HandDev& H = S.H;
    for (int k = tid; k < K; k += NT) hmax[k] = -INFINITY;
    if (tid == 0) S.total = 0;
    for (int g0 = 0; g0 < H.nchunks; g0 += kQBatchChunks) {
      if (tid == 0) S.count = 0;
      __syncthreads();
      const int g1 = min(g0 + kQBatchChunks, H.nchunks);
      for (int j = g0 + warp; j < g1; j += kQW) {
        const int i = 32 * j + lane;
        const bool valid = i < H.P;
        const float4 sp = __ldg(H.pts + (valid ? i : 32 * j));
        float p[3];
        world_point(S.frame4[(int)sp.w], sp, p);
        SdfSample smp;
        sdf_lookup<false, ANY>(S.O, p, smp);
        const bool hit = valid && smp.phi < tau;
        const unsigned bal = __ballot_sync(kFull, hit);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&S.count, __popc(bal));
        base = __shfl_sync(kFull, base, 0);
        if (hit) {
          const float g2 = smp.g[0] * smp.g[0] + smp.g[1] * smp.g[1] + smp.g[2] * smp.g[2];
          const float rg = rsqrt_or_zero(g2);
          const float n[3] = {smp.g[0] * rg, smp.g[1] * rg, smp.g[2] * rg};
          // Duff et al. (2017): s = sign(n_z) (+1 at 0), a = -1/(s + n_z), b = n_x n_y a
          const float sg = n[2] >= 0.0f ? 1.0f : -1.0f;
          const float aa = -1.0f / (sg + n[2]);
          const float bb = n[0] * n[1] * aa;
          const float t1[3] = {1.0f + sg * n[0] * n[0] * aa, sg * bb, -sg * n[0]};
          const float t2[3] = {bb, sg + n[1] * n[1] * aa, -n[1]};
          ContactRec& r = rec[base + __popc(bal & ((1u << lane) - 1u))];
          r.a = make_float4(p[0], p[1], p[2], n[0]);
          r.b = make_float4(n[1], n[2], t1[0], t1[1]);
          r.c = make_float4(t1[2], t2[0], t2[1], t2[2]);
        }
      }
      __syncthreads();
      const int nc = S.count;
      // kQD directions per thread per pass: each contact record read from shared
      // memory serves all of them
      for (int k0 = tid; k0 < K; k0 += NT * kQD) {
        float uf[kQD][3], ut[kQD][3], h[kQD];
#pragma unroll
        for (int d = 0; d < kQD; ++d) {
          const int k = min(k0 + d * NT, K - 1);              // repeats the last direction past K
          const float* u = dirs + (size_t)k * 6;
#pragma unroll
          for (int c3 = 0; c3 < 3; ++c3) {
            uf[d][c3] = __ldg(u + c3);
            ut[d][c3] = __ldg(u + 3 + c3) * tscale;
          }
          h[d] = k0 + d * NT < K ? hmax[k] : -INFINITY;       // each thread keeps to its own entries
        }
        for (int jc = 0; jc < nc; ++jc) {
          const float4 ra = rec[jc].a, rb = rec[jc].b, rc = rec[jc].c;
#pragma unroll
          for (int d = 0; d < kQD; ++d) {
            // a = u_f + s (u_t x p)
            const float ax = uf[d][0] + (ut[d][1] * ra.z - ut[d][2] * ra.y);
            const float ay = uf[d][1] + (ut[d][2] * ra.x - ut[d][0] * ra.z);
            const float az = uf[d][2] + (ut[d][0] * ra.y - ut[d][1] * ra.x);
            const float an = ax * ra.w + ay * rb.x + az * rb.y;
            const float a1 = ax * rb.z + ay * rb.w + az * rc.x;
            const float a2 = ax * rc.y + ay * rc.z + az * rc.w;
            float best = -INFINITY;
            for (int e = 0; e < k_edges; ++e) best = fmaxf(best, S.ce[e] * a1 + S.se[e] * a2);
            h[d] = fmaxf(h[d], mu * best - an);
          }
        }
#pragma unroll
        for (int d = 0; d < kQD; ++d)
          if (k0 + d * NT < K) hmax[k0 + d * NT] = h[d];
      }
      if (tid == 0) S.total += nc;
      __syncthreads();
    }
    float m = INFINITY;
    for (int k = tid; k < K; k += NT) m = fminf(m, hmax[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(kFull, m, o));
    if (lane == 0) S.red[warp] = m;
    __syncthreads();
    if (tid == 0) {
      float t = INFINITY;
#pragma unroll
      for (int w = 0; w < kQW; ++w) t = fminf(t, S.red[w]);
      eps[c] = t;
      if (ncontact) ncontact[c] = S.total;
    }
  }
  work_done(a.work);
}

template <class Kern>
cudaError_t grid_for_kernel(Kern k, size_t dyn, int B, int* grid) {
  int bps = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kQW * 32, dyn);
  if (e != cudaSuccess) return e;
  if (bps < 1) bps = 1;
  long long g = (long long)device_sm_count() * bps;
  if (g > B) g = B;
  *grid = (int)g;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_contact_measure(const FusedArgs& a0, const float* weights, float tau, float* out, cudaStream_t st) {
  if (a0.B <= 0) return cudaSuccess;
  FusedArgs a = a0;
  cudaError_t ew = work_pair(&a.work, st);
  if (ew != cudaSuccess) return ew;
  int grid = 0;
  if (a.any_mesh) {
    cudaError_t e = grid_for_kernel(measure_kernel<true>, 0, a.B, &grid);
    if (e != cudaSuccess) return e;
    measure_kernel<true><<<grid, kQW * 32, 0, st>>>(a, weights, tau, out);
  } else {
    cudaError_t e = grid_for_kernel(measure_kernel<false>, 0, a.B, &grid);
    if (e != cudaSuccess) return e;
    measure_kernel<false><<<grid, kQW * 32, 0, st>>>(a, weights, tau, out);
  }
  return cudaGetLastError();
}

size_t epsilon_smem_bytes(int K) { return sizeof(ContactRec) * kQBatch + sizeof(float) * (size_t)K; }

cudaError_t launch_grasp_epsilon(const FusedArgs& a0, float tau, float mu, int k_edges, float tscale,
                                 const float* dirs, int K, float* eps, int* ncontact, cudaStream_t st) {
  if (a0.B <= 0) return cudaSuccess;
  FusedArgs a = a0;
  cudaError_t ew = work_pair(&a.work, st);
  if (ew != cudaSuccess) return ew;
  const size_t dyn = epsilon_smem_bytes(K);
  static size_t attr_set[2][64] = {{0}, {0}};
  int dev = 0;
  cudaGetDevice(&dev);
  const int v = a.any_mesh ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (dyn > attr_set[v][dev & 63]) {
    e = a.any_mesh ? cudaFuncSetAttribute(epsilon_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)
                   : cudaFuncSetAttribute(epsilon_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    attr_set[v][dev & 63] = dyn;
  }
  int grid = 0;
  if (a.any_mesh) {
    e = grid_for_kernel(epsilon_kernel<true>, dyn, a.B, &grid);
    if (e != cudaSuccess) return e;
    epsilon_kernel<true><<<grid, kQW * 32, dyn, st>>>(a, tau, mu, k_edges, tscale, dirs, K, eps, ncontact);
  } else {
    e = grid_for_kernel(epsilon_kernel<false>, dyn, a.B, &grid);
    if (e != cudaSuccess) return e;
    epsilon_kernel<false><<<grid, kQW * 32, dyn, st>>>(a, tau, mu, k_edges, tscale, dirs, K, eps, ncontact);
  }
  return cudaGetLastError();
}

}  // namespace fg

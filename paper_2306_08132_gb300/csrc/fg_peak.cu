// FP32 arithmetic throughput of the GPU, measured: the denominator of the ALU
// roofline of the kernels above.  Every thread runs kChains independent chains
// of fused multiply-adds (x <- x a + b), enough independent work per warp to hide
// the pipe's latency, in one of two instruction forms: scalar FFMA (one lane,
// 2 flops) or packed f32x2 FMA (two lanes of a register pair, 4 flops).  The
// chains stay bounded (|a| < 1) and their sum is stored, so no chain is dead code.
#include <cuda_runtime.h>

#include "fg_internal.h"

namespace fg {

constexpr int kChains = 8;

template <bool PACKED>
__global__ void __launch_bounds__(256) fma_peak_kernel(float* out, int iters, float a, float b) {
  const float seed = 1e-3f * (float)(threadIdx.x & 63);
  float acc = 0.0f;
  if (PACKED) {
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = make_float2(seed + k, seed - k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += x[k].x + x[k].y;
  } else {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = seed + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], a, b);
    }
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc += x[k];
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace fg

using namespace fg;

extern "C" fg_status fg_fp32_peak_launch(int packed, int blocks, int iters, float* out, double* flops,
                                         void* stream) {
  if (blocks < 1 || iters < 1 || !out) {
    set_error("fg_fp32_peak_launch: need blocks >= 1, iters >= 1 and out");
    return FG_ERR_INVALID;
  }
  const int threads = 256;
  if (packed)
    fma_peak_kernel<true><<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-3f);
  else
    fma_peak_kernel<false><<<blocks, threads, 0, (cudaStream_t)stream>>>(out, iters, 0.999f, 1e-3f);
  if (flops) *flops = (double)blocks * threads * iters * kChains * (packed ? 4.0 : 2.0);
  return cuda_status(cudaGetLastError(), "fg_fp32_peak_launch");
}

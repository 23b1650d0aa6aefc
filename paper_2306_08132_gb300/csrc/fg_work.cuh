// Candidates claimed from a counter by persistent CTAs.
//
// A persistent grid over candidates whose cost varies (contacts make a candidate
// several times dearer) ends when its busiest CTA ends, so CTAs take the next
// candidate from a counter instead of a fixed stride.  A counter is a pair of words
// (the next candidate; the number of CTAs that found none left).  Each launch draws
// its own pair from a pool of this translation unit, and the last CTA to finish sets
// both words back to zero, so the pair is clean for the next launch that draws it.
// Eager launches cycle through the first kWorkSlots pairs.  A launch captured in a
// graph keeps its pair on every replay, so captured launches draw from a separate
// range of kCapturedSlots pairs that eager launches never use: a graph's replays
// never share a counter with eager launches, nor with another graph unless
// kCapturedSlots launches were captured in between.  One graph must not be
// replayed on two streams at once.
#pragma once

#include <atomic>

#include <cuda_runtime.h>

namespace fg {

constexpr int kWorkSlots = 1024;
constexpr int kCapturedSlots = 16384;
static __device__ unsigned g_work_pool[kWorkSlots + kCapturedSlots][2];
static std::atomic<unsigned> g_work_seq{0};
static std::atomic<unsigned> g_captured_seq{0};

// Host: the counter pair of one launch on `stream` on the current device.
static inline cudaError_t work_pair(unsigned** out, cudaStream_t stream) {
  static unsigned* pool[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  unsigned*& p = pool[dev & 63];
  if (p == nullptr) {
    void* q = nullptr;
    e = cudaGetSymbolAddress(&q, g_work_pool);
    if (e != cudaSuccess) return e;
    p = static_cast<unsigned*>(q);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  if (cap == cudaStreamCaptureStatusActive)
    *out = p + 2 * (kWorkSlots + g_captured_seq.fetch_add(1u) % kCapturedSlots);
  else
    *out = p + 2 * (g_work_seq.fetch_add(1u) % kWorkSlots);
  return cudaSuccess;
}

// Device, every thread of the CTA: the next candidate (>= B once none is left).
// slot is a shared-memory word; the barriers on both sides make the claim uniform.
__device__ __forceinline__ int next_candidate(unsigned* work, int* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = (int)atomicAdd(work, 1u);
  __syncthreads();
  return *slot;
}

// Device, after the CTA's last claim: the last CTA of the grid resets the pair.
__device__ __forceinline__ void work_done(unsigned* work) {
  if (threadIdx.x == 0 && atomicAdd(work + 1, 1u) == gridDim.x - 1) {
    atomicExch(work, 0u);
    atomicExch(work + 1, 0u);
  }
}

}  // namespace fg

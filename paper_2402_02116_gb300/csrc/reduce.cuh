// Deterministic FP64 reductions shared by the operator and Krylov kernels.
//
// A reduction is two-stage: every CTA sums its threads' values in a fixed tree and stores one
// partial per slot; every consumer sums a problem's partials in a fixed order. The same inputs
// therefore always give the same bits, whichever kernel consumes them.
#pragma once

#include "common.cuh"

namespace dbi {

// Sum NS values over the CTA (blockDim.x a multiple of 32, at most 1024) in a fixed order;
// thread 0 stores the sums to out[0..NS). Every thread of the CTA must call it. The warp stage
// adds in the type of the per-thread sums (float for complex64 work: FP64 arithmetic runs at a
// small fraction of the FP32 rate on this GPU, and a CTA-wide FP64 shuffle tree per partial cost
// more than the memory pass it reduces); the CTA stage adds the warp sums in FP64.
template <int NS, typename T> __device__ __forceinline__ void block_sum_store(T (&v)[NS], double *out) {
  __shared__ double sh[NS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    T a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) sh[k][warp] = double(a);
  }
  __syncthreads();
  if (threadIdx.x < NS) {  // one thread per value: the warp sums in order
    const int nw = blockDim.x >> 5;
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += sh[threadIdx.x][w];
    out[threadIdx.x] = a;
  }
  __syncthreads();
}

// Sum slot k (k < NS) of `count` partials of one problem in a fixed order; every thread of the
// CTA gets the sums. Every thread of the CTA must call it.
template <int NS> __device__ __forceinline__ void gather_n(const double *part, int count, double (&out)[NS]) {
  __shared__ double sh[NS];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double a = 0.0;
      for (int i = lane; i < count; i += 32) a += part[i * kRedSlots + k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
      if (lane == 0) sh[k] = a;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NS; ++k) out[k] = sh[k];
  __syncthreads();
}

// Maximum of v over the CTA; thread 0 stores it to out[0]. Every thread of the CTA must call it.
__device__ __forceinline__ void block_max_store(double v, double *out) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) a = fmax(a, sh[w]);
    out[0] = a;
  }
  __syncthreads();
}

// Maximum of slot 0 of `count` partials (stride kRedSlots); every thread of the CTA gets it.
__device__ __forceinline__ double gather_max(const double *part, int count) {
  __shared__ double sh;
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int i = threadIdx.x; i < count; i += 32) a = fmax(a, part[i * kRedSlots]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, off));
    if (threadIdx.x == 0) sh = a;
  }
  __syncthreads();
  const double r = sh;
  __syncthreads();
  return r;
}

}  // namespace dbi

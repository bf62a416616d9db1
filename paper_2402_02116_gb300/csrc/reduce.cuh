// Deterministic FP64 reductions shared by the operator and Krylov kernels.
//
// A reduction is two-stage: every CTA sums its threads' values in a fixed tree and stores one
// partial per slot; every consumer sums a problem's partials in a fixed order. The same inputs
// therefore always give the same bits, whichever kernel consumes them.
#pragma once

#include "common.cuh"

namespace dbi {

// Sum NS values over the CTA (blockDim.x a multiple of 32, at most 1024) in a fixed order;
// thread 0 stores the sums to out[0..NS). Every thread of the CTA must call it.
template <int NS> __device__ __forceinline__ void block_sum_store(double (&v)[NS], double *out) {
  __shared__ double sh[NS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
    if (lane == 0) sh[k][warp] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double a = 0.0;
      for (int w = 0; w < nw; ++w) a += sh[k][w];
      out[k] = a;
    }
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

}  // namespace dbi

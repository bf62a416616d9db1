// Device helpers of the batched Krylov solvers (BiCGSTAB in krylov.cu, GMRES in gmres.cu).
#pragma once

#include "operator.cuh"

namespace dbi {

template <typename C> struct Acc;                         // per-thread accumulation type
template <> struct Acc<float2> { using type = float; };   // short per-thread sums, then FP64
template <> struct Acc<double2> { using type = double; };

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C from_z(double2 z) {
  using R = typename RealOf<C>::type;
  return mk<C>(R(z.x), R(z.y));
}

// Grid-stride loop over the n elements of problem b (unrolled for memory parallelism).
// Problem of this CTA: plist[blockIdx.y] when the launch runs a compacted list of problems.
__device__ __forceinline__ int problem_at(const int *plist, int slot) { return plist ? plist[slot] : slot; }

#define DBI_PROBLEM_LOOP(sp)                                                                  \
  const size_t off = (sp).offset(b), cnt = (sp).count(b);                                     \
  _Pragma("unroll 4")                                                                         \
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cnt; i += size_t(gridDim.x) * blockDim.x)

// Grid-stride loop over the elements of problem b calling f.template operator()<N>(o) for the N
// consecutive elements from offset o: N = 2 (a 16-byte pair of complex64 values, loaded and stored
// with one instruction by ldN / stN) when the problem's offset and count are even, else N = 1.
template <typename C, typename F>
__device__ __forceinline__ void problem_loop_pairs(const Span &sp, int b, F &&f) {
  const size_t off = sp.offset(b), cnt = sp.count(b);
  const size_t i0 = size_t(blockIdx.x) * blockDim.x + threadIdx.x, step = size_t(gridDim.x) * blockDim.x;
  if (sizeof(C) == sizeof(float2) && ((off | cnt) & 1) == 0) {
#pragma unroll 2
    for (size_t i = i0; i < cnt / 2; i += step) f.template operator()<2>(off + 2 * i);
  } else {
#pragma unroll 4
    for (size_t i = i0; i < cnt; i += step) f.template operator()<1>(off + i);
  }
}
template <int N, typename C> __device__ __forceinline__ void ldN(const C *p, C (&v)[N]) {
  if constexpr (N == 2 && sizeof(C) == sizeof(float2)) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = mk<C>(q.x, q.y);
    v[1] = mk<C>(q.z, q.w);
  } else {
#pragma unroll
    for (int n = 0; n < N; ++n) v[n] = p[n];
  }
}
template <int N, typename C> __device__ __forceinline__ void stN(C *p, const C (&v)[N]) {
  if constexpr (N == 2 && sizeof(C) == sizeof(float2)) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  } else {
#pragma unroll
    for (int n = 0; n < N; ++n) p[n] = v[n];
  }
}

// 2^-e with m in [2^e, 2^(e+1)), or 1 when m = 0.
__device__ __forceinline__ double pow2_below(double m) { return m > 0.0 ? ldexp(1.0, -ilogb(m)) : 1.0; }

}  // namespace dbi

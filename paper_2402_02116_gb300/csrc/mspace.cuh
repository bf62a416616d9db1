// Model-space vectors of the Tikhonov normal-equation CG (Eq. 23, 24), FP64, shared by the 2D
// (products.cu) and 3D (ls3d.cu) drivers. Kernels are static: each translation unit has its own.
#pragma once

#include "common.cuh"

namespace dbi {

constexpr int kMBlocks = 64, kMThreads = 256;

static __global__ void k_mdot(size_t n, const double *a, const double *b, double *part) {
  __shared__ double sh[kMThreads / 32];
  double acc = 0.0;
  for (size_t i = size_t(blockIdx.x) * kMThreads + threadIdx.x; i < n; i += size_t(kMBlocks) * kMThreads)
    acc += a[i] * b[i];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kMThreads / 32; ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

static __device__ __forceinline__ double sum_parts(const double *part) {
  double s = 0.0;
  for (int i = 0; i < kMBlocks; ++i) s += part[i];
  return s;
}

// Scalar steps of CG and of the power iteration; sc holds the FP64 scalars:
// 0 rr, 1 alpha, 2 beta, 3 lambda, 4 scratch (1/norm), 5 lambda_rel
enum { S_RR = 0, S_ALPHA = 1, S_BETA = 2, S_LAMBDA = 3, S_INV = 4, S_LREL = 5 };

static __global__ void k_scalar(int what, const double *part, double *sc, double *hist, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double s = sum_parts(part);
  switch (what) {
    case 0:  // rr = s, hist[0]
      sc[S_RR] = s;
      hist[0] = sqrt(s);
      break;
    case 1:  // alpha = rr / <p, q>
      sc[S_ALPHA] = s != 0.0 ? sc[S_RR] / s : 0.0;
      break;
    case 2:  // beta = rr_new / rr, hist[k]
      sc[S_BETA] = sc[S_RR] != 0.0 ? s / sc[S_RR] : 0.0;
      sc[S_RR] = s;
      hist[k] = sqrt(s);
      break;
    case 3:  // 1 / ||v||
      sc[S_INV] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
      break;
    case 4:  // lambda = lambda_rel * <v, H v>
      sc[S_LAMBDA] = sc[S_LREL] * s;
      break;
  }
}

// y = alpha_sel * x + beta_sel * y elementwise with scalars picked from sc (or 1 / 0)
static __global__ void k_maxpy(size_t n, int mode, const double *sc, const double *x, double *y,
                        const double *q, double *r) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    switch (mode) {
      case 0:  // x += alpha p (y = x, x = p); r -= alpha q
        y[i] += sc[S_ALPHA] * x[i];
        r[i] -= sc[S_ALPHA] * q[i];
        break;
      case 1:  // p = r + beta p  (y = p, x = r)
        y[i] = x[i] + sc[S_BETA] * y[i];
        break;
      case 2:  // y = x * inv
        y[i] = x[i] * sc[S_INV];
        break;
      case 3:  // q += lambda p  (y = q, x = p)
        y[i] += sc[S_LAMBDA] * x[i];
        break;
      case 4:  // copy
        y[i] = x[i];
        break;
    }
  }
}

// y[p][cell] = s_p * x[p][cell] for the np parameters, converting between model-space types
struct MScale {
  double s[6];
};
template <typename TI, typename TO>
static __global__ void k_mscale(int np, size_t plane, const TI *x, TO *y, MScale sc) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np * plane; i += size_t(gridDim.x) * blockDim.x)
    y[i] = TO(double(x[i]) * sc.s[i / plane]);
}

}  // namespace dbi

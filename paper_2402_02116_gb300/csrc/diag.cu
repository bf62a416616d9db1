// Diagnostics without a counterpart in the paper: a probe of the FP32 FMA issue rate, which sets
// the arithmetic roofline of the FFT-bound operator kernels (they run on the FP32 pipes, not on
// tensor cores).
#include "common.cuh"

namespace dbi {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent dependency chains per thread hide the FMA latency

// Every thread runs kProbeChains chains a <- a * m + c for `iters` steps; nothing else is issued in
// the loop. The result is written so that the chains cannot be removed.
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, float m, float c, float *out) {
  float a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = float(threadIdx.x + k) * 1e-3f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  out[size_t(blockIdx.x) * kProbeThreads + threadIdx.x] = s;
}

}  // namespace dbi

using namespace dbi;

extern "C" long long dbi_fma_probe(int blocks, int iters, float *out, dbi_stream stream) {
  clear_error();
  if (blocks < 1 || iters < 1 || !out) {
    set_error("dbi_fma_probe needs blocks >= 1, iters >= 1 and a device output of blocks x 256 floats");
    return DBI_ERR_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_fma_probe<<<blocks, kProbeThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, out);
  const int rc = check_launch("k_fma_probe");
  if (rc) return rc;
  return 2LL * kProbeChains * kProbeThreads * (long long)blocks * (long long)iters;
}

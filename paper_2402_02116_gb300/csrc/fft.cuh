// Shared-memory Stockham FFTs of lines held in shared memory.
//
// A CTA transforms NL lines of length L stored at s[line * LS + k]. Each pass of radix R runs
// NL * L / R butterflies split evenly over the NT threads: butterfly j of a line (j < L / R) reads
// the R points j + r L / R, multiplies them by W_{Ns R}^{r (j mod Ns)}, takes an R-point DFT in
// registers and writes the results to (j - j mod Ns) R + j mod Ns + r Ns, with Ns the product of
// the radices of the earlier passes (the self-sorting Stockham order: no bit reversal). Every
// thread keeps its butterflies in registers between the reads and the writes, so one buffer
// suffices, with a barrier on each side of the writes.
//
// Twiddles come from one table tw[m] = exp(-2 pi i m / 3072); a length-L transform reads it with
// stride 3072 / L. Forward transforms use exp(-2 pi i jk / L), inverse ones exp(+2 pi i jk / L),
// both unnormalised.
#pragma once

#include "common.cuh"

namespace dbi {

template <typename C, bool INV> __host__ __device__ __forceinline__ C hmul_mi(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C hadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C hsub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C hmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}

// 2-point DFT
template <typename C, bool INV> __host__ __device__ __forceinline__ void dft2(C *v) {
  C a = v[0], b = v[1];
  v[0] = hadd(a, b);
  v[1] = hsub(a, b);
}

// 4-point DFT: y_q = sum_r v_r W4^{rq}, W4 = -i (forward) or +i (inverse)
template <typename C, bool INV> __host__ __device__ __forceinline__ void dft4(C *v) {
  C t0 = hadd(v[0], v[2]), t1 = hsub(v[0], v[2]);
  C t2 = hadd(v[1], v[3]), t3 = hmul_mi<C, INV>(hsub(v[1], v[3]));
  v[0] = hadd(t0, t2);
  v[2] = hsub(t0, t2);
  v[1] = hadd(t1, t3);
  v[3] = hsub(t1, t3);
}

// 8-point DFT as two 4-point DFTs (even and odd inputs) joined by W8^q
template <typename C, bool INV> __host__ __device__ __forceinline__ void dft8(C *v) {
  using R = typename RealOf<C>::type;
  const R h = R(0.70710678118654752440);  // 1/sqrt(2)
  C e[4] = {v[0], v[2], v[4], v[6]};
  C o[4] = {v[1], v[3], v[5], v[7]};
  dft4<C, INV>(e);
  dft4<C, INV>(o);
  C w1, w2, w3;
  // o1 * W8^1, o2 * W8^2, o3 * W8^3 with W8 = (1 - i)/sqrt 2 forward, (1 + i)/sqrt 2 inverse
  if (INV) {
    w1.x = (o[1].x - o[1].y) * h; w1.y = (o[1].x + o[1].y) * h;
    w3.x = -(o[3].x + o[3].y) * h; w3.y = (o[3].x - o[3].y) * h;
  } else {
    w1.x = (o[1].x + o[1].y) * h; w1.y = (o[1].y - o[1].x) * h;
    w3.x = (o[3].y - o[3].x) * h; w3.y = -(o[3].x + o[3].y) * h;
  }
  w2 = hmul_mi<C, INV>(o[2]);
  v[0] = hadd(e[0], o[0]); v[4] = hsub(e[0], o[0]);
  v[1] = hadd(e[1], w1);   v[5] = hsub(e[1], w1);
  v[2] = hadd(e[2], w2);   v[6] = hsub(e[2], w2);
  v[3] = hadd(e[3], w3);   v[7] = hsub(e[3], w3);
}

// 8-point DFT of v[0..3] with v[4..7] = 0 (never read): the first pass of a transform whose
// input line is zero beyond its first half. Each 4-point DFT of two non-zero inputs a, b gives
// a + b, a + W4 b, a - b, a - W4 b.
template <typename C, bool INV> __host__ __device__ __forceinline__ void dft8_half_in(C *v) {
  using R = typename RealOf<C>::type;
  const R h = R(0.70710678118654752440);
  const C me = hmul_mi<C, INV>(v[2]), mo = hmul_mi<C, INV>(v[3]);
  C e[4] = {hadd(v[0], v[2]), hadd(v[0], me), hsub(v[0], v[2]), hsub(v[0], me)};
  C o[4] = {hadd(v[1], v[3]), hadd(v[1], mo), hsub(v[1], v[3]), hsub(v[1], mo)};
  C w1, w2, w3;
  if (INV) {
    w1.x = (o[1].x - o[1].y) * h; w1.y = (o[1].x + o[1].y) * h;
    w3.x = -(o[3].x + o[3].y) * h; w3.y = (o[3].x - o[3].y) * h;
  } else {
    w1.x = (o[1].x + o[1].y) * h; w1.y = (o[1].y - o[1].x) * h;
    w3.x = (o[3].y - o[3].x) * h; w3.y = -(o[3].x + o[3].y) * h;
  }
  w2 = hmul_mi<C, INV>(o[2]);
  v[0] = hadd(e[0], o[0]); v[4] = hsub(e[0], o[0]);
  v[1] = hadd(e[1], w1);   v[5] = hsub(e[1], w1);
  v[2] = hadd(e[2], w2);   v[6] = hsub(e[2], w2);
  v[3] = hadd(e[3], w3);   v[7] = hsub(e[3], w3);
}

template <typename C, int R, bool INV> __host__ __device__ __forceinline__ void dft(C *v) {
  if constexpr (R == 2) dft2<C, INV>(v);
  else if constexpr (R == 4) dft4<C, INV>(v);
  else if constexpr (R == 8) dft8<C, INV>(v);
  else static_assert(R == 2 || R == 4 || R == 8, "radix");
}

// Load, twiddle and transform the BPT butterflies of thread `tid` in one pass.
template <typename C, int L, int R, int NS, int NL, int LS, int NT, bool INV>
__host__ __device__ __forceinline__ void pass_compute(const C *s, const C *__restrict__ tw, int tid,
                                                      C (&v)[(NL * (L / R)) / NT][R]) {
  constexpr int Q = L / R;
  constexpr int BPT = (NL * Q) / NT;
  static_assert((NL * Q) % NT == 0, "threads must divide the butterflies of a pass");
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int q = tid + i * NT;
    const int line = q / Q, j = q - line * Q;
    const C *src = s + line * LS + j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = src[r * Q];
    if constexpr (NS > 1) {
      const int k = j % NS;
      constexpr int step = (kTwiddleN / L) * (L / (NS * R));
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * step];
        if (INV) w.y = -w.y;
        v[i][r] = hmul(v[i][r], w);
      }
    }
    dft<C, R, INV>(v[i]);
  }
}

template <typename C, int L, int R, int NS, int NL, int LS, int NT>
__host__ __device__ __forceinline__ void pass_store(C *s, int tid, const C (&v)[(NL * (L / R)) / NT][R]) {
  constexpr int Q = L / R;
  constexpr int BPT = (NL * Q) / NT;
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int q = tid + i * NT;
    const int line = q / Q, j = q - line * Q;
    const int k = j % NS;
    C *dst = s + line * LS + (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * NS] = v[i][r];
  }
}

#ifdef __CUDACC__
template <typename C, int L, int NS, int NL, int LS, int NT, bool INV, int R, int... REST>
__device__ __forceinline__ void fft_passes(C *s, const C *__restrict__ tw) {
  C v[(NL * (L / R)) / NT][R];
  pass_compute<C, L, R, NS, NL, LS, NT, INV>(s, tw, threadIdx.x, v);
  __syncthreads();
  pass_store<C, L, R, NS, NL, LS, NT>(s, threadIdx.x, v);
  __syncthreads();
  if constexpr (sizeof...(REST) > 0) fft_passes<C, L, NS * R, NL, LS, NT, INV, REST...>(s, tw);
}
#endif

// Radix sequence of each supported length (product = L).
template <int L> struct Plan;
#define DBI_PLAN(L_, ...)                                                                     \
  template <> struct Plan<L_> {                                                               \
    template <typename C, int NL, int LS, int NT, bool INV>                                   \
    __device__ __forceinline__ static void run(C *s, const C *__restrict__ tw) {              \
      fft_passes<C, L_, 1, NL, LS, NT, INV, __VA_ARGS__>(s, tw);                              \
    }                                                                                         \
  };
#ifdef __CUDACC__
DBI_PLAN(16, 4, 4)
DBI_PLAN(32, 8, 4)
DBI_PLAN(64, 8, 8)
DBI_PLAN(128, 8, 4, 4)
DBI_PLAN(256, 8, 8, 4)
DBI_PLAN(512, 8, 8, 8)
DBI_PLAN(1024, 8, 8, 4, 4)
#endif
#undef DBI_PLAN

// Call F.template operator()<L>() for the runtime length L (one of the supported lengths).
template <typename F> __host__ bool dispatch_len(int L, F &&f) {
  switch (L) {
    case 16: f.template operator()<16>(); return true;
    case 32: f.template operator()<32>(); return true;
    case 64: f.template operator()<64>(); return true;
    case 128: f.template operator()<128>(); return true;
    case 256: f.template operator()<256>(); return true;
    case 512: f.template operator()<512>(); return true;
    case 1024: f.template operator()<1024>(); return true;
    default: return false;
  }
}

}  // namespace dbi

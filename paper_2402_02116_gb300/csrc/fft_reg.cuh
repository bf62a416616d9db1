// Register-resident Stockham FFTs for the LS-operator kernels.
//
// A line of length L is transformed by T = L/8 threads; thread t holds the eight points
// x[t + m T], m = 0..7, in registers before and after the transform (the "natural" pattern,
// which makes the first pass read and the last pass write coalesced global addresses).
// Every radix-R pass (R = 2, 4 or 8) runs 8/R butterflies per thread: butterfly j = t + i T reads
// the points j + r L/R = t + (i + r 8/R) T of the registers, multiplies them by W_{Ns R}^{r (j mod
// Ns)} (Ns = product of the earlier radices), takes an R-point DFT and writes position
// (j - j mod Ns) R + j mod Ns + r Ns of the line (self-sorting Stockham order). Between passes the
// line goes through shared memory, padded as i + i/16 so that the strided writes of a warp hit
// distinct banks; the last pass writes position j + r L/R = t + (i + r 8/R) T, i.e. straight back
// into the registers in natural order.
//
// Forward transforms use exp(-2 pi i jk/L), inverse ones exp(+2 pi i jk/L), unnormalised;
// each butterfly reads one twiddle from tw[m] = exp(-2 pi i m / 3072) and forms its powers.
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace dbi {

// w^0 .. w^(R-1) from w^1 by at most three complex products each (error of a few ulp).
template <typename C, int R>
__host__ __device__ __forceinline__ void twiddle_powers(C w1, C (&w)[R]) {
  w[0].x = 1; w[0].y = 0;
  if constexpr (R > 1) w[1] = w1;
  if constexpr (R > 2) w[2] = hmul(w1, w1);
  if constexpr (R > 3) w[3] = hmul(w[2], w1);
  if constexpr (R > 4) w[4] = hmul(w[2], w[2]);
  if constexpr (R > 5) w[5] = hmul(w[4], w1);
  if constexpr (R > 6) w[6] = hmul(w[3], w[3]);
  if constexpr (R > 7) w[7] = hmul(w[4], w[3]);
}

template <typename C, int L> struct RegFFT {
  static constexpr int T = L / 8;                 // threads per line
  static constexpr int LP = L + L / 16 + 2;       // padded line length in shared memory
  static constexpr int TWS = kTwiddleN / L;       // table stride of W_L

  // One padding slot per 16 points: every store and gather pattern of the radix-8 passes then
  // needs the minimum two shared-memory wavefronts per warp (8-byte points).
  __host__ __device__ __forceinline__ static int pad(int i) { return i + (i >> 4); }

  // One radix-R pass from registers (pass input in natural order) into a shared-memory line.
  // HIN: the line is zero beyond its first half (first pass only: R = 8, NS = 1, so v[4..7]
  // are those zeros and are not read).
  template <int R, int NS, bool INV, bool HIN = false>
  __host__ __device__ __forceinline__ static void pass(const C (&v)[8], C *line, int t,
                                                      const C *__restrict__ tw) {
    constexpr int NB = 8 / R;
    static_assert(!HIN || (R == 8 && NS == 1), "half-zero input only in a first radix-8 pass");
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * T;
      C x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = (HIN && r >= 4) ? v[0] : v[i + r * NB];
      const int k = j % NS;
      if constexpr (NS > 1) {
        C w1 = tw[k * (L / (NS * R)) * TWS];
        if (INV) w1.y = -w1.y;
        C w[R];
        twiddle_powers<C, R>(w1, w);
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = hmul(x[r], w[r]);
      }
      if constexpr (HIN) dft8_half_in<C, INV>(x);
      else dft<C, R, INV>(x);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[pad(base + r * NS)] = x[r];
    }
  }

  // Load the next pass's input (natural order) from a shared-memory line.
  __host__ __device__ __forceinline__ static void gather(C (&v)[8], const C *line, int t) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = line[pad(t + m * T)];
  }

  // The last pass (NS = L / R): its outputs land in the registers in natural order.
  template <int R, bool INV>
  __host__ __device__ __forceinline__ static void last(C (&v)[8], int t, const C *__restrict__ tw) {
    constexpr int NB = 8 / R, NS = L / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * T;
      C x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = v[i + r * NB];
      C w1 = tw[j * TWS];  // W_{NS R}^{r j} = W_L^{r j}
      if (INV) w1.y = -w1.y;
      C w[R];
      twiddle_powers<C, R>(w1, w);
#pragma unroll
      for (int r = 1; r < R; ++r) x[r] = hmul(x[r], w[r]);
      dft<C, R, INV>(x);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i + r * NB] = x[r];
      (void)NS;
    }
  }
};

// Radix plans (8 values per thread; the product of the radices is L). run() transforms the NLT
// lines held by the calling thread; sync() must order the shared-memory accesses of every thread
// that shares those lines (a barrier over at least the line's T threads).
template <int N> using IC = std::integral_constant<int, N>;

// HIN: every line is zero beyond its first half (v[l][4..7] = 0 on entry; they are not read).
template <int L> struct RegPlan {
  template <typename C, int NLT, bool INV, bool HIN = false, typename Sync>
  __host__ __device__ __forceinline__ static void run(C (&v)[NLT][8], C *const (&lines)[NLT], int t,
                                                      const C *__restrict__ tw, Sync &&sync) {
    using F = RegFFT<C, L>;
    auto step = [&](auto r_, auto ns_) {
      constexpr int R = decltype(r_)::value, NS = decltype(ns_)::value;
      constexpr bool H = HIN && NS == 1;
#pragma unroll
      for (int l = 0; l < NLT; ++l) F::template pass<R, NS, INV, H>(v[l], lines[l], t, tw);
      sync();
#pragma unroll
      for (int l = 0; l < NLT; ++l) F::gather(v[l], lines[l], t);
      sync();
    };
    auto fin = [&](auto r_) {
      constexpr int R = decltype(r_)::value;
#pragma unroll
      for (int l = 0; l < NLT; ++l) F::template last<R, INV>(v[l], t, tw);
    };
    if constexpr (L == 16) { step(IC<8>{}, IC<1>{}); fin(IC<2>{}); }
    else if constexpr (L == 32) { step(IC<8>{}, IC<1>{}); fin(IC<4>{}); }
    else if constexpr (L == 64) { step(IC<8>{}, IC<1>{}); fin(IC<8>{}); }
    else if constexpr (L == 128) { step(IC<8>{}, IC<1>{}); step(IC<8>{}, IC<8>{}); fin(IC<2>{}); }
    else if constexpr (L == 256) { step(IC<8>{}, IC<1>{}); step(IC<8>{}, IC<8>{}); fin(IC<4>{}); }
    else if constexpr (L == 512) { step(IC<8>{}, IC<1>{}); step(IC<8>{}, IC<8>{}); fin(IC<8>{}); }
    else if constexpr (L == 1024) {
      step(IC<8>{}, IC<1>{}); step(IC<8>{}, IC<8>{}); step(IC<8>{}, IC<64>{}); fin(IC<2>{});
    } else {
      static_assert(L == 16, "unsupported FFT length");
    }
  }
};

}  // namespace dbi

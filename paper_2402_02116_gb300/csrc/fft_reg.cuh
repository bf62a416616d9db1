// Register-resident Stockham FFTs for the LS-operator kernels.
//
// A line of length L is transformed by T = L/8 threads; thread t holds the eight points
// x[t + m T], m = 0..7, in registers before and after the transform (the "natural" pattern,
// which makes the first pass read and the last pass write coalesced global addresses).
// Every radix-R pass (R = 2, 4 or 8) runs 8/R butterflies per thread: butterfly j = t + i T reads
// the points j + r L/R = t + (i + r 8/R) T of the registers, multiplies them by W_{Ns R}^{r (j mod
// Ns)} (Ns = product of the earlier radices), takes an R-point DFT and writes position
// (j - j mod Ns) R + j mod Ns + r Ns of the line (self-sorting Stockham order). Between passes the
// line goes through shared memory, laid out so that the strided writes of a warp hit distinct banks
// (padding or an XOR swizzle, per exchange); the last pass writes position j + r L/R = t +
// (i + r 8/R) T, i.e. straight back into the registers in natural order.
//
// Forward transforms use exp(-2 pi i jk/L), inverse ones exp(+2 pi i jk/L), unnormalised.
// A thread's twiddles depend only on t and the pass, so each kernel reads them once from the
// table tw[m] = exp(-2 pi i m / 3072) into a TwReg (one base twiddle per butterfly of every
// twiddled pass); each pass forms the powers once and applies them to all the thread's lines.
//
// Radix plans: V = 0 puts the radix-8 passes first and a smaller radix last; V = 1 puts the
// smaller radix first (the two coincide when L is a power of 8). Both are exact orderings of the
// same factorisation; which one runs faster depends on the length and is measured at run time.
#pragma once

#include <type_traits>
#include <utility>

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

// R-point DFT of x[0 .. R/2) with x[R/2 .. R) = 0 (not read).
template <typename C, int R, bool INV> __host__ __device__ __forceinline__ void dft_half_in(C *x) {
  if constexpr (R == 2) {
    x[1] = x[0];
  } else if constexpr (R == 4) {
    const C a = x[0], b = x[1], mb = hmul_mi<C, INV>(b);
    x[0] = hadd(a, b); x[1] = hadd(a, mb); x[2] = hsub(a, b); x[3] = hsub(a, mb);
  } else {
    dft8_half_in<C, INV>(x);
  }
}

// Radix sequence of a plan.
template <int L, int V> struct Radices;
template <> struct Radices<16, 0> { static constexpr int n = 2, r[2] = {8, 2}; };
template <> struct Radices<16, 1> { static constexpr int n = 2, r[2] = {2, 8}; };
template <> struct Radices<32, 0> { static constexpr int n = 2, r[2] = {8, 4}; };
template <> struct Radices<32, 1> { static constexpr int n = 2, r[2] = {4, 8}; };
template <> struct Radices<64, 0> { static constexpr int n = 2, r[2] = {8, 8}; };
template <> struct Radices<64, 1> { static constexpr int n = 2, r[2] = {8, 8}; };
template <> struct Radices<128, 0> { static constexpr int n = 3, r[3] = {8, 8, 2}; };
template <> struct Radices<128, 1> { static constexpr int n = 3, r[3] = {2, 8, 8}; };
template <> struct Radices<256, 0> { static constexpr int n = 3, r[3] = {8, 8, 4}; };
template <> struct Radices<256, 1> { static constexpr int n = 3, r[3] = {4, 8, 8}; };
template <> struct Radices<512, 0> { static constexpr int n = 3, r[3] = {8, 8, 8}; };
template <> struct Radices<512, 1> { static constexpr int n = 3, r[3] = {8, 8, 8}; };
template <> struct Radices<1024, 0> { static constexpr int n = 4, r[4] = {8, 8, 8, 2}; };
template <> struct Radices<1024, 1> { static constexpr int n = 4, r[4] = {2, 8, 8, 8}; };

template <int L, int V> struct PlanInfo {
  using Rd = Radices<L, V>;
  static constexpr int np = Rd::n;
  static constexpr int radix(int p) { return Rd::r[p]; }
  static constexpr int ns(int p) {  // product of the radices before pass p
    int s = 1;
    for (int q = 0; q < p; ++q) s *= Rd::r[q];
    return s;
  }
  static constexpr int woff(int p) {  // first base twiddle of pass p in the TwReg
    int o = 0;
    for (int q = 1; q < p; ++q) o += 8 / Rd::r[q];
    return o;
  }
  static constexpr int nw = woff(np);  // base twiddles per thread (passes 1 .. np-1)
};

// Line layout of exchange p (after pass p) of each plan: the cheapest layout (RegFFT::pad) whose
// stores and loads need the fewest shared-memory wavefronts, found by counting the wavefronts of
// every access of every layout for each plan, with 8-byte points served half a warp at a time
// (one line per warp from L = 256; two or more below, at the line pitch RegFFT::LP, chosen with
// the layouts for L <= 64).
template <int L, int V> constexpr int layout_of(int p) {
  if constexpr (L == 16) return V == 0 ? 3 : 0;
  else if constexpr (L == 32) return 3;
  else if constexpr (L == 64) return 3;
  else if constexpr (L == 128 || L == 256) return (p == 1 && V == 0) ? 2 : 1;
  else if constexpr (L == 512) return p == 0 ? 1 : 2;
  else return p == 0 ? 1 : (p == 1 ? (V == 0 ? 2 : 1) : 0);
}

template <typename C, int L, int V = 0> struct TwReg {
  static constexpr int NW = PlanInfo<L, V>::nw;
  C w[NW];
  // Base twiddles W_{Ns R}^{j mod Ns} of thread t's butterflies j = t + i L/8 in every pass > 0.
  __host__ __device__ __forceinline__ TwReg(int t, const C *__restrict__ tw) {
    using P = PlanInfo<L, V>;
    constexpr int TWS = kTwiddleN / L, T = L / 8;
    [&]<int... p>(std::integer_sequence<int, p...>) {
      (
          [&] {
            constexpr int q = p + 1, R = P::radix(q), NS = P::ns(q), NB = 8 / R;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
              const int k = (t + i * T) % NS;
              w[P::woff(q) + i] = tw[k * (L / (NS * R)) * TWS];
            }
          }(),
          ...);
    }(std::make_integer_sequence<int, P::np - 1>{});
  }
};

template <typename C, int L> struct RegFFT {
  static constexpr int T = L / 8;                 // threads per line
  // padded line length (and pitch of consecutive lines) in shared memory
  static constexpr int LP = L == 16 ? 18 : L == 64 ? 72 : L + L / 16 + 2;
  static constexpr int TWS = kTwiddleN / L;       // table stride of W_L

  // Position of point i of a line in shared memory, by layout (chosen per exchange, see
  // layout_of): 0 = i; 1 = i + i/16 (one padding slot per 16 points); 2 = inside each 16-point
  // block, the low four bits XORed with the block index (bits 0-2) and with bit 2 of the block
  // index moved to bit 3 (a bijection on every block); 3 = i + i/8 (one padding slot per 8
  // points: with several lines per warp at a pitch of 8 mod 16 the scatter of the first radix-8
  // pass and the natural-order gather both spread two lines over 16 bank slots).
  template <int LAY> __host__ __device__ __forceinline__ static int pad(int i) {
    if constexpr (LAY == 0) {
      return i;
    } else if constexpr (LAY == 1) {
      return i + (i >> 4);
    } else if constexpr (LAY == 3) {
      return i + (i >> 3);
    } else {
      const int h = i >> 4;
      return (i & ~15) | ((i & 15) ^ ((((h >> 2) & 1) << 3) | (h & 7)));
    }
  }

  // The NB = 8/R butterflies of one pass on registers in natural order: twiddle by the powers
  // wp[i][r] (NS > 1), R-point DFT. HIN (first pass only): v[4..7] are zero and not read.
  template <int R, int NS, bool INV, bool HIN>
  __host__ __device__ __forceinline__ static void butterflies(C (&v)[8], const C (&wp)[8 / R][R]) {
    constexpr int NB = 8 / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      C x[R];
#pragma unroll
      for (int r = 0; r < R; ++r) x[r] = (HIN && i + r * NB >= 4) ? v[0] : v[i + r * NB];
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = hmul(x[r], wp[i][r]);
      }
      if constexpr (HIN) dft_half_in<C, R, INV>(x);
      else dft<C, R, INV>(x);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i + r * NB] = x[r];
    }
  }

  // Store a pass's outputs (held in v as produced by butterflies()) at their Stockham positions.
  template <int R, int NS, int LAY>
  __host__ __device__ __forceinline__ static void scatter(const C (&v)[8], C *line, int t) {
    constexpr int NB = 8 / R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * T, k = j % NS, base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[pad<LAY>(base + r * NS)] = v[i + r * NB];
    }
  }

  // Load the next pass's input (natural order) from a shared-memory line.
  template <int LAY> __host__ __device__ __forceinline__ static void gather(C (&v)[8], const C *line, int t) {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = line[pad<LAY>(t + m * T)];
  }
};

// Powers of the NB base twiddles of one pass (conjugated for an inverse transform).
template <typename C, int R, bool INV, int NB>
__host__ __device__ __forceinline__ void pass_powers(const C *w1, C (&wp)[NB][R]) {
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    C b = w1[i];
    if (INV) b.y = -b.y;
    C pw[R];
    twiddle_powers<C, R>(b, pw);
#pragma unroll
    for (int r = 0; r < R; ++r) wp[i][r] = pw[r];
  }
}

// run() transforms the NLT lines held by the calling thread; sync() must order the shared-memory
// accesses of every thread that shares those lines (a barrier over at least the line's T threads).
// HIN: every line is zero beyond its first half (v[l][4..7] = 0 on entry; they are not read).
template <int L, int V = 0> struct RegPlan {
  template <typename C, int NLT, bool INV, bool HIN = false, typename Sync>
  __host__ __device__ __forceinline__ static void run(C (&v)[NLT][8], C *const (&lines)[NLT], int t,
                                                      const TwReg<C, L, V> &tr, Sync &&sync) {
    using F = RegFFT<C, L>;
    using P = PlanInfo<L, V>;
    [&]<int... p>(std::integer_sequence<int, p...>) {
      (
          [&] {
            constexpr int R = P::radix(p), NS = P::ns(p), NB = 8 / R;
            constexpr bool H = HIN && p == 0, LAST = p == P::np - 1;
            C wp[NB][R];
            if constexpr (NS > 1) pass_powers<C, R, INV, NB>(tr.w + P::woff(p), wp);
#pragma unroll
            for (int l = 0; l < NLT; ++l) F::template butterflies<R, NS, INV, H>(v[l], wp);
            if constexpr (!LAST) {
              constexpr int LAY = layout_of<L, V>(p);
#pragma unroll
              for (int l = 0; l < NLT; ++l) F::template scatter<R, NS, LAY>(v[l], lines[l], t);
              sync();
#pragma unroll
              for (int l = 0; l < NLT; ++l) F::template gather<LAY>(v[l], lines[l], t);
              sync();
            }
          }(),
          ...);
    }(std::make_integer_sequence<int, P::np>{});
  }
};

}  // namespace dbi

// Tile bodies of the three LS-operator stages (Eq. 6, 10, 12), shared by the batched kernels of
// one grid size (ls_operator.cu) and the persistent kernels over problems of uneven sizes
// (group.cu). A tile is the work of one 256-thread CTA:
//   rows_forward_tile  : ROWS = 2048 / L rows of one problem: contrast source by central
//                        differences (fields zero outside D), zero-pad to lx, forward FFT along x,
//                        transpose through shared memory into the column-major spectra T[c][kx][z]
//   cols_tile          : CC = 2048 / L columns kx of one problem: forward FFT along z of the nz
//                        non-zero rows padded to lz, 2x2 multiply by Ghat(kz, kx), inverse FFT
//                        along z, keep z < nz
//   rows_inverse_tile  : ROWS rows: transpose back, inverse FFT along x, keep x < nx,
//                        out = ident - result (or the result), with the Krylov inner products of
//                        the output fused into the epilogue (EPI 1, 2)
// Ghat already carries h^2 / (lz lx), so no other scaling is applied.
#pragma once

#include "fft_reg.cuh"
#include "reduce.cuh"

namespace dbi {

// Launch shapes: 256 threads per CTA for every length. Rows: ROWS rows per CTA, T = L/8 threads
// per row (t fastest), both components of a row held by each thread. Columns: CC columns per CTA,
// thread (c, t) with t fastest so that a warp reads a contiguous run of one column.
template <typename C> struct Cfg;
#ifndef DBI_COLS_MIN_BLOCKS
#define DBI_COLS_MIN_BLOCKS 4
#endif
#ifndef DBI_ROWS_INV_MIN_BLOCKS
#define DBI_ROWS_INV_MIN_BLOCKS 4
#endif
#ifndef DBI_ROWS_FWD_MIN_BLOCKS
#define DBI_ROWS_FWD_MIN_BLOCKS 4
#endif
template <> struct Cfg<float2> {
  static constexpr int threads = 256;
  static constexpr int colMinBlocks = DBI_COLS_MIN_BLOCKS, rowInvMinBlocks = DBI_ROWS_INV_MIN_BLOCKS;
  // rows forward: 4 CTAs per SM up to L = 512 (64 registers); L = 1024 tiles need 99 KB of shared
  // memory, so only 2 fit and the registers are left free
  static constexpr int rowFwdMinBlocks(int L) { return L >= 1024 ? 2 : DBI_ROWS_FWD_MIN_BLOCKS; }
};
template <> struct Cfg<double2> {
  static constexpr int threads = 256, colMinBlocks = 1, rowInvMinBlocks = 1;
  static constexpr int rowFwdMinBlocks(int) { return 2; }
};
constexpr int kTileThreads = 256;

template <typename C, int LX> struct RowCfg {
  static constexpr int T = LX / 8;
  static constexpr int ROWS = kTileThreads / T;
  static constexpr int NT = ROWS * T;
  static constexpr int LP = RegFFT<C, LX>::LP;
};
template <typename C, int LZ> struct ColCfg {
  static constexpr int T = LZ / 8;
  static constexpr int CC = kTileThreads / T;  // named barriers 1..CC only when T > 32 (CC <= 4)
  static constexpr int NT = CC * T;
  static constexpr int LP = RegFFT<C, LZ>::LP;
};
// Every line holds its data in its first half: the entry points require lz >= 2 nz - 1 and
// lx >= 2 nx - 1, so a cell index t + m L/8 < n <= L/2 has m < 4. Points m = 4..7 are zero on
// input to a forward transform and never needed on output of an inverse one.
constexpr int kHalf = 4;

// Transposition tile of the rows kernels: [2][LX][ROWS + 1] (padded against bank conflicts).
template <typename C, int LX> constexpr size_t tile_elems() {
  return size_t(2) * LX * (RowCfg<C, LX>::ROWS + 1);
}

// Lengths whose stencil uses the strip form (one column per thread, few rows per tile).
#ifndef DBI_STRIP_256
#define DBI_STRIP_256 0  // at L = 256 the strip needs 150 registers and loses to the shared-memory form
#endif
#ifndef DBI_STRIP_1024
#define DBI_STRIP_1024 1
#endif
template <typename C, int LX>
constexpr bool kStripStencil = LX == 512 || (LX == 1024 && DBI_STRIP_1024 && sizeof(C) == 8) ||
                               (LX == 256 && DBI_STRIP_256);  // complex128 at 1024 would spill

// Shared memory of the strip stencil (bytes): u at ROWS + 2 rows, sigma1 and sigma5 at ROWS rows.
template <typename C, int LX> inline size_t stencil_strip_smem(int nx) {
  constexpr int ROWS = RowCfg<C, LX>::ROWS;
  return (size_t(2) * (ROWS + 2) + size_t(2) * ROWS) * (nx + 2) * sizeof(C);
}

// Dynamic shared memory of each stage (bytes).
template <typename C, int LX> inline size_t rows_forward_smem(int nx, bool stencil) {
  using RC = RowCfg<C, LX>;
  const size_t lines = size_t(2) * RC::ROWS * RC::LP * sizeof(C);
  const size_t tile = tile_elems<C, LX>() * sizeof(C);
  size_t sg = 0;
  if (stencil) {
    if constexpr (kStripStencil<C, LX>) sg = stencil_strip_smem<C, LX>(nx);
    else sg = (size_t(3) * (RC::ROWS + 2) + size_t(2) * (RC::ROWS + 4)) * (nx + 2) * sizeof(C);
  }
  return std::max(std::max(lines, tile), sg);
}
template <typename C, int LZ> inline size_t cols_smem() {
  using CF = ColCfg<C, LZ>;
  return size_t(2) * CF::CC * CF::LP * sizeof(C);
}
template <typename C, int LX> inline size_t rows_inverse_smem() {
  using RC = RowCfg<C, LX>;
  return std::max(size_t(2) * RC::ROWS * RC::LP, tile_elems<C, LX>()) * sizeof(C);
}

// Barrier over the threads that share a line: the T threads of one row or column.
template <int T> struct RowSync {
  int id;
  __device__ __forceinline__ void operator()() const {
    if constexpr (T <= 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(T) : "memory");
    }
  }
};

// Everything a tile needs about its problem (one (source, frequency) wavefield on one grid).
// The tile bodies read it through an accessor with the member functions below: TileArgs holds the
// values (the persistent kernels build one per tile); the batched kernels of one grid use an
// accessor that reads its kernel parameters where they are used (ls_operator.cu).
template <typename C> struct TileArgs {
  using Rl = typename RealOf<C>::type;
  int nz_, nx_, lz_, lx_;
  Rl inv2h_;
  int b_, f_;                  // the problem (scale index) and its frequency
  const double *omega_;        // [nf] angular frequencies
  const double *in_scale_;     // [B] power-of-two input scales or NULL (1)
  const double *out_scale_;    // [B] output scales or NULL (1)
  const double *m_scale_;      // [1] contrast scale or NULL (1)
  const Rl *m_;                // [5][nz][nx] model or perturbation
  Rl ref_[5];                  // subtracted from m
  const C *in_;                // [2][nz][nx] this problem's input
  const C *ident_;             // [2][nz][nx] identity term or NULL
  C *out_;                     // [2][nz][nx]
  C *T_;                       // [2][lx][nz] this problem's column-major spectra
  const C *G_;                 // [3][lx][lz] Ghat of the problem's frequency (column-major)
  const C *tw_;                // twiddle table
  const C *krhat_;             // [2][nz][nx] shadow residual (EPI 1)
  double *part_;               // [row tiles][kRedSlots] fused inner-product partials (EPI 1, 2)
  __device__ __forceinline__ int nz() const { return nz_; }
  __device__ __forceinline__ int nx() const { return nx_; }
  __device__ __forceinline__ int lx() const { return lx_; }
  __device__ __forceinline__ Rl inv2h() const { return inv2h_; }
  __device__ __forceinline__ Rl ref(int i) const { return ref_[i]; }
  __device__ __forceinline__ const Rl *m() const { return m_; }
  __device__ __forceinline__ const C *in() const { return in_; }
  __device__ __forceinline__ const C *ident() const { return ident_; }
  __device__ __forceinline__ C *out() const { return out_; }
  __device__ __forceinline__ C *T() const { return T_; }
  __device__ __forceinline__ const C *G() const { return G_; }
  __device__ __forceinline__ const C *tw() const { return tw_; }
  __device__ __forceinline__ const C *krhat() const { return krhat_; }
  __device__ __forceinline__ double *part() const { return part_; }
  __device__ __forceinline__ Rl w2() const {
    const double om = omega_[f_];
    return Rl(om * om);
  }
  __device__ __forceinline__ Rl isc() const { return in_scale_ ? Rl(in_scale_[b_]) : Rl(1); }
  __device__ __forceinline__ Rl osc() const { return out_scale_ ? Rl(out_scale_[b_]) : Rl(1); }
  __device__ __forceinline__ Rl ms() const { return m_scale_ ? Rl(m_scale_[0]) : Rl(1); }
};

// Stress sigma = dC eps at cell (z, x) of D (zero outside D), from the staged u (rows z0 - 2 ..
// z0 + ROWS + 1 with a zero column on each side; u already multiplied by its input scale).
template <typename C, typename A>
__device__ __forceinline__ void stress_at(const A &a, const C *su, int RS, int W, int z0, int z,
                                          int x, typename RealOf<C>::type ms, C &s1, C &s3, C &s5) {
  using Rl = typename RealOf<C>::type;
  const int nz = a.nz(), nx = a.nx();
  if (z < 0 || z >= nz || x < 0 || x >= nx) {
    s1 = s3 = s5 = czero<C>();
    return;
  }
  auto U = [&](int c, int zz, int xx) { return su[(c * RS + (zz - z0 + 2)) * W + xx + 1]; };
  const Rl f = a.inv2h();
  const C e1 = cscale(csub(U(0, z, x + 1), U(0, z, x - 1)), f);
  const C e3 = cscale(csub(U(1, z + 1, x), U(1, z - 1, x)), f);
  const C e5 = cscale(cadd(csub(U(0, z + 1, x), U(0, z - 1, x)), csub(U(1, z, x + 1), U(1, z, x - 1))), f);
  const size_t cell = size_t(z) * nx + x, plane = size_t(nz) * nx;
  const Rl d11 = (__ldg(a.m() + 1 * plane + cell) - a.ref(1)) * ms;
  const Rl d13 = (__ldg(a.m() + 2 * plane + cell) - a.ref(2)) * ms;
  const Rl d33 = (__ldg(a.m() + 3 * plane + cell) - a.ref(3)) * ms;
  const Rl d55 = (__ldg(a.m() + 4 * plane + cell) - a.ref(4)) * ms;
  s1 = cadd(cscale(e1, d11), cscale(e3, d13));
  s3 = cadd(cscale(e1, d13), cscale(e3, d33));
  s5 = cscale(e5, d55);
}

// Contrast source of the tile's ROWS rows with KC = L/512 columns per thread (the "strip" form,
// for lengths whose tiles have few rows): the thread keeps its columns' u and stress in registers
// along z, so only the x-neighbours go through shared memory (u at the stress rows, sigma1 and
// sigma5 at the output rows); the sources then pass through shared memory once more into the FFT
// layout v[c][m] = s_c(z0 + rr, t + m L/8). Columns x = threadIdx.x + k blockDim.x, k < KC.
template <typename C, int LX, typename A>
__device__ __forceinline__ void stencil_strip(const A &a, int z0, C *smem, C (&v)[2][8]) {
  using Rl = typename RealOf<C>::type;
  using RC = RowCfg<C, LX>;
  constexpr int ROWS = RC::ROWS, T = RC::T, RS = ROWS + 4, RG = ROWS + 2;
  constexpr int KC = (LX / 2 + kTileThreads - 1) / kTileThreads;  // nx <= L/2 columns
  const int nz = a.nz(), nx = a.nx(), W = nx + 2;
  const size_t plane = size_t(nz) * nx;
  const C *u1 = a.in(), *u3 = u1 + plane;
  C *su = smem;                               // [2][RG][W]: u at the stress rows z0 - 1 .. z0 + ROWS
  C *sg = smem + size_t(2) * RG * W;          // [2][ROWS][W]: sigma1, sigma5 at the output rows
  C *so = smem;                               // [2][ROWS][nx]: the sources (reuses su)
  // u of the columns at rows z0 - 2 .. z0 + ROWS + 1 (zero outside D), scaled
  const Rl isc = a.isc();
  C U1[KC][RS], U3[KC][RS];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int x = threadIdx.x + k * kTileThreads;
#pragma unroll
    for (int r = 0; r < RS; ++r) {
      const int zz = z0 - 2 + r;
      const bool in = x < nx && zz >= 0 && zz < nz;
      U1[k][r] = in ? cscale(__ldg(u1 + size_t(zz) * nx + x), isc) : czero<C>();
      U3[k][r] = in ? cscale(__ldg(u3 + size_t(zz) * nx + x), isc) : czero<C>();
    }
  }
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int x = threadIdx.x + k * kTileThreads;
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      if (x < nx) {
        su[(0 * RG + r) * W + x + 1] = U1[k][r + 1];
        su[(1 * RG + r) * W + x + 1] = U3[k][r + 1];
      }
    }
  }
  if (threadIdx.x < 2 * RG) {  // the zero columns x = -1 and x = nx of every staged row
    su[size_t(threadIdx.x) * W] = czero<C>();
    su[size_t(threadIdx.x) * W + nx + 1] = czero<C>();
  } else if (threadIdx.x < 2 * RG + 2 * ROWS) {
    const int q = threadIdx.x - 2 * RG;
    sg[size_t(q) * W] = czero<C>();
    sg[size_t(q) * W + nx + 1] = czero<C>();
  }
  __syncthreads();
  // stress at rows z0 - 1 .. z0 + ROWS (zero outside D): sigma3, sigma5 kept in registers for the
  // z-derivatives, sigma1 and sigma5 of the output rows stored for the x-derivatives
  const Rl f = a.inv2h(), ms = a.ms();
  C S3[KC][RG], S5[KC][RG];
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int x = threadIdx.x + k * kTileThreads;
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      const int zz = z0 - 1 + r;
      C s1 = czero<C>(), s3 = czero<C>(), s5 = czero<C>();
      if (x < nx && zz >= 0 && zz < nz) {
        const C *r1 = su + (0 * RG + r) * W + x + 1, *r3 = su + (1 * RG + r) * W + x + 1;
        const C e1 = cscale(csub(r1[1], r1[-1]), f);
        const C e3 = cscale(csub(U3[k][r + 2], U3[k][r]), f);
        const C e5 = cscale(cadd(csub(U1[k][r + 2], U1[k][r]), csub(r3[1], r3[-1])), f);
        const size_t cell = size_t(zz) * nx + x;
        const Rl d11 = (__ldg(a.m() + 1 * plane + cell) - a.ref(1)) * ms;
        const Rl d13 = (__ldg(a.m() + 2 * plane + cell) - a.ref(2)) * ms;
        const Rl d33 = (__ldg(a.m() + 3 * plane + cell) - a.ref(3)) * ms;
        const Rl d55 = (__ldg(a.m() + 4 * plane + cell) - a.ref(4)) * ms;
        s1 = cadd(cscale(e1, d11), cscale(e3, d13));
        s3 = cadd(cscale(e1, d13), cscale(e3, d33));
        s5 = cscale(e5, d55);
      }
      S3[k][r] = s3;
      S5[k][r] = s5;
      if (r >= 1 && r <= ROWS && x < nx) {
        sg[(0 * ROWS + r - 1) * W + x + 1] = s1;
        sg[(1 * ROWS + r - 1) * W + x + 1] = s5;
      }
    }
  }
  __syncthreads();
  // s1 = w^2 drho u1 + d1 sigma1 + d3 sigma5, s3 = w^2 drho u3 + d1 sigma5 + d3 sigma3
  const Rl w2 = a.w2();
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int x = threadIdx.x + k * kTileThreads;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int z = z0 + r;
      if (x < nx && z < nz) {
        const C *g1 = sg + (0 * ROWS + r) * W + x + 1, *g5 = sg + (1 * ROWS + r) * W + x + 1;
        C o1 = cadd(csub(g1[1], g1[-1]), csub(S5[k][r + 2], S5[k][r]));
        C o3 = cadd(csub(g5[1], g5[-1]), csub(S3[k][r + 2], S3[k][r]));
        o1 = cscale(o1, f);
        o3 = cscale(o3, f);
        const Rl wr = w2 * (__ldg(a.m() + size_t(z) * nx + x) - a.ref(0)) * ms;
        so[(0 * ROWS + r) * nx + x] = cadd(o1, cscale(U1[k][r + 2], wr));
        so[(1 * ROWS + r) * nx + x] = cadd(o3, cscale(U3[k][r + 2], wr));
      }
    }
  }
  __syncthreads();
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int xm = t + m * T;
    const bool in = m < kHalf && z < nz && xm < nx;
    v[0][m] = in ? so[(0 * ROWS + rr) * nx + xm] : czero<C>();
    v[1][m] = in ? so[(1 * ROWS + rr) * nx + xm] : czero<C>();
  }
  __syncthreads();  // the FFT lines reuse the buffers
}

// Contrast source (or the raw source) of ROWS rows, zero-padded to LX, forward FFT along x.
//   stencil: stress of rows z0-1 .. z0+ROWS (each computed once, kept in shared memory), then
//            s1 = w^2 drho u1 + d1 sigma1 + d3 sigma5, s3 = w^2 drho u3 + d1 sigma5 + d3 sigma3.
template <typename C, int LX, bool STENCIL, int V, typename A>
__device__ __forceinline__ void rows_forward_tile(const A &a, int tile, C *smem) {
  using Rl = typename RealOf<C>::type;
  using RC = RowCfg<C, LX>;
  constexpr int ROWS = RC::ROWS, T = RC::T, LP = RC::LP;
  const int z0 = tile * ROWS;
  const int nz = a.nz(), nx = a.nx();
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  const size_t plane = size_t(nz) * nx;
  const C *u1 = a.in(), *u3 = u1 + plane;
  const Rl isc = a.isc();
  const TwReg<C, LX, V> tr(t, a.tw());
  C v[2][8];

  if constexpr (STENCIL && kStripStencil<C, LX>) {
    stencil_strip<C, LX>(a, z0, smem, v);
  } else if constexpr (STENCIL) {
    const int W = nx + 2;          // rows with one zero column on each side
    constexpr int RS = ROWS + 4;   // staged u rows z0 - 2 .. z0 + ROWS + 1
    C *sg = smem;                  // [3][ROWS + 2][W] stress
    C *su = smem + size_t(3) * (ROWS + 2) * W;  // [2][RS][W] u
    // stage u (rows x columns loops: no runtime division in the index arithmetic)
    constexpr int KW = (LX / 2 + 2 + RC::NT - 1) / RC::NT;  // column sweeps: W <= LX / 2 + 2
    constexpr int UR = RS <= 12 ? RS : 2;                    // full unroll for the few-row shapes
#pragma unroll UR
    for (int r = 0; r < RS; ++r) {
      const int zz = z0 - 2 + r;
      const bool row = zz >= 0 && zz < nz;
      C c1[KW], c3[KW];
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int xx = int(threadIdx.x) - 1 + k * RC::NT;
        const bool in = row && xx >= 0 && xx < nx;
        c1[k] = in ? cscale(__ldg(u1 + size_t(zz) * nx + xx), isc) : czero<C>();
        c3[k] = in ? cscale(__ldg(u3 + size_t(zz) * nx + xx), isc) : czero<C>();
      }
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int xx = int(threadIdx.x) - 1 + k * RC::NT;
        if (xx <= nx) {
          su[(0 * RS + r) * W + xx + 1] = c1[k];
          su[(1 * RS + r) * W + xx + 1] = c3[k];
        }
      }
    }
    __syncthreads();
    const Rl ms = a.ms();
#pragma unroll UR
    for (int r2 = 0; r2 < ROWS + 2; ++r2) {
      const int zz = z0 - 1 + r2;
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int xx = int(threadIdx.x) - 1 + k * RC::NT;
        if (xx <= nx) {
          C a1, a3, a5;
          stress_at(a, su, RS, W, z0, zz, xx, ms, a1, a3, a5);
          sg[(0 * (ROWS + 2) + r2) * W + xx + 1] = a1;
          sg[(1 * (ROWS + 2) + r2) * W + xx + 1] = a3;
          sg[(2 * (ROWS + 2) + r2) * W + xx + 1] = a5;
        }
      }
    }
    __syncthreads();
    const Rl w2 = a.w2();
    auto S = [&](int c, int r2, int xx) { return sg[(c * (ROWS + 2) + r2) * W + xx + 1]; };
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x = t + m * T;
      C o1 = czero<C>(), o3 = czero<C>();
      if (m < kHalf && z < nz && x < nx) {
        const int r2 = rr + 1;
        o1 = cadd(csub(S(0, r2, x + 1), S(0, r2, x - 1)), csub(S(2, r2 + 1, x), S(2, r2 - 1, x)));
        o3 = cadd(csub(S(2, r2, x + 1), S(2, r2, x - 1)), csub(S(1, r2 + 1, x), S(1, r2 - 1, x)));
        o1 = cscale(o1, a.inv2h());
        o3 = cscale(o3, a.inv2h());
        const size_t cell = size_t(z) * nx + x;
        const Rl wr = w2 * (__ldg(a.m() + cell) - a.ref(0)) * ms;
        o1 = cadd(o1, cscale(su[(0 * RS + rr + 2) * W + x + 1], wr));
        o3 = cadd(o3, cscale(su[(1 * RS + rr + 2) * W + x + 1], wr));
      }
      v[0][m] = o1;
      v[1][m] = o3;
    }
    __syncthreads();  // the FFT lines reuse the staging buffers
  } else {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x = t + m * T;
      const bool in = m < kHalf && z < nz && x < nx;
      v[0][m] = in ? cscale(__ldg(u1 + size_t(z) * nx + x), isc) : czero<C>();
      v[1][m] = in ? cscale(__ldg(u3 + size_t(z) * nx + x), isc) : czero<C>();
    }
  }
  C *const lines[2] = {smem + size_t(rr) * LP, smem + size_t(ROWS + rr) * LP};
  RegPlan<LX, V>::template run<C, 2, false, true>(v, lines, t, tr, RowSync<T>{1 + rr});
  // transpose through shared memory: tile[c][kx][rr], then ROWS consecutive z per kx
  __syncthreads();
  constexpr int RP = ROWS + 1;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) smem[(size_t(c) * LX + t + m * T) * RP + rr] = v[c][m];
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * LX * ROWS; idx += RC::NT) {
    const int r = idx % ROWS, ck = idx / ROWS;  // ck = c * LX + kx
    if (z0 + r < nz) a.T()[size_t(ck) * nz + z0 + r] = smem[size_t(ck) * RP + r];
  }
}

// For CC columns kx: forward FFT along z of the nz non-zero rows padded to LZ, 2x2 multiply by
// Ghat(kz, kx), inverse FFT along z, keep z < nz. Thread (col, t), t fastest: a warp reads a
// contiguous run of one column; the T threads of a column share a barrier.
template <typename C, int LZ, int V, typename A>
__device__ __forceinline__ void cols_tile(const A &a, int tile, C *smem) {
  using CF = ColCfg<C, LZ>;
  constexpr int CC = CF::CC, T = CF::T, LP = CF::LP;
  const int col = threadIdx.x / T, t = threadIdx.x - col * T;
  const int kx = tile * CC + col;
  const int nz = a.nz(), lx = a.lx();
  const bool live = kx < lx;
  const C *c0 = a.T() + size_t(kx) * nz, *c1 = a.T() + (size_t(lx) + kx) * nz;
  const TwReg<C, LZ, V> tr(t, a.tw());
  C v[2][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int z = t + m * T;
    const bool in = m < kHalf && live && z < nz;
    v[0][m] = in ? c0[z] : czero<C>();
    v[1][m] = in ? c1[z] : czero<C>();
  }
  C *const lines[2] = {smem + size_t(col) * LP, smem + size_t(CC + col) * LP};
  RegPlan<LZ, V>::template run<C, 2, false, true>(v, lines, t, tr, RowSync<T>{1 + col});
  if (live) {
    const size_t plane = size_t(lx) * LZ;
    const C *G = a.G() + size_t(kx) * LZ;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int kz = t + m * T;
      const C g11 = __ldg(G + kz), g13 = __ldg(G + plane + kz), g33 = __ldg(G + 2 * plane + kz);
      const C s1 = v[0][m], s3 = v[1][m];
      v[0][m] = cadd(cmul(g11, s1), cmul(g13, s3));
      v[1][m] = cadd(cmul(g13, s1), cmul(g33, s3));
    }
  }
  RegPlan<LZ, V>::template run<C, 2, true>(v, lines, t, tr, RowSync<T>{1 + col});
  if (live) {
    C *o0 = a.T() + size_t(kx) * nz, *o1 = a.T() + (size_t(lx) + kx) * nz;
#pragma unroll
    for (int m = 0; m < kHalf; ++m) {
      const int z = t + m * T;
      if (z < nz) {
        o0[z] = v[0][m];
        o1[z] = v[1][m];
      }
    }
  }
}

// Inverse FFT along x of ROWS rows, keep x < nx, out = ident - osc * result (or the scaled
// result when there is no identity term).
template <typename C, int LX, int EPI, int V, typename A>
__device__ __forceinline__ void rows_inverse_tile(const A &a, int tile, C *smem) {
  using Rl = typename RealOf<C>::type;
  using RC = RowCfg<C, LX>;
  constexpr int ROWS = RC::ROWS, T = RC::T, LP = RC::LP;
  const int z0 = tile * ROWS;
  const int nz = a.nz(), nx = a.nx();
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  const TwReg<C, LX, V> tr(t, a.tw());
  // ROWS consecutive z of every (c, kx) into tile[c][kx][r], then each thread takes its row
  constexpr int RP = ROWS + 1, NLD = 2 * LX * ROWS / RC::NT;
  static_assert((2 * LX * ROWS) % RC::NT == 0, "tile load");
  {
    C ld[NLD];
#pragma unroll
    for (int i = 0; i < NLD; ++i) {  // all loads in flight before the shared-memory stores
      const int idx = threadIdx.x + i * RC::NT, r = idx % ROWS, ck = idx / ROWS;
      ld[i] = z0 + r < nz ? a.T()[size_t(ck) * nz + z0 + r] : czero<C>();
    }
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int idx = threadIdx.x + i * RC::NT, r = idx % ROWS, ck = idx / ROWS;
      smem[size_t(ck) * RP + r] = ld[i];
    }
  }
  __syncthreads();
  C v[2][8];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) v[c][m] = smem[(size_t(c) * LX + t + m * T) * RP + rr];
  __syncthreads();  // the FFT lines reuse the tile
  C *const lines[2] = {smem + size_t(rr) * LP, smem + size_t(ROWS + rr) * LP};
  RegPlan<LX, V>::template run<C, 2, true>(v, lines, t, tr, RowSync<T>{1 + rr});
  const Rl osc = a.osc();
  const size_t base = size_t(z) * nx;
  // per-thread partials of the fused inner products: FP32 for complex64, FP64 for complex128
  using PA = typename RealOf<C>::type;
  PA a0 = 0, a1 = 0, a2 = 0;
  if (z < nz) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // every load of the component first (ident and rhat are read-only here), then the stores
      C id[kHalf], h[kHalf];
#pragma unroll
      for (int m = 0; m < kHalf; ++m) {
        const int x = t + m * T;
        const size_t o = base + size_t(c) * nz * nx + x;
        id[m] = (a.ident() && x < nx) ? __ldg(a.ident() + o) : czero<C>();
        if constexpr (EPI == 1) h[m] = x < nx ? __ldg(a.krhat() + o) : czero<C>();
      }
#pragma unroll
      for (int m = 0; m < kHalf; ++m) {
        const int x = t + m * T;
        if (x < nx) {
          const size_t o = base + size_t(c) * nz * nx + x;
          const C r = cscale(v[c][m], osc);
          const C w = a.ident() ? csub(id[m], r) : r;
          a.out()[o] = w;
          if constexpr (EPI == 1) {  // conj(rhat) w
            a0 += h[m].x * w.x + h[m].y * w.y;
            a1 += h[m].x * w.y - h[m].y * w.x;
          } else if constexpr (EPI == 2) {  // conj(w) id and |w|^2
            a0 += w.x * id[m].x + w.y * id[m].y;
            a1 += w.x * id[m].y - w.y * id[m].x;
            a2 += w.x * w.x + w.y * w.y;
          }
        }
      }
    }
  }
  if constexpr (EPI == 1) {
    PA acc[2] = {a0, a1};
    block_sum_store<2>(acc, a.part() + size_t(tile) * kRedSlots);
  } else if constexpr (EPI == 2) {
    PA acc[3] = {a0, a1, a2};
    block_sum_store<3>(acc, a.part() + size_t(tile) * kRedSlots);
  }
}

// Calls f.template operator()<L>() for the run-time FFT length L (a power of two in [16, 1024]).
template <typename F> __host__ __device__ __forceinline__ void with_len(int L, F &&f) {
  switch (L) {
    case 16: f.template operator()<16>(); break;
    case 32: f.template operator()<32>(); break;
    case 64: f.template operator()<64>(); break;
    case 128: f.template operator()<128>(); break;
    case 256: f.template operator()<256>(); break;
    case 512: f.template operator()<512>(); break;
    case 1024: f.template operator()<1024>(); break;
    default: break;
  }
}

}  // namespace dbi

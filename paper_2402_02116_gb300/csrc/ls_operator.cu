// The batched LS operator A u = u - h^2 G * (w^2 drho u + div(dC : eps(u))) (Eq. 6, 10) and the
// plain Green's convolution, both evaluated by Eq. 12 on the zero-padded lz x lx grid as three
// kernels per batch:
//   k_rows_forward : contrast source by central differences (fields zero outside D) for a few rows,
//                    zero-pad each row to lx, forward FFT along x  -> T[b][c][kx][z]   (z < nz)
//                    (the stress of each cell is formed once, in shared memory; the spectra are
//                    transposed through shared memory so that T is column-major)
//   k_cols         : for a few kx columns, forward FFT along z of the nz non-zero rows padded to
//                    lz, 2x2 multiply by Ghat(kz, kx), inverse FFT along z, keep z < nz -> T
//                    (contiguous column reads and writes, one named barrier per column)
//   k_rows_inverse : transpose rows back, inverse FFT along x, keep x < nx,
//                    out = ident - result (or the result).
// Ghat already carries h^2 / (lz lx), so no other scaling is applied.
#include <algorithm>

#include "fft_reg.cuh"
#include "operator.cuh"
#include "reduce.cuh"

namespace dbi {

template <typename C> struct OpP {
  using Rl = typename RealOf<C>::type;
  int nz, nx, lz, lx, nf;
  Rl inv2h;
  const double *omega;
  const int *fidx;
  const Rl *m;
  Rl ref[5];
  const C *in;
  const C *ident;
  C *out;
  C *T;
  const C *Ghat;
  const C *tw;
  const int *active;
  const int *plist;  // slot -> problem (NULL: problem = s0 + slot)
  int s0;            // first slot of this launch
  const double *in_scale, *m_scale, *out_scale;
  const C *krhat;
  double *part_out;
  int part_count;
};

// Launch shapes. Rows kernels: ROWS rows per CTA, T = L/8 threads per row (t fastest), both
// components of a row held by each thread. Column kernel: CC columns per CTA, thread (c, t) with c
// fastest so that a warp reads CC adjacent columns of a row.
template <typename C> struct Cfg;
#ifndef DBI_COLS_MIN_BLOCKS
#define DBI_COLS_MIN_BLOCKS 3
#endif
#ifndef DBI_ROWS_INV_MIN_BLOCKS
#define DBI_ROWS_INV_MIN_BLOCKS 4
#endif
template <> struct Cfg<float2> {
  static constexpr int rowThreads = 256, colThreads = 256;
  static constexpr int colMinBlocks = DBI_COLS_MIN_BLOCKS, rowInvMinBlocks = DBI_ROWS_INV_MIN_BLOCKS;
};
template <> struct Cfg<double2> {
  static constexpr int rowThreads = 256, colThreads = 256, colMinBlocks = 1, rowInvMinBlocks = 1;
};

template <typename C, int LX> struct RowCfg {
  static constexpr int T = LX / 8;
  static constexpr int ROWS = Cfg<C>::rowThreads / T > 0 ? Cfg<C>::rowThreads / T : 1;
  static constexpr int NT = ROWS * T;
  static constexpr int LP = RegFFT<C, LX>::LP;
};
template <typename C, int LZ> struct ColCfg {
  static constexpr int T = LZ / 8;
  static constexpr int CCr = Cfg<C>::colThreads / T;
  static constexpr int CC = CCr > 15 ? 15 : (CCr > 0 ? CCr : 1);  // named barriers 1..15
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

// Problem of this CTA's launch slot (blockIdx.y); the spectral scratch is indexed by the slot.
template <typename C> __device__ __forceinline__ int problem_of(const OpP<C> &p) {
  const int sl = p.s0 + int(blockIdx.y);
  return p.plist ? p.plist[sl] : sl;
}

// Barrier over the threads that share a line: the T threads of one row (rows kernels).
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
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Stress sigma = dC eps at cell (z, x) of D (zero outside D), from the staged u (rows z0 - 2 ..
// z0 + ROWS + 1 with a zero column on each side; u already multiplied by its input scale).
template <typename C>
__device__ __forceinline__ void stress_at(const OpP<C> &p, const C *su, int RS, int W, int z0, int z, int x,
                                          typename RealOf<C>::type ms, C &s1, C &s3, C &s5) {
  using Rl = typename RealOf<C>::type;
  const int nz = p.nz, nx = p.nx;
  if (z < 0 || z >= nz || x < 0 || x >= nx) {
    s1 = s3 = s5 = czero<C>();
    return;
  }
  auto U = [&](int c, int zz, int xx) { return su[(c * RS + (zz - z0 + 2)) * W + xx + 1]; };
  const Rl f = p.inv2h;
  const C e1 = cscale(csub(U(0, z, x + 1), U(0, z, x - 1)), f);
  const C e3 = cscale(csub(U(1, z + 1, x), U(1, z - 1, x)), f);
  const C e5 = cscale(cadd(csub(U(0, z + 1, x), U(0, z - 1, x)), csub(U(1, z, x + 1), U(1, z, x - 1))), f);
  const size_t cell = size_t(z) * nx + x, plane = size_t(nz) * nx;
  const Rl d11 = (__ldg(p.m + 1 * plane + cell) - p.ref[1]) * ms;
  const Rl d13 = (__ldg(p.m + 2 * plane + cell) - p.ref[2]) * ms;
  const Rl d33 = (__ldg(p.m + 3 * plane + cell) - p.ref[3]) * ms;
  const Rl d55 = (__ldg(p.m + 4 * plane + cell) - p.ref[4]) * ms;
  s1 = cadd(cscale(e1, d11), cscale(e3, d13));
  s3 = cadd(cscale(e1, d13), cscale(e3, d33));
  s5 = cscale(e5, d55);
}

// Contrast source (or the raw source) of ROWS rows, zero-padded to LX, forward FFT along x.
//   stencil: stress of rows z0-1 .. z0+ROWS (each computed once, kept in shared memory), then
//            s1 = w^2 drho u1 + d1 sigma1 + d3 sigma5, s3 = w^2 drho u3 + d1 sigma5 + d3 sigma3.
template <typename C, int LX, bool STENCIL>
__global__ void __launch_bounds__(RowCfg<C, LX>::NT) k_rows_forward(OpP<C> p) {
  using Rl = typename RealOf<C>::type;
  using RC = RowCfg<C, LX>;
  constexpr int ROWS = RC::ROWS, T = RC::T, LP = RC::LP;
  const int b = problem_of(p), slot = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(p.fidx[b]) >= unsigned(p.nf)) return;
  const int z0 = blockIdx.x * ROWS;
  const int nz = p.nz, nx = p.nx;
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  const size_t plane = size_t(nz) * nx;
  const C *u1 = p.in + size_t(b) * 2 * plane, *u3 = u1 + plane;
  const Rl isc = p.in_scale ? Rl(p.in_scale[b]) : Rl(1);
  const TwReg<C, LX> tr(t, p.tw);
  C v[2][8];

  if constexpr (STENCIL) {
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
      C a[KW], c3[KW];
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int xx = int(threadIdx.x) - 1 + k * RC::NT;
        const bool in = row && xx >= 0 && xx < nx;
        a[k] = in ? cscale(__ldg(u1 + size_t(zz) * nx + xx), isc) : czero<C>();
        c3[k] = in ? cscale(__ldg(u3 + size_t(zz) * nx + xx), isc) : czero<C>();
      }
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int xx = int(threadIdx.x) - 1 + k * RC::NT;
        if (xx <= nx) {
          su[(0 * RS + r) * W + xx + 1] = a[k];
          su[(1 * RS + r) * W + xx + 1] = c3[k];
        }
      }
    }
    __syncthreads();
    const Rl ms = p.m_scale ? Rl(p.m_scale[0]) : Rl(1);
#pragma unroll UR
    for (int r2 = 0; r2 < ROWS + 2; ++r2) {
      const int zz = z0 - 1 + r2;
#pragma unroll
      for (int k = 0; k < KW; ++k) {
        const int xx = int(threadIdx.x) - 1 + k * RC::NT;
        if (xx <= nx) {
          C a1, a3, a5;
          stress_at(p, su, RS, W, z0, zz, xx, ms, a1, a3, a5);
          sg[(0 * (ROWS + 2) + r2) * W + xx + 1] = a1;
          sg[(1 * (ROWS + 2) + r2) * W + xx + 1] = a3;
          sg[(2 * (ROWS + 2) + r2) * W + xx + 1] = a5;
        }
      }
    }
    __syncthreads();
    const Rl w2 = Rl(p.omega[p.fidx[b]] * p.omega[p.fidx[b]]);
    auto S = [&](int c, int r2, int xx) { return sg[(c * (ROWS + 2) + r2) * W + xx + 1]; };
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x = t + m * T;
      C o1 = czero<C>(), o3 = czero<C>();
      if (m < kHalf && z < nz && x < nx) {
        const int r2 = rr + 1;
        o1 = cadd(csub(S(0, r2, x + 1), S(0, r2, x - 1)), csub(S(2, r2 + 1, x), S(2, r2 - 1, x)));
        o3 = cadd(csub(S(2, r2, x + 1), S(2, r2, x - 1)), csub(S(1, r2 + 1, x), S(1, r2 - 1, x)));
        o1 = cscale(o1, p.inv2h);
        o3 = cscale(o3, p.inv2h);
        const size_t cell = size_t(z) * nx + x;
        const Rl wr = w2 * (__ldg(p.m + cell) - p.ref[0]) * ms;
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
  RegPlan<LX>::template run<C, 2, false, true>(v, lines, t, tr, RowSync<T>{1 + rr});
  // transpose through shared memory: tile[c][kx][rr], then ROWS consecutive z per kx
  __syncthreads();
  constexpr int RP = ROWS + 1;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) smem[(size_t(c) * LX + t + m * T) * RP + rr] = v[c][m];
  __syncthreads();
  C *Tb = p.T + size_t(slot) * 2 * LX * nz;
  for (int idx = threadIdx.x; idx < 2 * LX * ROWS; idx += RC::NT) {
    const int r = idx % ROWS, ck = idx / ROWS;  // ck = c * LX + kx
    if (z0 + r < nz) Tb[size_t(ck) * nz + z0 + r] = smem[size_t(ck) * RP + r];
  }
}

// For CC columns kx: forward FFT along z of the nz non-zero rows padded to LZ, 2x2 multiply by
// Ghat(kz, kx), inverse FFT along z, keep z < nz. Thread (col, t), t fastest: a warp reads a
// contiguous run of one column; the T threads of a column share a named barrier.
template <typename C, int LZ>
__global__ void __launch_bounds__(ColCfg<C, LZ>::NT, Cfg<C>::colMinBlocks) k_cols(OpP<C> p) {
  using CF = ColCfg<C, LZ>;
  constexpr int CC = CF::CC, T = CF::T, LP = CF::LP;
  const int b = problem_of(p), slot = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(p.fidx[b]) >= unsigned(p.nf)) return;
  const int col = threadIdx.x / T, t = threadIdx.x - col * T;
  const int kx = blockIdx.x * CC + col;
  const int nz = p.nz, lx = p.lx;
  const bool live = kx < lx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  C *Tb = p.T + size_t(slot) * 2 * lx * nz;
  const C *c0 = Tb + size_t(kx) * nz, *c1 = Tb + (size_t(lx) + kx) * nz;
  const TwReg<C, LZ> tr(t, p.tw);
  C v[2][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int z = t + m * T;
    const bool in = m < kHalf && live && z < nz;
    v[0][m] = in ? c0[z] : czero<C>();
    v[1][m] = in ? c1[z] : czero<C>();
  }
  C *const lines[2] = {smem + size_t(col) * LP, smem + size_t(CC + col) * LP};
  RegPlan<LZ>::template run<C, 2, false, true>(v, lines, t, tr, RowSync<T>{1 + col});
  if (live) {
    const size_t plane = size_t(lx) * LZ;
    const C *G = p.Ghat + size_t(p.fidx[b]) * 3 * plane + size_t(kx) * LZ;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int kz = t + m * T;
      const C g11 = __ldg(G + kz), g13 = __ldg(G + plane + kz), g33 = __ldg(G + 2 * plane + kz);
      const C s1 = v[0][m], s3 = v[1][m];
      v[0][m] = cadd(cmul(g11, s1), cmul(g13, s3));
      v[1][m] = cadd(cmul(g13, s1), cmul(g33, s3));
    }
  }
  RegPlan<LZ>::template run<C, 2, true>(v, lines, t, tr, RowSync<T>{1 + col});
  if (live) {
    C *o0 = Tb + size_t(kx) * nz, *o1 = Tb + (size_t(lx) + kx) * nz;
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

// Inverse FFT along x of ROWS rows, keep x < nx, out = ident - out_scale * result (or the scaled
// result when there is no identity term).
template <typename C, int LX, int EPI>
__global__ void __launch_bounds__(RowCfg<C, LX>::NT, Cfg<C>::rowInvMinBlocks) k_rows_inverse(OpP<C> p) {
  using Rl = typename RealOf<C>::type;
  using RC = RowCfg<C, LX>;
  constexpr int ROWS = RC::ROWS, T = RC::T, LP = RC::LP;
  const int b = problem_of(p), slot = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(p.fidx[b]) >= unsigned(p.nf)) return;
  const int z0 = blockIdx.x * ROWS;
  const int nz = p.nz, nx = p.nx;
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  const C *Tb = p.T + size_t(slot) * 2 * LX * nz;
  const TwReg<C, LX> tr(t, p.tw);
  // ROWS consecutive z of every (c, kx) into tile[c][kx][r], then each thread takes its row
  constexpr int RP = ROWS + 1, NLD = 2 * LX * ROWS / RC::NT;
  static_assert((2 * LX * ROWS) % RC::NT == 0, "tile load");
  {
    C ld[NLD];
#pragma unroll
    for (int i = 0; i < NLD; ++i) {  // all loads in flight before the shared-memory stores
      const int idx = threadIdx.x + i * RC::NT, r = idx % ROWS, ck = idx / ROWS;
      ld[i] = z0 + r < nz ? Tb[size_t(ck) * nz + z0 + r] : czero<C>();
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
  RegPlan<LX>::template run<C, 2, true>(v, lines, t, tr, RowSync<T>{1 + rr});
  const Rl osc = p.out_scale ? Rl(p.out_scale[b]) : Rl(1);
  const size_t base = size_t(b) * 2 * nz * nx + size_t(z) * nx;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;  // per-thread partials of the fused inner products
  if (z < nz) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      // every load of the component first (ident and rhat are read-only here), then the stores
      C id[kHalf], h[kHalf];
#pragma unroll
      for (int m = 0; m < kHalf; ++m) {
        const int x = t + m * T;
        const size_t o = base + size_t(c) * nz * nx + x;
        id[m] = (p.ident && x < nx) ? __ldg(p.ident + o) : czero<C>();
        if constexpr (EPI == 1) h[m] = x < nx ? __ldg(p.krhat + o) : czero<C>();
      }
#pragma unroll
      for (int m = 0; m < kHalf; ++m) {
        const int x = t + m * T;
        if (x < nx) {
          const size_t o = base + size_t(c) * nz * nx + x;
          const C r = cscale(v[c][m], osc);
          const C w = p.ident ? csub(id[m], r) : r;
          p.out[o] = w;
          if constexpr (EPI == 1) {  // conj(rhat) w
            a0 += float(h[m].x) * float(w.x) + float(h[m].y) * float(w.y);
            a1 += float(h[m].x) * float(w.y) - float(h[m].y) * float(w.x);
          } else if constexpr (EPI == 2) {  // conj(w) id and |w|^2
            a0 += float(w.x) * float(id[m].x) + float(w.y) * float(id[m].y);
            a1 += float(w.x) * float(id[m].y) - float(w.y) * float(id[m].x);
            a2 += float(w.x) * float(w.x) + float(w.y) * float(w.y);
          }
        }
      }
    }
  }
  if constexpr (EPI == 1) {
    double acc[2] = {double(a0), double(a1)};
    block_sum_store<2>(acc, p.part_out + (size_t(b) * p.part_count + blockIdx.x) * kRedSlots);
  } else if constexpr (EPI == 2) {
    double acc[3] = {double(a0), double(a1), double(a2)};
    block_sum_store<3>(acc, p.part_out + (size_t(b) * p.part_count + blockIdx.x) * kRedSlots);
  }
}


// The three kernels for launch slots [s0, s0 + nb) (problems plist[slot], or the slots themselves),
// each slot using its own part of the spectral scratch.
template <typename C> static int run_chunk(const OpArgs &a, int s0, int nb, cudaStream_t s) {
  using Rl = typename RealOf<C>::type;
  OpP<C> p;
  p.nz = a.nz; p.nx = a.nx; p.lz = a.lz; p.lx = a.lx; p.nf = a.nf;
  p.inv2h = Rl(1.0 / (2.0 * a.h));
  p.omega = a.omega; p.fidx = a.fidx;
  p.m = static_cast<const Rl *>(a.m);
  for (int i = 0; i < 5; ++i) p.ref[i] = Rl(a.ref[i]);
  p.in = static_cast<const C *>(a.in);
  p.ident = static_cast<const C *>(a.ident);
  p.out = static_cast<C *>(a.out);
  p.T = static_cast<C *>(a.T);
  p.Ghat = static_cast<const C *>(a.Ghat);
  p.tw = static_cast<const C *>(a.tw);
  p.active = a.active;
  p.plist = a.plist;
  p.s0 = s0;
  p.in_scale = a.in_scale;
  p.m_scale = a.m_scale;
  p.out_scale = a.out_scale;
  p.part_count = operator_parts(a.nz, a.lx, a.precision);
  p.krhat = static_cast<const C *>(a.krhat);
  p.part_out = a.part_out;
  int rc = DBI_OK;
  const bool stencil = a.stencil;
  prof_mark(PROF_ROWS_FORWARD, false, s);
  dispatch_len(a.lx, [&]<int LX>() {
    using RC = RowCfg<C, LX>;
    const size_t lines = size_t(2) * RC::ROWS * RC::LP * sizeof(C);
    const size_t tile = tile_elems<C, LX>() * sizeof(C);
    const size_t sg = stencil ? (size_t(3) * (RC::ROWS + 2) + size_t(2) * (RC::ROWS + 4)) * (a.nx + 2) * sizeof(C) : 0;
    const size_t bytes = std::max(std::max(lines, tile), sg);
    dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, nb);
    cudaError_t e;
    auto launch = [&](auto kernel) {
      e = allow_smem(kernel, bytes);
      if (e == cudaSuccess) kernel<<<grid, RC::NT, bytes, s>>>(p);
    };
    if (stencil) launch(k_rows_forward<C, LX, true>);
    else launch(k_rows_forward<C, LX, false>);
    rc = e != cudaSuccess ? cuda_fail("k_rows_forward smem", e) : check_launch("k_rows_forward");
  });
  prof_mark(PROF_ROWS_FORWARD, true, s);
  if (rc) return rc;
  prof_mark(PROF_COLS, false, s);
  dispatch_len(a.lz, [&]<int LZ>() {
    using CF = ColCfg<C, LZ>;
    const size_t bytes = size_t(2) * CF::CC * CF::LP * sizeof(C);
    dim3 grid((a.lx + CF::CC - 1) / CF::CC, nb);
    cudaError_t e = allow_smem(k_cols<C, LZ>, bytes);
    if (e == cudaSuccess) k_cols<C, LZ><<<grid, CF::NT, bytes, s>>>(p);
    rc = e != cudaSuccess ? cuda_fail("k_cols smem", e) : check_launch("k_cols");
  });
  prof_mark(PROF_COLS, true, s);
  if (rc) return rc;
  prof_mark(PROF_ROWS_INVERSE, false, s);
  dispatch_len(a.lx, [&]<int LX>() {
    using RC = RowCfg<C, LX>;
    const size_t bytes = std::max(size_t(2) * RC::ROWS * RC::LP, tile_elems<C, LX>()) * sizeof(C);
    dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, nb);
    cudaError_t e;
    auto launch = [&](auto kernel) {
      e = allow_smem(kernel, bytes);
      if (e == cudaSuccess) kernel<<<grid, RC::NT, bytes, s>>>(p);
    };
    if (a.epi == 1) launch(k_rows_inverse<C, LX, 1>);
    else if (a.epi == 2) launch(k_rows_inverse<C, LX, 2>);
    else launch(k_rows_inverse<C, LX, 0>);
    rc = e != cudaSuccess ? cuda_fail("k_rows_inverse smem", e) : check_launch("k_rows_inverse");
  });
  prof_mark(PROF_ROWS_INVERSE, true, s);
  return rc;
}

template <typename C> static int run_typed(const OpArgs &a, cudaStream_t s) {
  const int nb = a.plist ? a.nb : a.B;
  if (nb <= 0) return DBI_OK;
  dbi_grid g{a.nz, a.nx, a.lz, a.lx, a.h};
  const int chunk = spectral_chunk(&g, a.B, a.precision);
  int rc = DBI_OK;
  prof_mark(PROF_OPERATOR, false, s);
  for (int s0 = 0; s0 < nb && rc == DBI_OK; s0 += chunk)
    rc = run_chunk<C>(a, s0, std::min(chunk, nb - s0), s);
  prof_mark(PROF_OPERATOR, true, s);
  return rc;
}

int operator_parts(int nz, int lx, int precision) {
  int rows = 1;
  auto pick = [&](auto tag) {
    using C = decltype(tag);
    dispatch_len(lx, [&]<int LX>() { rows = RowCfg<C, LX>::ROWS; });
  };
  if (precision == DBI_C64) pick(float2{});
  else pick(double2{});
  return (nz + rows - 1) / rows;
}

int run_operator(const OpArgs &a, cudaStream_t s) {
  return a.precision == DBI_C64 ? run_typed<float2>(a, s) : run_typed<double2>(a, s);
}

}  // namespace dbi

using namespace dbi;

// Common validation of the operator entry points.
static int check_op(const dbi_grid *g, const dbi_batch *batch, const void *Ghat, const void *in,
                    const void *out, int precision, void *work, size_t work_bytes, int op) {
  int rc;
  if ((rc = check_grid(g)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (batch->B > 0 && (!Ghat || !in || !out)) { set_error("NULL Ghat, input or output"); return DBI_ERR_ARG; }
  if (in == out && batch->B > 0) { set_error("input and output must be distinct buffers"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes(g, batch->B, precision, op);
  if (batch->B > 0 && (!work || work_bytes < need)) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  return DBI_OK;
}

extern "C" int green_convolve(const dbi_grid *g, const dbi_batch *batch, const void *Ghat,
                              const void *src, void *out, int precision, void *work,
                              size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_op(g, batch, Ghat, src, out, precision, work, work_bytes, DBI_OP_CONVOLVE);
  if (rc || batch->B == 0) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral(g, batch->B, precision));
  Scales sc = carve_scales(ar, batch->B);
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  if ((rc = pow2_scales(src, precision, false, batch->B, size_t(2) * g->nz * g->nx, sc.part, sc.scale, sc.inv,
                        nullptr, s)))
    return rc;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.stencil = false; a.in = src; a.ident = nullptr; a.out = out; a.T = T; a.Ghat = Ghat; a.tw = tw;
  a.in_scale = sc.scale; a.out_scale = sc.inv;
  return run_operator(a, s);
}

extern "C" int ls_apply(const dbi_model *model, const dbi_batch *batch, const void *Ghat,
                        const void *u, void *out, int precision, void *work, size_t work_bytes,
                        dbi_stream stream) {
  clear_error();
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  const dbi_grid *g = &model->grid;
  int rc = check_op(g, batch, Ghat, u, out, precision, work, work_bytes, DBI_OP_APPLY);
  if (rc || batch->B == 0) return rc;
  if (!model->m) { set_error("model->m is NULL"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral(g, batch->B, precision));
  Scales sc = carve_scales(ar, batch->B);
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  if ((rc = pow2_scales(u, precision, false, batch->B, size_t(2) * g->nz * g->nx, sc.part, sc.scale, sc.inv,
                        nullptr, s)))
    return rc;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.m = model->m; reference_values(model->ref, a.ref);
  a.stencil = true; a.in = u; a.ident = u; a.out = out; a.T = T; a.Ghat = Ghat; a.tw = tw;
  a.in_scale = sc.scale; a.out_scale = sc.inv;
  return run_operator(a, s);
}

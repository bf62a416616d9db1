// LS-operator stages for an FFT length L = 2M = 1024 (complex64), where every transform of the
// operator is half-pruned: the forward row and column transforms read nz <= M (nx <= M) non-zero
// points, and the inverse ones are needed at the first M points only (lz >= 2 nz - 1).
//
// A half-pruned length-L transform is two length-M transforms. Forward, with x_j = 0 for j >= M:
//   X[2m + q] = sum_{j<M} (x_j W_L^{jq}) W_M^{jm},      q = 0, 1,
// i.e. the M-point DFTs of x and of x_j W_L^j give the even and the odd outputs. Inverse, for the
// first M outputs:
//   y_j = sum_m Y[2m] W_M^{-jm} + W_L^{-j} sum_m Y[2m + 1] W_M^{-jm},   j < M.
// The register FFT of length M = 512 (three radix-8 passes, two shared-memory exchanges) replaces
// the length-1024 one (four passes, three exchanges, half of the first or last pass idle), which
// cuts the exchanges by a third; with 64 threads per line a 256-thread CTA takes four rows, so
// the row stages read and write the column-major spectra in 32-byte runs (one sector).
//
// The contrast source is formed by its own kernel (source_rows) into a scratch field, so that the
// row transform needs no halo rows and few registers.
#pragma once

#include "op_tiles.cuh"

namespace dbi {

constexpr int kSplitL = 1024, kSplitM = 512;
constexpr int kSplitT = kSplitM / 8;                  // threads per line (64)
constexpr int kSplitRows = kTileThreads / kSplitT;    // rows (or columns) per 256-thread tile (4)
constexpr int kSplitLP = RegFFT<float2, kSplitM>::LP; // padded line in shared memory
static_assert(kSplitL == 1024, "the per-point twiddles come from the contiguous W_1024 table");

// Transposition tile of the row stages, one component at a time: [rows][KP]. A thread's pair of
// points (2k, 2k + 1) is one 16-byte access (a quarter warp covers 128 contiguous bytes); the
// column-major 8-byte reads and writes of four rows at a time are served half a warp at a time,
// and with KP = 4 mod 16 the four rows x four kx of a half warp hit 16 distinct 8-byte bank slots.
constexpr int kSplitKP = kSplitL + 4;

// Shared memory (bytes) of the split stages: the lines of one parity (two per row or column) and,
// for the row stages, the transposition tile of one component.
// The row stages run the two parities one after the other through two lines per row (one per
// component); the column stage runs all four lines of a column at once (the twiddle powers formed
// once, half the barriers: measured faster there and slower in the row stages).
__host__ __device__ constexpr size_t split_lines_smem() { return size_t(2) * kSplitRows * kSplitLP * sizeof(float2); }
__host__ __device__ constexpr size_t split_cols_lines_smem() {
  return size_t(4) * kSplitRows * kSplitLP * sizeof(float2);
}
__host__ __device__ constexpr size_t split_tile_smem() { return size_t(kSplitRows) * kSplitKP * sizeof(float2); }
__host__ __device__ constexpr size_t split_rows_smem() {
  return split_lines_smem() > split_tile_smem() ? split_lines_smem() : split_tile_smem();
}
__host__ __device__ constexpr size_t split_cols_smem() { return split_cols_lines_smem(); }
// The inverse row stage stages the tiles of both components at once: [2][rows][KP].
__host__ __device__ constexpr size_t split_rows_inverse_smem() {
  return split_lines_smem() > 2 * split_tile_smem() ? split_lines_smem() : 2 * split_tile_smem();
}

// Contrast source of the stencil kernel: one thread per column (nx <= M = 512 columns, the zero
// columns x = -1 and x = nx on either side), a chunk of kSrcRows rows per CTA walked downwards.
constexpr int kSrcThreads = kSplitM, kSrcRows = 32, kSrcW = kSrcThreads + 2;
inline size_t source_smem() { return size_t(8) * kSrcW * sizeof(float2); }

// s = w^2 drho u + div(dC : eps(u)) (Eq. 6) on rows [zb, zb + kSrcRows) of one problem, written to
// S [2][nz][nx]. Step j: the stress sigma = dC eps(u) of row j is formed from u one row up and down
// (registers) and u one column left and right (shared memory, stored by the step before), and the
// source of row j - 1 from sigma5, sigma3 of rows j and j - 2 (registers) and sigma1, sigma5 of row
// j - 1 one column left and right (shared memory, stored by the step before); then u of row j + 1
// and sigma of row j are stored for the next step. The reads and writes of a step touch different
// parity slots, so one barrier per row suffices. The global loads of a step are issued one step
// ahead (u two rows down, the stiffness one row down, the density of the current row) so that
// their latency overlaps a step's work. Every thread takes part in every barrier.
template <typename A>
__device__ __forceinline__ void source_rows(const A &a, int chunk, float2 *smem, float2 *S) {
  using C = float2;
  const int nz = a.nz(), nx = a.nx(), x = threadIdx.x, zb = chunk * kSrcRows;
  const int ze = min(zb + kSrcRows, nz);
  const size_t plane = size_t(nz) * nx;
  const bool col = x < nx;
  const int xc = col ? x : 0;
  const float isc = a.isc(), ms = a.ms(), f = a.inv2h(), w2 = a.w2();
  const float r0 = a.ref(0), r1 = a.ref(1), r2 = a.ref(2), r3 = a.ref(3), r4 = a.ref(4);
  // this thread's column (row 0) of every field; row z lies z * nx further
  const C *u1p = a.in() + xc, *u3p = u1p + plane;
  const float *m0 = a.m() + xc;
  C *o1p = S + xc, *o3p = o1p + plane;
  // shared rows (index x + 1; entries 0 and nx + 1 .. stay zero): u1, u3 and sigma1, sigma5, two
  // slots each by row parity
  C *su = smem, *sg = smem + 4 * kSrcW;
  auto U = [&](int slot, int c) { return su + (slot * 2 + c) * kSrcW + 1; };
  auto G = [&](int slot, int c) { return sg + (slot * 2 + c) * kSrcW + 1; };
  for (int i = threadIdx.x; i < 8 * kSrcW; i += kSrcThreads) smem[i] = czero<C>();
  auto in_d = [&](int z) { return col && unsigned(z) < unsigned(nz); };
  auto load_u = [&](int z, C &v1, C &v3) {
    const bool in = in_d(z);
    const int o = in ? z * nx : 0;
    v1 = in ? __ldg(u1p + o) : czero<C>();
    v3 = in ? __ldg(u3p + o) : czero<C>();
  };
  struct Stiff {
    float d11, d13, d33, d55;
  };
  auto load_stiff = [&](int z, Stiff &d) {
    const bool in = in_d(z);
    const float *mz = m0 + (in ? z * nx : 0);
    d.d11 = in ? __ldg(mz + 1 * plane) : r1;
    d.d13 = in ? __ldg(mz + 2 * plane) : r2;
    d.d33 = in ? __ldg(mz + 3 * plane) : r3;
    d.d55 = in ? __ldg(mz + 4 * plane) : r4;
  };
  auto load_rho = [&](int z) { return in_d(z) ? __ldg(m0 + z * nx) : r0; };
  // window: u at rows j - 1, j (scaled); sigma3, sigma5 at rows j - 2, j - 1
  C ua1, ua3, ub1, ub3;
  C s3a = czero<C>(), s5a = czero<C>(), s3b = czero<C>(), s5b = czero<C>();
  const int j0 = zb - 1;  // odd: zb is a multiple of kSrcRows (even), so step parities are static
  load_u(j0 - 1, ua1, ua3);
  load_u(j0, ub1, ub3);
  ua1 = cscale(ua1, isc); ua3 = cscale(ua3, isc);
  ub1 = cscale(ub1, isc); ub3 = cscale(ub3, isc);
  C nu1, nu3;  // u(j + 1), loaded one step ahead
  Stiff nd;    // stiffness of row j
  float nrho;  // density of row j - 1
  load_u(j0 + 1, nu1, nu3);
  load_stiff(j0, nd);
  nrho = load_rho(j0 - 1);
  __syncthreads();  // the zero fill precedes every row store
  U(j0 & 1, 0)[x] = ub1;
  U(j0 & 1, 1)[x] = ub3;
  __syncthreads();
  auto step = [&]<int P>(int j) {  // P = j & 1
    const C uc1 = cscale(nu1, isc), uc3 = cscale(nu3, isc);
    const Stiff d = nd;
    const float rho = nrho;
    load_u(j + 2, nu1, nu3);  // the next step's loads
    load_stiff(j + 1, nd);
    nrho = load_rho(j);
    // sigma(j, x)
    C s1 = czero<C>(), s3 = czero<C>(), s5 = czero<C>();
    if (in_d(j)) {
      const C *r1u = U(P, 0), *r3u = U(P, 1);
      const C e1 = cscale(csub(r1u[x + 1], r1u[x - 1]), f);
      const C e3 = cscale(csub(uc3, ua3), f);
      const C e5 = cscale(cadd(csub(uc1, ua1), csub(r3u[x + 1], r3u[x - 1])), f);
      const float d11 = (d.d11 - r1) * ms, d13 = (d.d13 - r2) * ms, d33 = (d.d33 - r3) * ms, d55 = (d.d55 - r4) * ms;
      s1 = cadd(cscale(e1, d11), cscale(e3, d13));
      s3 = cadd(cscale(e1, d13), cscale(e3, d33));
      s5 = cscale(e5, d55);
    }
    // source at row j - 1
    const int z = j - 1;
    if (col && z >= zb && z < ze) {
      const C *g1 = G(P ^ 1, 0), *g5 = G(P ^ 1, 1);
      const C o1 = cscale(cadd(csub(g1[x + 1], g1[x - 1]), csub(s5, s5a)), f);
      const C o3 = cscale(cadd(csub(g5[x + 1], g5[x - 1]), csub(s3, s3a)), f);
      const int cell = z * nx;
      const float wr = w2 * (rho - r0) * ms;
      o1p[cell] = cadd(o1, cscale(ua1, wr));  // u(j - 1)
      o3p[cell] = cadd(o3, cscale(ua3, wr));
    }
    // u(j + 1) and sigma(j) for the next step (slots read by the step before)
    U(P ^ 1, 0)[x] = uc1;
    U(P ^ 1, 1)[x] = uc3;
    G(P, 0)[x] = s1;
    G(P, 1)[x] = s5;
    __syncthreads();
    ua1 = ub1; ua3 = ub3; ub1 = uc1; ub3 = uc3;
    s3a = s3b; s5a = s5b; s3b = s3; s5b = s5;
  };
  int j = j0;
  for (; j + 1 <= ze; j += 2) {
    step.template operator()<1>(j);
    step.template operator()<0>(j + 1);
  }
  if (j <= ze) step.template operator()<1>(j);
}

// The two parities of the two components, each an M-point transform held as 8 points per thread:
// v[q][c][m] is point t + m T of the line of component c and parity q.
struct SplitLines {
  float2 *l[2][2];
};

// M-point transforms of both parities, one parity at a time through the two lines of the
// components (the row stages).
template <bool INV, typename Sync>
__device__ __forceinline__ void split_fft(float2 (&v)[2][2][8], float2 *const (&lines)[2], int t,
                                          const TwReg<float2, kSplitM, 0> &tr, Sync &&sync) {
#pragma unroll
  for (int q = 0; q < 2; ++q) RegPlan<kSplitM, 0>::template run<float2, 2, INV>(v[q], lines, t, tr, sync);
}

// M-point transforms of both parities and both components at once, four lines through one
// exchange set (the column stage).
template <bool INV, typename Sync>
__device__ __forceinline__ void split_fft4(float2 (&v)[2][2][8], float2 *const (&lines)[4], int t,
                                           const TwReg<float2, kSplitM, 0> &tr, Sync &&sync) {
  RegPlan<kSplitM, 0>::template run<float2, 4, INV>(reinterpret_cast<float2(&)[4][8]>(v), lines, t, tr, sync);
}


// Shared memory of the column stage with the column's Green's tables staged: the lines, then
// Ghat(:, kx) of the three tables [3][L].
__host__ __device__ constexpr size_t split_cols_staged_smem() {
  return split_cols_lines_smem() + size_t(3) * kSplitL * sizeof(float2);
}

// Column kx of one problem, by the 64 threads of group g of the CTA (named barrier 1 + g): the
// forward transform along z (even and odd kz), the 2 x 2 multiply by Ghat(kz, kx), the inverse
// transform; the nz outputs written back in place. Ghat comes from Gs (the column's three tables
// staged in shared memory, [3][L]) or, when Gs is null, from global memory. STAGED: the CTA stages
// the tables with asynchronous copies; every thread of the CTA (live or not) waits for them at the
// barrier between the transforms. `live` is uniform over the group.
template <bool STAGED, typename A>
__device__ __forceinline__ void cols_column_split(const A &a, int kx, int g, bool live, float2 *smem,
                                                  const float4 *Gs) {
  using C = float2;
  constexpr int T = kSplitT, CC = kSplitRows;
  const int t = threadIdx.x - g * T;
  const int nz = a.nz(), lx = a.lx();
  const C *tw = a.tw();
  C *c0 = a.T() + size_t(kx) * nz, *c1 = a.T() + (size_t(lx) + kx) * nz;
  const TwReg<C, kSplitM, 0> tr(t, tw);
  C *lines[4];  // (parity q, component c) of column group g
#pragma unroll
  for (int l = 0; l < 4; ++l) lines[l] = smem + size_t(l * CC + g) * kSplitLP;
  C v[2][2][8];
  if (live) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int z = t + m * T;
      const bool in = z < nz;
      const C x0 = in ? c0[z] : czero<C>(), x1 = in ? c1[z] : czero<C>();
      const C w = __ldg(tw + kTw1024 + z);  // W_L^z
      v[0][0][m] = x0;
      v[0][1][m] = x1;
      v[1][0][m] = hmul(x0, w);
      v[1][1][m] = hmul(x1, w);
    }
    split_fft4<false>(v, lines, t, tr, RowSync<T>{1 + g});
  }
  if constexpr (STAGED) {
    cp_async_wait_all();
    __syncthreads();  // every thread's table copies have landed
  }
  if (!live) return;
  {
    const size_t plane = size_t(lx) * kSplitL;
    const float4 *G = reinterpret_cast<const float4 *>(a.G() + size_t(kx) * kSplitL);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * T;  // kz = 2k (even) and 2k + 1 (odd): one 16-byte load per table
      float4 g11, g13, g33;
      if (Gs) {
        g11 = Gs[k]; g13 = Gs[kSplitL / 2 + k]; g33 = Gs[kSplitL + k];
      } else {
        g11 = __ldg(G + k); g13 = __ldg(G + plane / 2 + k); g33 = __ldg(G + plane + k);
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const C a11 = q ? make_float2(g11.z, g11.w) : make_float2(g11.x, g11.y);
        const C a13 = q ? make_float2(g13.z, g13.w) : make_float2(g13.x, g13.y);
        const C a33 = q ? make_float2(g33.z, g33.w) : make_float2(g33.x, g33.y);
        const C s1 = v[q][0][m], s3 = v[q][1][m];
        v[q][0][m] = cadd(cmul(a11, s1), cmul(a13, s3));
        v[q][1][m] = cadd(cmul(a13, s1), cmul(a33, s3));
      }
    }
  }
  split_fft4<true>(v, lines, t, tr, RowSync<T>{1 + g});
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int z = t + m * T;
    if (z < nz) {
      const C w = cconj(__ldg(tw + kTw1024 + z));  // W_L^{-z}
      c0[z] = cadd(v[0][0][m], cmul(w, v[1][0][m]));
      c1[z] = cadd(v[0][1][m], cmul(w, v[1][1][m]));
    }
  }
}

// For CC = 4 columns kx = 4 tile .. 4 tile + 3 of one problem (the uneven-batch tiles).
template <typename A>
__device__ __forceinline__ void cols_tile_split(const A &a, int tile, float2 *smem) {
  const int g = threadIdx.x / kSplitT, kx = tile * kSplitRows + g;
  cols_column_split<false>(a, kx, g, kx < a.lx(), smem, nullptr);
}

// Four rows z0 .. z0 + 3: the source rows (from the stencil kernel, or the raw input times its
// scale), the forward transform along x (even and odd kx), transposed through shared memory into
// the column-major spectra T[c][kx][z] in runs of four rows.
template <typename A>
__device__ __forceinline__ void rows_forward_tile_split(const A &a, int tile, float2 *smem, const float2 *src,
                                                        float scale) {
  using C = float2;
  constexpr int T = kSplitT, ROWS = kSplitRows, KP = kSplitKP;
  const int z0 = tile * ROWS;
  const int nz = a.nz(), nx = a.nx();
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  const size_t plane = size_t(nz) * nx;
  const C *tw = a.tw();
  const TwReg<C, kSplitM, 0> tr(t, tw);
  C v[2][2][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int x = t + m * T;
    const bool in = z < nz && x < nx;
    const C s0 = in ? cscale(__ldg(src + size_t(z) * nx + x), scale) : czero<C>();
    const C s1 = in ? cscale(__ldg(src + plane + size_t(z) * nx + x), scale) : czero<C>();
    const C w = __ldg(tw + kTw1024 + x);  // W_L^x
    v[0][0][m] = s0;
    v[0][1][m] = s1;
    v[1][0][m] = hmul(s0, w);
    v[1][1][m] = hmul(s1, w);
  }
  C *const lines[2] = {smem + size_t(rr) * kSplitLP, smem + size_t(ROWS + rr) * kSplitLP};
  split_fft<false>(v, lines, t, tr, RowSync<T>{1 + rr});
  // transpose one component at a time through tile[rr][kx] (the lines' memory is free now)
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    __syncthreads();
    float4 *row = reinterpret_cast<float4 *>(smem + size_t(rr) * KP);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const C e = v[0][c][m], o = v[1][c][m];  // kx = 2k and 2k + 1
      row[t + m * T] = make_float4(e.x, e.y, o.x, o.y);
    }
    __syncthreads();
    C *Tc = a.T() + size_t(c) * a.lx() * nz;
    for (int idx = threadIdx.x; idx < kSplitL * ROWS; idx += kTileThreads) {
      const int r = idx % ROWS, kx = idx / ROWS;
      if (z0 + r < nz) Tc[size_t(kx) * nz + z0 + r] = smem[size_t(r) * KP + kx];
    }
  }
}

// Four rows: the spectra T[c][kx][z0 .. z0 + 3] through a transposition tile, the inverse
// transform along x (even and odd kx), y_x = even + W_L^{-x} odd for x < nx, then the epilogue of
// rows_inverse_tile: out = ident - scale * y (or the scaled y) with the fused inner products.
template <int EPI, typename A>
__device__ __forceinline__ void rows_inverse_tile_split(const A &a, int tile, float2 *smem) {
  using C = float2;
  constexpr int T = kSplitT, ROWS = kSplitRows, KP = kSplitKP;
  const int z0 = tile * ROWS;
  const int nz = a.nz(), nx = a.nx();
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  const C *tw = a.tw();
  const TwReg<C, kSplitM, 0> tr(t, tw);
  C v[2][2][8];
  // the spectra of both components into tile[c][r][kx] by asynchronous copies (zeros for rows
  // beyond nz), all in flight at once and without register staging
  constexpr int NLD = 2 * kSplitL * ROWS / kTileThreads;  // 32 copies per thread
  {
    const int r = threadIdx.x % ROWS;  // the same row for all of a thread's copies
    const bool in = z0 + r < nz;
    const C *T0 = a.T() + (in ? z0 + r : 0);
    const size_t cplane = size_t(a.lx()) * nz;
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int idx = threadIdx.x + i * kTileThreads, kx = (idx / ROWS) % kSplitL, c = idx / (ROWS * kSplitL);
      cp_async8(smem + size_t(c * ROWS + r) * KP + kx, T0 + c * cplane + size_t(kx) * nz, in);
    }
  }
  cp_async_wait_all();
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const float4 *row = reinterpret_cast<const float4 *>(smem + size_t(c * ROWS + rr) * KP);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 eo = row[t + m * T];  // kx = 2k and 2k + 1
      v[0][c][m] = make_float2(eo.x, eo.y);
      v[1][c][m] = make_float2(eo.z, eo.w);
    }
  }
  __syncthreads();  // the lines reuse the tile's memory
  C *const lines[2] = {smem + size_t(rr) * kSplitLP, smem + size_t(ROWS + rr) * kSplitLP};
  split_fft<true>(v, lines, t, tr, RowSync<T>{1 + rr});
  C y[2][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const C w = cconj(__ldg(tw + kTw1024 + t + m * T));  // W_L^{-x}
#pragma unroll
    for (int c = 0; c < 2; ++c) y[c][m] = cadd(v[0][c][m], cmul(w, v[1][c][m]));
  }
  const float osc = a.osc();
  const size_t base = size_t(z) * nx;
  float a0 = 0, a1 = 0, a2 = 0;
  if (z < nz) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      C id[8], h[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int x = t + m * T;
        const size_t o = base + size_t(c) * nz * nx + x;
        id[m] = (a.ident() && x < nx) ? __ldg(a.ident() + o) : czero<C>();
        if constexpr (EPI == 1) h[m] = x < nx ? __ldg(a.krhat() + o) : czero<C>();
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int x = t + m * T;
        if (x < nx) {
          const size_t o = base + size_t(c) * nz * nx + x;
          const C r = cscale(y[c][m], osc);
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
    float acc[2] = {a0, a1};
    block_sum_store<2>(acc, a.part() + size_t(tile) * kRedSlots);
  } else if constexpr (EPI == 2) {
    float acc[3] = {a0, a1, a2};
    block_sum_store<3>(acc, a.part() + size_t(tile) * kRedSlots);
  }
}

}  // namespace dbi

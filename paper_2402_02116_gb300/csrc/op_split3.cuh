// LS-operator stages for the FFT length L = 3M = 768 (complex64), for grids of up to 384 cells
// along the axis (L >= 2N - 1). Every transform of the operator is half-pruned (N <= L/2 = 1.5 M
// non-zero inputs, or the first N outputs only), and a length-3M transform is three M-point
// transforms. Forward, with x_j = 0 for j >= 1.5 M:
//   X[3m + q] = sum_{i<M} W_L^{iq} (x_i + W_3^q x_{i+M}) W_M^{im},   q = 0, 1, 2,
// (x_{i+M} is non-zero only for i < M/2). Inverse, for the first 1.5 M outputs:
//   y_j = sum_q W_L^{-jq} v_q[j mod M],   v_q = the unnormalised inverse M-point DFT of Y[3m + q].
// With M = 256 a line is one warp (32 threads x 8 points), so its exchanges need only warp
// barriers; each warp takes one residue q of one row or column, and the three residues of a row
// or column meet once, through shared memory. Compared with L = 1024 the FFT grid of a 384-cell
// axis shrinks by a quarter, and the transforms by more (three 256-point lines instead of two
// 512-point ones).
#pragma once

#include "op_split.cuh"

namespace dbi {

constexpr int kS3L = 768, kS3M = 256;
constexpr int kS3T = kS3M / 8;                    // threads per line: one warp
constexpr int kS3Units = 4;                       // rows or columns per CTA
constexpr int kS3Threads = kS3Units * 3 * kS3T;   // 384: a warp per (unit, residue)
constexpr int kS3LP = RegFFT<float2, kS3M>::LP;   // padded line in shared memory
// Transposition tile row of the row stages. 8-byte accesses are served half a warp at a time: with
// KP = 4 mod 16 the column-major accesses (four rows x four kx per half warp) hit 16 distinct
// 8-byte bank slots, and so do the residue-strided accesses 3k + q of a warp (3 is odd).
constexpr int kS3KP = kS3L + 4;
constexpr int kS3UnitThreads = 3 * kS3T;          // 96 threads per row or column
constexpr int kS3Tw = kTwiddleN / kS3L;           // W_L^j = tw[j * kS3Tw]
constexpr int kS3Third = kTwiddleN / 3;           // W_3 = tw[kS3Third]

// Shared memory (bytes): two lines per warp (one per component); the row stages' transposition
// tile [c][rr][KP] of both components reuses that memory, and so do the residues' inverse
// transforms that the combine step reads. Every stage takes the same amount.
__host__ __device__ constexpr size_t s3_lines_smem() { return size_t(kS3Units) * 3 * 2 * kS3LP * sizeof(float2); }
__host__ __device__ constexpr size_t s3_tile_smem() { return size_t(2) * kS3Units * kS3KP * sizeof(float2); }
__host__ __device__ constexpr size_t s3_smem() {
  return s3_lines_smem() > s3_tile_smem() ? s3_lines_smem() : s3_tile_smem();
}

// Warp barrier: a line's exchanges stay inside its warp.
struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// The folded, twiddled input of residue q of both components at the thread's points
// i = t + m T (m < 8): W_L^{iq} (x_c(i) + W_3^q x_c(i + M)), from a reader x(c, j) of the line's
// points (zero where j >= n). W_L^{iq} = W_L^{tq} W_24^{mq} (T = 32 = L / 24): one per-thread table
// load and a warp-uniform one per m, instead of a 32-byte-strided load per point.
template <typename Read>
__device__ __forceinline__ void s3_fold(float2 (&v)[2][8], int t, int q, int n, const float2 *tw, Read &&x) {
  using C = float2;
  const C w3 = __ldg(tw + q * kS3Third);                  // W_3^q
  const C wt = __ldg(tw + ((t * q) % kS3L) * kS3Tw);      // W_L^{tq}
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int i = t + m * kS3T;
    const C wm = cmul(wt, __ldg(tw + ((m * q) % 24) * (kTwiddleN / 24)));  // W_L^{iq}
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      C a = i < n ? x(c, i) : czero<C>();
      if (m < 4 && i + kS3M < n) a = cadd(a, cmul(w3, x(c, i + kS3M)));
      v[c][m] = cmul(a, wm);
    }
  }
}

// The residues' inverse transforms of one row or column (held by its three warps in natural
// order) combined: y_j = sum_q W_L^{-jq} v_q[j mod M] for the unit's points j = u + 96 i (i < 4).
// The warps first store v_q into their own lines; one CTA barrier later every thread reads the
// three residues of its points. Every thread of the CTA must call it.
__device__ __forceinline__ void s3_combine(const float2 (&v)[2][8], float2 *smem, int w, int t, const float2 *tw,
                                           float2 (&y)[2][4]) {
  using C = float2;
  C *own = smem + size_t(2 * w) * kS3LP;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    own[t + m * kS3T] = v[0][m];
    own[kS3LP + t + m * kS3T] = v[1][m];
  }
  __syncthreads();
  const int unit = w / 3, u = threadIdx.x - unit * kS3UnitThreads;
  const C *base = smem + size_t(6 * unit) * kS3LP;  // lines of warps 3 unit + q: [q][c][LP]
  // W_L^{-j} = W_L^{-u} W_8^{-i} and W_L^{-2j} = W_L^{-2u} W_4^{-i} for j = u + 96 i (96 = L / 8)
  const C wu1 = cconj(__ldg(tw + u * kS3Tw)), wu2 = cconj(__ldg(tw + 2 * u * kS3Tw));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = u + i * kS3UnitThreads, jm = j & (kS3M - 1);
    const C w1 = i ? cmulc(wu1, __ldg(tw + i * (kTwiddleN / 8))) : wu1;
    const C w2 = i ? cmulc(wu2, __ldg(tw + i * (kTwiddleN / 4))) : wu2;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const C v0 = base[c * kS3LP + jm], v1 = base[(2 + c) * kS3LP + jm], v2 = base[(4 + c) * kS3LP + jm];
      y[c][i] = cadd(v0, cadd(cmul(w1, v1), cmul(w2, v2)));
    }
  }
}

// Columns kx = 4 tile .. 4 tile + 3: warp (column, q) folds the column's nz points (both
// components), transforms them forward (the spectra at kz = 3k + q), multiplies by Ghat(kz, kx) and
// transforms back; the three residues are combined into the nz outputs, written back in place.
// Ghat at lz = 768 is stored residue-major (slot q M + k holds kz = 3k + q), so a warp reads its
// residue's entries contiguously.
template <typename A>
__device__ __forceinline__ void cols_tile_s3(const A &a, int tile, float2 *smem) {
  using C = float2;
  const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int cc = w / 3, q = w - 3 * cc;
  const int kx = tile * kS3Units + cc;
  const int nz = a.nz(), lx = a.lx();
  const bool live = kx < lx;
  const C *tw = a.tw();
  C *col[2] = {a.T() + size_t(kx) * nz, a.T() + (size_t(lx) + kx) * nz};
  const TwReg<C, kS3M, 0> tr(t, tw);
  const int n = live ? nz : 0;
  C v[2][8];
  s3_fold(v, t, q, n, tw, [&](int c, int j) { return col[c][j]; });
  C *const lines[2] = {smem + size_t(2 * w) * kS3LP, smem + size_t(2 * w + 1) * kS3LP};
  RegPlan<kS3M, 0>::template run<C, 2, false>(v, lines, t, tr, WarpSync{});
  if (live) {
    const size_t plane = size_t(lx) * kS3L;
    const C *G = a.G() + size_t(kx) * kS3L + q * kS3M;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * kS3T;
      const C g11 = __ldg(G + k), g13 = __ldg(G + plane + k), g33 = __ldg(G + 2 * plane + k);
      const C s1 = v[0][m], s3 = v[1][m];
      v[0][m] = cadd(cmul(g11, s1), cmul(g13, s3));
      v[1][m] = cadd(cmul(g13, s1), cmul(g33, s3));
    }
  }
  RegPlan<kS3M, 0>::template run<C, 2, true>(v, lines, t, tr, WarpSync{});
  C y[2][4];
  s3_combine(v, smem, w, t, tw, y);
  if (live) {
    const int u = threadIdx.x - cc * kS3UnitThreads;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int z = u + i * kS3UnitThreads;
      if (z < nz) {
        col[0][z] = y[0][i];
        col[1][z] = y[1][i];
      }
    }
  }
}

// Rows z0 .. z0 + 3: warp (row, q) folds the row (the source rows from the stencil kernel, or the
// raw input times its scale) and transforms it (the spectra at kx = 3k + q); both components go
// through the transposition tile into the column-major spectra T[c][kx][z] in runs of four rows.
template <typename A>
__device__ __forceinline__ void rows_forward_tile_s3(const A &a, int tile, float2 *smem, const float2 *src,
                                                     float scale) {
  using C = float2;
  const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int rr = w / 3, q = w - 3 * rr;
  const int z0 = tile * kS3Units, z = z0 + rr;
  const int nz = a.nz(), nx = a.nx();
  const size_t plane = size_t(nz) * nx;
  const C *tw = a.tw();
  const TwReg<C, kS3M, 0> tr(t, tw);
  const int n = z < nz ? nx : 0;
  const C *row = src + size_t(z < nz ? z : 0) * nx;
  C v[2][8];
  s3_fold(v, t, q, n, tw, [&](int c, int j) { return cscale(__ldg(row + c * plane + j), scale); });
  C *const lines[2] = {smem + size_t(2 * w) * kS3LP, smem + size_t(2 * w + 1) * kS3LP};
  RegPlan<kS3M, 0>::template run<C, 2, false>(v, lines, t, tr, WarpSync{});
  __syncthreads();  // every warp is done with its lines: the tile reuses their memory
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    C *trow = smem + size_t(c * kS3Units + rr) * kS3KP;
#pragma unroll
    for (int m = 0; m < 8; ++m) trow[3 * (t + m * kS3T) + q] = v[c][m];
  }
  __syncthreads();
  const size_t cplane = size_t(a.lx()) * nz;
  constexpr int NST = 2 * kS3L * kS3Units / kS3Threads;  // 16 stores per thread
  const int r = threadIdx.x % kS3Units;                  // the same row for all of a thread's stores
  if (z0 + r < nz) {
#pragma unroll
    for (int i = 0; i < NST; ++i) {
      const int idx = threadIdx.x + i * kS3Threads, kx = (idx / kS3Units) % kS3L, c = idx / (kS3Units * kS3L);
      a.T()[c * cplane + size_t(kx) * nz + z0 + r] = smem[size_t(c * kS3Units + r) * kS3KP + kx];
    }
  }
}

// Rows z0 .. z0 + 3: the spectra T[c][kx][z0 .. z0 + 3] of both components through the
// transposition tile, warp (row, q) the inverse transform of residue q, the residues combined
// into y_x for x < nx, then the epilogue of rows_inverse_tile: out = ident - scale * y (or the
// scaled y) with the fused inner products.
template <int EPI, typename A>
__device__ __forceinline__ void rows_inverse_tile_s3(const A &a, int tile, float2 *smem) {
  using C = float2;
  const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int rr = w / 3, q = w - 3 * rr;
  const int z0 = tile * kS3Units, z = z0 + rr;
  const int nz = a.nz(), nx = a.nx();
  const C *tw = a.tw();
  const TwReg<C, kS3M, 0> tr(t, tw);
  const size_t cplane = size_t(a.lx()) * nz;
  constexpr int NLD = 2 * kS3L * kS3Units / kS3Threads;  // 16 loads per thread
  const int r = threadIdx.x % kS3Units;
  {
    C ld[NLD];
#pragma unroll
    for (int i = 0; i < NLD; ++i) {  // all loads in flight before the shared-memory stores
      const int idx = threadIdx.x + i * kS3Threads, kx = (idx / kS3Units) % kS3L, c = idx / (kS3Units * kS3L);
      ld[i] = z0 + r < nz ? a.T()[c * cplane + size_t(kx) * nz + z0 + r] : czero<C>();
    }
#pragma unroll
    for (int i = 0; i < NLD; ++i) {
      const int idx = threadIdx.x + i * kS3Threads, kx = (idx / kS3Units) % kS3L, c = idx / (kS3Units * kS3L);
      smem[size_t(c * kS3Units + r) * kS3KP + kx] = ld[i];
    }
  }
  __syncthreads();
  C v[2][8];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const C *trow = smem + size_t(c * kS3Units + rr) * kS3KP;
#pragma unroll
    for (int m = 0; m < 8; ++m) v[c][m] = trow[3 * (t + m * kS3T) + q];
  }
  __syncthreads();  // the lines reuse the tile's memory
  C *const lines[2] = {smem + size_t(2 * w) * kS3LP, smem + size_t(2 * w + 1) * kS3LP};
  RegPlan<kS3M, 0>::template run<C, 2, true>(v, lines, t, tr, WarpSync{});
  C y[2][4];
  s3_combine(v, smem, w, t, tw, y);
  const int u = threadIdx.x - rr * kS3UnitThreads;
  const float osc = a.osc();
  const size_t base = size_t(z) * nx, fplane = size_t(nz) * nx;
  float a0 = 0, a1 = 0, a2 = 0;
  if (z < nz) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      C id[4], h[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int x = u + i * kS3UnitThreads;
        const size_t o = base + c * fplane + x;
        id[i] = (a.ident() && x < nx) ? __ldg(a.ident() + o) : czero<C>();
        if constexpr (EPI == 1) h[i] = x < nx ? __ldg(a.krhat() + o) : czero<C>();
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int x = u + i * kS3UnitThreads;
        if (x < nx) {
          const size_t o = base + c * fplane + x;
          const C rv = cscale(y[c][i], osc);
          const C wv = a.ident() ? csub(id[i], rv) : rv;
          a.out()[o] = wv;
          if constexpr (EPI == 1) {  // conj(rhat) w
            a0 += h[i].x * wv.x + h[i].y * wv.y;
            a1 += h[i].x * wv.y - h[i].y * wv.x;
          } else if constexpr (EPI == 2) {  // conj(w) id and |w|^2
            a0 += wv.x * id[i].x + wv.y * id[i].y;
            a1 += wv.x * id[i].y - wv.y * id[i].x;
            a2 += wv.x * wv.x + wv.y * wv.y;
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

// 3D LS operator (the paper's 3D extension: Eq. A-1 and its 3D VTI example), batched over
// (source, frequency) problems on one grid [nz][ny][nx] of cubic cells:
//   A u = u - h^3 G * (w^2 drho u + div(dC : eps(u))),   u = (u1, u2, u3), x3 the depth,
// with the 3D VTI contrast (rho, C11, C13, C33, C55 = C44, C66; C12 = C11 - 2 C66) against an
// isotropic reference, central differences with fields zero outside the grid, and the isotropic
// 3D Green's tensor written for the exp(+i w t) convention of the 2D tensor (the complex conjugate
// of Eq. A-1 as printed). Kernels per operator pass:
//   k3_stress       sigma = dC : eps(u)  (6 Voigt components)              -> T2
//   k3_source       w^2 drho u + div sigma                                 -> T rows (x < nx)
//   k3_fft_x        forward FFT along x of every row, zero-padded to lx    (in place in T; register
//                   FFTs in k3_fft_x_reg for complex64 and lx <= 512)
//   k3_fft_y        forward FFT along y (rows y >= ny read as zero)        (in place; register
//                   FFTs in k3_fft_y_reg for complex64 and ly <= 256)
//   k3_fft_z_reg    per (ky, kx) column: forward FFT along z of the three components, the
//                   symmetric 3 x 3 Ghat product, inverse FFT along z      (in place, z < nz kept)
//                   with register FFTs (complex64, lz <= 256; k3_fft_z_mul otherwise)
//   k3_fft_y        inverse, y < ny kept
//   k3_fft_x_epi    inverse FFT along x, x < nx kept, out = ident - result (k3_fft_x_reg likewise)
// Without the stencil (plain convolution of the input, for the adjoint source) k3_copy_source
// replaces the first two kernels. The FFTs are the shared-memory Stockham transforms of fft.cuh. Ghat [nf][6][lz][ly][lx]
// (components 11, 12, 13, 22, 23, 33) carries h^3 / (lz ly lx).
#include <algorithm>
#include <cmath>

#include <vector>

#include "fft.cuh"
#include "krylov.cuh"
#include "mspace.cuh"
#include "op_tiles.cuh"

namespace dbi {

struct Ref6 {  // reference values (rho, C11, C13, C33, C55, C66) subtracted from the model
  double v[6];
};

// Problem of a launch slot, or -1 when it is out of range or inactive.
__device__ __forceinline__ int slot_problem(const int *plist, const int *active, int slot) {
  const int b = plist ? plist[slot] : slot;
  return (active && !active[b]) ? -1 : b;
}

template <typename C>
__global__ void __launch_bounds__(128) k3_stress(int nz, int ny, int nx, typename RealOf<C>::type inv2h,
                                                 const typename RealOf<C>::type *m, Ref6 ref,
                                                 const C *u, const double *in_scale, const int *plist,
                                                 const int *active, C *sig) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int zy = blockIdx.y, z = zy / ny, y = zy - z * ny, slot = blockIdx.z;
  if (x >= nx) return;
  const int b = slot_problem(plist, active, slot);
  if (b < 0) return;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(z) * ny + y) * nx + x;
  const C *ub = u + size_t(b) * 3 * cells;
  const R sc = in_scale ? R(in_scale[b]) : R(1);
  auto U = [&](int c, int dz, int dy, int dx) -> C {
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || zz >= nz || yy < 0 || yy >= ny || xx < 0 || xx >= nx) return czero<C>();
    return ub[c * cells + (size_t(zz) * ny + yy) * nx + xx];
  };
  // d u_c / d x_k (k = 0: x, 1: y, 2: z)
  auto D = [&](int c, int k) -> C {
    const C p = U(c, k == 2, k == 1, k == 0), q = U(c, -(k == 2), -(k == 1), -(k == 0));
    return cscale(csub(p, q), inv2h * sc);
  };
  const C e1 = D(0, 0), e2 = D(1, 1), e3 = D(2, 2);
  const C e4 = cadd(D(1, 2), D(2, 1)), e5 = cadd(D(0, 2), D(2, 0)), e6 = cadd(D(0, 1), D(1, 0));
  auto dm = [&](int p) { return R(double(m[p * cells + cell]) - ref.v[p]); };
  const R c11 = dm(1), c13 = dm(2), c33 = dm(3), c55 = dm(4), c66 = dm(5), c12 = c11 - R(2) * c66;
  C *sb = sig + size_t(slot) * 6 * cells + cell;
  sb[0] = cadd(cadd(cscale(e1, c11), cscale(e2, c12)), cscale(e3, c13));
  sb[cells] = cadd(cadd(cscale(e1, c12), cscale(e2, c11)), cscale(e3, c13));
  sb[2 * cells] = cadd(cscale(cadd(e1, e2), c13), cscale(e3, c33));
  sb[3 * cells] = cscale(e4, c55);
  sb[4 * cells] = cscale(e5, c55);
  sb[5 * cells] = cscale(e6, c66);
}

template <typename C>
__global__ void __launch_bounds__(128) k3_source(int nz, int ny, int nx, int ly, int lx, int nf,
                                                 typename RealOf<C>::type inv2h, const typename RealOf<C>::type *m,
                                                 Ref6 ref, const C *u, const double *in_scale,
                                                 const double *omega, const int *fidx, const int *plist,
                                                 const int *active, const C *sig, C *T) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int zy = blockIdx.y, z = zy / ny, y = zy - z * ny, slot = blockIdx.z;
  if (x >= nx) return;
  const int b = slot_problem(plist, active, slot);
  if (b < 0 || unsigned(fidx[b]) >= unsigned(nf)) return;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(z) * ny + y) * nx + x;
  const C *sb = sig + size_t(slot) * 6 * cells;
  auto S = [&](int k, int dz, int dy, int dx) -> C {
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || zz >= nz || yy < 0 || yy >= ny || xx < 0 || xx >= nx) return czero<C>();
    return sb[k * cells + (size_t(zz) * ny + yy) * nx + xx];
  };
  // d sigma_k / d x_a (Voigt k: 0 s11, 1 s22, 2 s33, 3 s23, 4 s13, 5 s12)
  auto D = [&](int k, int a) -> C {
    return cscale(csub(S(k, a == 2, a == 1, a == 0), S(k, -(a == 2), -(a == 1), -(a == 0))), inv2h);
  };
  const double w = omega[fidx[b]];
  const R sc = in_scale ? R(in_scale[b]) : R(1);
  const R wr = R(w * w * (double(m[cell]) - ref.v[0])) * sc;
  const C *ub = u + size_t(b) * 3 * cells;
  const C d0 = cadd(cadd(D(0, 0), D(5, 1)), D(4, 2));
  const C d1 = cadd(cadd(D(5, 0), D(1, 1)), D(3, 2));
  const C d2 = cadd(cadd(D(4, 0), D(3, 1)), D(2, 2));
  const C dv[3] = {d0, d1, d2};
  C *Tb = T + size_t(slot) * 3 * nz * ly * lx;
  for (int c = 0; c < 3; ++c)
    Tb[((size_t(c) * nz + z) * ly + y) * lx + x] = cadd(dv[c], cscale(ub[c * cells + cell], wr));
}

// Plain convolution (no stencil): the input itself, times its scale, as the source rows of T.
template <typename C>
__global__ void __launch_bounds__(128) k3_copy_source(int nz, int ny, int nx, int ly, int lx, const C *u,
                                                      const double *in_scale, const int *plist, const int *active,
                                                      C *T) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int zy = blockIdx.y, z = zy / ny, y = zy - z * ny, slot = blockIdx.z;
  if (x >= nx) return;
  const int b = slot_problem(plist, active, slot);
  if (b < 0) return;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(z) * ny + y) * nx + x;
  const R sc = in_scale ? R(in_scale[b]) : R(1);
  C *Tb = T + size_t(slot) * 3 * nz * ly * lx;
  for (int c = 0; c < 3; ++c)
    Tb[((size_t(c) * nz + z) * ly + y) * lx + x] = cscale(u[size_t(b) * 3 * cells + c * cells + cell], sc);
}

// Forward FFT along x of the rows (slot, c, z, y < ny) of T: points x < nx read, the rest zero.
template <typename C, int LX>
__global__ void __launch_bounds__(256) k3_fft_x(int nb, int nz, int ny, int nx, int ly, const int *plist,
                                                const int *active, const C *tw, C *T) {
  constexpr int NL = 2048 / LX, LS = LX + 1, NT = NL * LX / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  const long rows = long(nb) * 3 * nz * ny, r0 = long(blockIdx.x) * NL;
  auto row_ptr = [&](long r, bool &live) -> C * {
    const long per = long(3) * nz * ny;
    const int slot = int(r / per);
    const long rem = r - slot * per;
    const int cz = int(rem / ny), y = int(rem - long(cz) * ny);
    live = r < rows && slot_problem(plist, active, slot) >= 0;
    return T + ((size_t(slot) * 3 * nz + cz) * ly + y) * LX;
  };
  for (int idx = threadIdx.x; idx < NL * LX; idx += NT) {
    const int l = idx / LX, k = idx - l * LX;
    bool live;
    const C *p = row_ptr(r0 + l, live);
    s[l * LS + k] = (live && k < nx) ? p[k] : czero<C>();
  }
  __syncthreads();
  Plan<LX>::template run<C, NL, LS, NT, false>(s, tw);
  for (int idx = threadIdx.x; idx < NL * LX; idx += NT) {
    const int l = idx / LX, k = idx - l * LX;
    bool live;
    C *p = row_ptr(r0 + l, live);
    if (live) p[k] = s[l * LS + k];
  }
}

// The x passes with register-resident FFTs (complex64, LX <= 512): a row's T = LX / 8 threads hold
// its points x = t + m T, so the row is read and written in place with coalesced accesses and no
// staging; ROWS = 256 / T rows per CTA, each exchanging through its own shared-memory line. Every
// row of the CTA runs the transform (rows past the batch or of inactive slots on zeros, without
// loads or stores), so the warp-level barriers of rows sharing a warp always meet. EPI = false: the
// forward transform of the nx source points of each row (the second half of the line is zero);
// EPI = true: the inverse transform of the lx spectra, out = ident - osc y for x < nx.
template <int LX> struct XRegCfg {
  static constexpr int T = LX / 8, ROWS = kTileThreads / T;
  static constexpr int LP = RegFFT<float2, LX>::LP;
  static constexpr size_t smem = size_t(ROWS) * LP * sizeof(float2);
};
template <int LX, bool EPI>
__global__ void __launch_bounds__(kTileThreads) k3_fft_x_reg(int nb, int nz, int ny, int nx, int ly, const int *plist,
                                                             const int *active, const float2 *tw, float2 *T,
                                                             const float2 *ident, const double *out_scale,
                                                             float2 *out) {
  using C = float2;
  using X = XRegCfg<LX>;
  constexpr int TX = X::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  const int rr = threadIdx.x / TX, t = threadIdx.x - rr * TX;
  const long per = long(3) * nz * ny, rows = long(nb) * per;
  const long r = long(blockIdx.x) * X::ROWS + rr;
  const int slot = int(r < rows ? r / per : 0);
  const long rem = r - long(slot) * per;
  const int cz = int(rem / ny), y = int(rem - long(cz) * ny);  // cz = c nz + z
  const int b = r < rows ? slot_problem(plist, active, slot) : -1;
  const bool live = b >= 0;
  C *row = T + ((size_t(slot) * 3 * nz + cz) * ly + y) * LX;
  const TwReg<C, LX> tr(t, tw);
  C *const line[1] = {s + size_t(rr) * X::LP};
  C v[1][8];
  if constexpr (!EPI) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x = t + m * TX;
      v[0][m] = (live && m < kHalf && x < nx) ? row[x] : czero<C>();
    }
    RegPlan<LX>::template run<C, 1, false, true>(v, line, t, tr, RowSync<TX>{1 + rr});
    if (live) {
#pragma unroll
      for (int m = 0; m < 8; ++m) row[t + m * TX] = v[0][m];
    }
  } else {
#pragma unroll
    for (int m = 0; m < 8; ++m) v[0][m] = live ? row[t + m * TX] : czero<C>();
    RegPlan<LX>::template run<C, 1, true>(v, line, t, tr, RowSync<TX>{1 + rr});
    if (live) {
      const size_t cells = size_t(nz) * ny * nx;
      const float osc = out_scale ? float(out_scale[b]) : 1.0f;
      const size_t o0 = size_t(b) * 3 * cells + (size_t(cz) * ny + y) * nx;
#pragma unroll
      for (int m = 0; m < kHalf; ++m) {
        const int x = t + m * TX;
        if (x < nx) {
          const C w = cscale(v[0][m], osc);
          out[o0 + x] = ident ? csub(ident[o0 + x], w) : w;
        }
      }
    }
  }
}

// FFT along y of the planes (slot, c, z) [ly][lx], CC columns per CTA. Forward: rows y >= ny read
// as zero, all ly written; inverse: all read, y < ny written.
template <typename C, int LY> struct YCfg {
  static constexpr int CC = 2048 / LY, LS = LY + 1, NT = CC * LY / 8;  // 256 threads
};
template <typename C, int LY, bool INV>
__global__ void __launch_bounds__(256) k3_fft_y(int nz, int ny, int lx, const int *plist, const int *active,
                                                const C *tw, C *T) {
  constexpr int CC = YCfg<C, LY>::CC, LS = YCfg<C, LY>::LS, NT = YCfg<C, LY>::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  const int plane = blockIdx.y, slot = plane / (3 * nz);
  if (slot_problem(plist, active, slot) < 0) return;  // uniform over the CTA
  C *M = T + size_t(plane) * LY * lx;
  const int c0 = blockIdx.x * CC;
  for (int idx = threadIdx.x; idx < CC * LY; idx += NT) {
    const int y = idx / CC, j = idx - y * CC;
    s[j * LS + y] = (c0 + j < lx && (INV || y < ny)) ? M[size_t(y) * lx + c0 + j] : czero<C>();
  }
  __syncthreads();
  Plan<LY>::template run<C, CC, LS, NT, INV>(s, tw);
  for (int idx = threadIdx.x; idx < CC * LY; idx += NT) {
    const int y = idx / CC, j = idx - y * CC;
    if (c0 + j < lx && (!INV || y < ny)) M[size_t(y) * lx + c0 + j] = s[j * LS + y];
  }
}

// The y passes with register-resident FFTs (complex64, LY <= 256): per plane (slot, c, z), CC =
// 256 / T columns per CTA staged through shared memory in runs of CC consecutive columns, each
// column's T = LY / 8 threads holding its line in registers. Forward: rows y < ny staged (the rest
// zero), all ly written; inverse: all staged, y < ny written.
// Line pitch of the staged y and z lines: odd (in 8-byte points), so that the staging loops, whose
// consecutive threads walk consecutive lines at one point, hit 16 distinct bank slots per half warp
// (with the even RegFFT pitch they hit 4 to 8).
template <int L> constexpr int staged_pitch() { return RegFFT<float2, L>::LP | 1; }
template <int LY> struct YRegCfg {
  using C = float2;
  static constexpr int T = LY / 8, NT = kTileThreads, CC = NT / T;
  static constexpr int LP = staged_pitch<LY>();
  static constexpr size_t smem = size_t(CC) * LP * sizeof(C);
};
template <int LY, bool INV>
__global__ void __launch_bounds__(kTileThreads, 4) k3_fft_y_reg(int nz, int ny, int lx, const int *plist,
                                                               const int *active, const float2 *tw, float2 *T) {
  using C = float2;
  using Y = YRegCfg<LY>;
  constexpr int TY = Y::T, CC = Y::CC, LP = Y::LP, NT = Y::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  const int plane = blockIdx.y, slot = plane / (3 * nz);
  if (slot_problem(plist, active, slot) < 0) return;  // uniform over the CTA
  C *M = T + size_t(plane) * LY * lx;
  const int c0 = blockIdx.x * CC;
  const int rows_in = INV ? LY : ny, rows_out = INV ? ny : LY;
  for (int idx = threadIdx.x; idx < CC * rows_in; idx += NT) {  // all copies in flight at once
    const int y = idx / CC, j = idx - y * CC;
    const bool in = c0 + j < lx;
    cp_async8(s + j * LP + y, M + (in ? size_t(y) * lx + c0 + j : 0), in);
  }
  cp_async_wait_all();
  __syncthreads();
  const int g = threadIdx.x / TY, t = threadIdx.x - g * TY;
  C *const line[1] = {s + size_t(g) * LP};
  const TwReg<C, LY> tr(t, tw);
  const RowSync<TY> sync{1 + g};
  C v[1][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int y = t + m * TY;
    v[0][m] = (INV || (m < kHalf && y < ny)) ? line[0][y] : czero<C>();
  }
  sync();  // the transform's first exchange overwrites the staged line
  RegPlan<LY>::template run<C, 1, INV, !INV>(v, line, t, tr, sync);
  // every thread of the column is past the transform's last exchange: its line is free
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int y = t + m * TY;
    if (!INV || (m < kHalf && y < ny)) line[0][y] = v[0][m];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < CC * rows_out; idx += NT) {
    const int y = idx / CC, j = idx - y * CC;
    if (c0 + j < lx) M[size_t(y) * lx + c0 + j] = s[j * LP + y];
  }
}

// Per (ky, kx) column q of a slot: the three components' z-lines (z < nz, zero-padded to LZ),
// forward FFT, out_i = sum_j Ghat_ij(kz, q) v_j, inverse FFT, z < nz written back, with the
// shared-memory FFTs of fft.cuh (complex128, and complex64 beyond LZ = 256).
// CC = 1024 / LZ columns per CTA (384 threads up to LZ = 1024): small CTAs, several per SM. Wider
// tiles (32 columns, 768 threads at LZ = 64) gave longer row runs but fewer resident warps and
// were 60 % slower.
#ifndef DBI_3D_ZCOLS
#define DBI_3D_ZCOLS 1024
#endif
template <typename C, int LZ> struct ZCfg {
  static constexpr int CC = DBI_3D_ZCOLS / LZ > 0 ? DBI_3D_ZCOLS / LZ : 1;
  static constexpr int NL = 3 * CC, LS = LZ + 1, NT = NL * LZ / 8;
  // complex64: 8 CTAs per SM up to 192 threads, 4 up to 384; complex128 would spill
  static constexpr int MIN_BLOCKS = sizeof(C) == 8 ? (NT <= 192 ? 8 : (NT <= 384 ? 4 : 2)) : 1;
};
template <typename C, int LZ>
__global__ void __launch_bounds__(ZCfg<C, LZ>::NT, ZCfg<C, LZ>::MIN_BLOCKS) k3_fft_z_mul(int nb, int nz, int nf, size_t plane, const int *plist,
                                                                const int *active, const int *fidx, const C *Ghat,
                                                                const C *tw, C *T) {
  using Z = ZCfg<C, LZ>;
  constexpr int CC = Z::CC, NL = Z::NL, LS = Z::LS, NT = Z::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  // slot fastest: the CTAs in flight cover every slot of a few column tiles, so the slots of one
  // frequency read each tile of Ghat together and all but the first find it in L2 (one frequency's
  // table can exceed L2, and the slots of one frequency would otherwise each stream all of it)
  const int slot = int(blockIdx.x % unsigned(nb));
  const int b = slot_problem(plist, active, slot);
  if (b < 0 || unsigned(fidx[b]) >= unsigned(nf)) return;
  C *Tb = T + size_t(slot) * 3 * nz * plane;
  const size_t q0 = size_t(blockIdx.x / unsigned(nb)) * CC;
  for (int idx = threadIdx.x; idx < NL * LZ; idx += NT) {
    const int z = idx / NL, l = idx - z * NL, c = l / CC, j = l - c * CC;
    s[l * LS + z] = (z < nz && q0 + j < plane) ? Tb[(size_t(c) * nz + z) * plane + q0 + j] : czero<C>();
  }
  __syncthreads();
  Plan<LZ>::template run<C, NL, LS, NT, false>(s, tw);
  const C *G = Ghat + size_t(fidx[b]) * 6 * LZ * plane;
  for (int idx = threadIdx.x; idx < CC * LZ; idx += NT) {
    const int kz = idx / CC, j = idx - kz * CC;
    if (q0 + j >= plane) continue;
    const size_t o = size_t(kz) * plane + q0 + j;
    const C g11 = G[o], g12 = G[LZ * plane + o], g13 = G[2 * LZ * plane + o];
    const C g22 = G[3 * LZ * plane + o], g23 = G[4 * LZ * plane + o], g33 = G[5 * LZ * plane + o];
    const C v1 = s[j * LS + kz], v2 = s[(CC + j) * LS + kz], v3 = s[(2 * CC + j) * LS + kz];
    s[j * LS + kz] = cadd(cadd(cmul(g11, v1), cmul(g12, v2)), cmul(g13, v3));
    s[(CC + j) * LS + kz] = cadd(cadd(cmul(g12, v1), cmul(g22, v2)), cmul(g23, v3));
    s[(2 * CC + j) * LS + kz] = cadd(cadd(cmul(g13, v1), cmul(g23, v2)), cmul(g33, v3));
  }
  __syncthreads();
  Plan<LZ>::template run<C, NL, LS, NT, true>(s, tw);
  for (int idx = threadIdx.x; idx < NL * nz; idx += NT) {
    const int z = idx / NL, l = idx - z * NL, c = l / CC, j = l - c * CC;
    if (q0 + j < plane) Tb[(size_t(c) * nz + z) * plane + q0 + j] = s[l * LS + z];
  }
}

// The z pass with register-resident FFTs (complex64, LZ <= 256: a column's T = LZ / 8 threads are
// one warp or part of one). A CTA of 256 threads takes CC = 256 / T columns: the nz rows of its
// 3 CC lines are staged through shared memory with runs of CC consecutive columns (rows [z][line]),
// each column's T threads read its three components' lines into registers (8 points each) and
// exchange through lines at the transforms' own pitch and layout (aliasing the staged rows), and
// the result goes back the same way.
#ifndef DBI_3D_ZREG_MINB
#define DBI_3D_ZREG_MINB 2  // CTAs per SM: 128 registers; 3 (80 registers) was 15 % slower, 4 no faster
#endif
template <int LZ> struct ZRegCfg {
  using C = float2;
  static constexpr int T = LZ / 8, NT = kTileThreads, CC = NT / T, NL = 3 * CC;
  static constexpr int LP = RegFFT<C, LZ>::LP;  // the lines of the transforms' exchanges
  // The staged rows [z][NL] (z < nz <= LZ / 2) alias the lines. Row pitch PL = 16 / min(T, 16) mod
  // 16: the staging loops (consecutive lines) and the threads' own reads and writes (a half warp
  // holds 16 / T lines x T points, or 16 points of one line) hit 16 distinct 8-byte bank slots.
  static constexpr int PQ = 16 / (T < 16 ? T : 16);
  static constexpr int PL = NL + ((PQ - NL % 16) + 16) % 16;
  static constexpr size_t lines = size_t(NL) * LP, rows = size_t(LZ / 2) * PL;
  static constexpr size_t smem = (lines > rows ? lines : rows) * sizeof(C);
};
template <int LZ>
__global__ void __launch_bounds__(kTileThreads, DBI_3D_ZREG_MINB) k3_fft_z_reg(int nb, int nz, int nf, size_t plane, const int *plist,
                                                               const int *active, const int *fidx, const float2 *Ghat,
                                                               const float2 *tw, float2 *T) {
  using C = float2;
  using Z = ZRegCfg<LZ>;
  constexpr int TZ = Z::T, CC = Z::CC, LP = Z::LP, NT = Z::NT, NL = Z::NL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  const int slot = int(blockIdx.x % unsigned(nb));  // slot fastest, as in k3_fft_z_mul
  const int b = slot_problem(plist, active, slot);
  if (b < 0 || unsigned(fidx[b]) >= unsigned(nf)) return;  // uniform over the CTA
  C *Tb = T + size_t(slot) * 3 * nz * plane;
  const size_t q0 = size_t(blockIdx.x / unsigned(nb)) * CC;
  constexpr int PL = Z::PL;
  for (int idx = threadIdx.x; idx < NL * nz; idx += NT) {  // rows [z][l], l = c CC + j (all in flight)
    const int z = idx / NL, l = idx - z * NL, c = l / CC, j = l - c * CC;
    const bool in = q0 + j < plane;
    cp_async8(s + z * PL + l, Tb + (in ? (size_t(c) * nz + z) * plane + q0 + j : 0), in);
  }
  cp_async_wait_all();
  __syncthreads();
  const int g = threadIdx.x / TZ, t = threadIdx.x - g * TZ;
  const size_t q = q0 + g;
  const bool live = q < plane;
  C *const lines[3] = {s + size_t(g) * LP, s + size_t(CC + g) * LP, s + size_t(2 * CC + g) * LP};
  const TwReg<C, LZ> tr(t, tw);
  const RowSync<TZ> sync{1 + g};
  C v[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int z = t + m * TZ;
      v[c][m] = (m < kHalf && z < nz) ? s[z * PL + c * CC + g] : czero<C>();
    }
  __syncthreads();  // every staged row has been read: the lines alias them
  RegPlan<LZ>::template run<C, 3, false, true>(v, lines, t, tr, sync);
  if (live) {
    const size_t e = size_t(LZ) * plane;
    const C *G = Ghat + size_t(fidx[b]) * 6 * e + q;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const size_t o = size_t(t + m * TZ) * plane;
      const C g11 = __ldg(G + o), g12 = __ldg(G + e + o), g13 = __ldg(G + 2 * e + o);
      const C g22 = __ldg(G + 3 * e + o), g23 = __ldg(G + 4 * e + o), g33 = __ldg(G + 5 * e + o);
      const C v1 = v[0][m], v2 = v[1][m], v3 = v[2][m];
      v[0][m] = cadd(cadd(cmul(g11, v1), cmul(g12, v2)), cmul(g13, v3));
      v[1][m] = cadd(cadd(cmul(g12, v1), cmul(g22, v2)), cmul(g23, v3));
      v[2][m] = cadd(cadd(cmul(g13, v1), cmul(g23, v2)), cmul(g33, v3));
    }
  }
  RegPlan<LZ>::template run<C, 3, true>(v, lines, t, tr, sync);
  __syncthreads();  // every line's last exchange is done: the rows alias them
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < kHalf; ++m) {
      const int z = t + m * TZ;
      if (z < nz) s[z * PL + c * CC + g] = v[c][m];
    }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NL * nz; idx += NT) {
    const int z = idx / NL, l = idx - z * NL, c = l / CC, j = l - c * CC;
    if (q0 + j < plane) Tb[(size_t(c) * nz + z) * plane + q0 + j] = s[z * PL + l];
  }
}

// Inverse FFT along x of the rows (slot, c, z, y < ny); out = ident - osc result (x < nx).
template <typename C, int LX>
__global__ void __launch_bounds__(256) k3_fft_x_epi(int nb, int nz, int ny, int nx, int ly, const int *plist,
                                                    const int *active, const C *tw, const C *T, const C *ident,
                                                    const double *out_scale, C *out) {
  using R = typename RealOf<C>::type;
  constexpr int NL = 2048 / LX, LS = LX + 1, NT = NL * LX / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *s = reinterpret_cast<C *>(smem_raw);
  const long per = long(3) * nz * ny, rows = long(nb) * per, r0 = long(blockIdx.x) * NL;
  const size_t cells = size_t(nz) * ny * nx;
  for (int idx = threadIdx.x; idx < NL * LX; idx += NT) {
    const int l = idx / LX, k = idx - l * LX;
    const long r = r0 + l;
    const int slot = int(r / per);
    const long rem = r - slot * per;
    const int cz = int(rem / ny), y = int(rem - long(cz) * ny);
    const bool live = r < rows && slot_problem(plist, active, slot) >= 0;
    s[l * LS + k] = live ? T[((size_t(slot) * 3 * nz + cz) * ly + y) * LX + k] : czero<C>();
  }
  __syncthreads();
  Plan<LX>::template run<C, NL, LS, NT, true>(s, tw);
  for (int idx = threadIdx.x; idx < NL * LX; idx += NT) {
    const int l = idx / LX, k = idx - l * LX;
    const long r = r0 + l;
    if (r >= rows || k >= nx) continue;
    const int slot = int(r / per);
    const int b = slot_problem(plist, active, slot);
    if (b < 0) continue;
    const long rem = r - slot * per;
    const int cz = int(rem / ny), y = int(rem - long(cz) * ny);
    const size_t o = size_t(b) * 3 * cells + (size_t(cz) * ny + y) * nx + k;  // cz = c nz + z
    const C v = cscale(s[l * LS + k], out_scale ? R(out_scale[b]) : R(1));
    out[o] = ident ? csub(ident[o], v) : v;
  }
}

template <typename C> static int run3_typed(const OpArgs &a, cudaStream_t s) {
  using R = typename RealOf<C>::type;
  const int nb = a.plist ? a.nb : a.B;
  if (nb <= 0) return DBI_OK;
  const R inv2h = R(1.0 / (2.0 * a.h));
  const R *m = static_cast<const R *>(a.m);
  const C *in = static_cast<const C *>(a.in), *tw = static_cast<const C *>(a.tw);
  C *T = static_cast<C *>(a.T), *sig = static_cast<C *>(a.T2);
  Ref6 ref;
  for (int i = 0; i < 6; ++i) ref.v[i] = a.ref[i];
  int rc;
  prof_mark(PROF_OPERATOR, false, s);
  const dim3 cg((a.nx + 127) / 128, a.nz * a.ny, nb);
  if (a.stencil) {
    k3_stress<C><<<cg, 128, 0, s>>>(a.nz, a.ny, a.nx, inv2h, m, ref, in, a.in_scale, a.plist, a.active, sig);
    if ((rc = check_launch("k3_stress"))) return rc;
    k3_source<C><<<cg, 128, 0, s>>>(a.nz, a.ny, a.nx, a.ly, a.lx, a.nf, inv2h, m, ref, in, a.in_scale, a.omega,
                                    a.fidx, a.plist, a.active, sig, T);
    if ((rc = check_launch("k3_source"))) return rc;
  } else {
    k3_copy_source<C><<<cg, 128, 0, s>>>(a.nz, a.ny, a.nx, a.ly, a.lx, in, a.in_scale, a.plist, a.active, T);
    if ((rc = check_launch("k3_copy_source"))) return rc;
  }
  rc = DBI_ERR_UNSUPPORTED;
  // the x passes: register FFTs for complex64 and lx <= 512, the shared-memory form otherwise
  auto fft_x_reg = [&](auto epi_tag) {
    constexpr bool EPI = decltype(epi_tag)::value;
    bool done = false;
    dispatch_len(a.lx, [&]<int LX>() {
      if constexpr (sizeof(C) == 8 && LX <= 512) {
        using X = XRegCfg<LX>;
        const long rows = long(nb) * 3 * a.nz * a.ny;
        cudaError_t e = allow_smem(k3_fft_x_reg<LX, EPI>, X::smem);
        if (e == cudaSuccess)
          k3_fft_x_reg<LX, EPI><<<unsigned((rows + X::ROWS - 1) / X::ROWS), kTileThreads, X::smem, s>>>(
              nb, a.nz, a.ny, a.nx, a.ly, a.plist, a.active, reinterpret_cast<const float2 *>(tw),
              reinterpret_cast<float2 *>(T), static_cast<const float2 *>(a.ident), a.out_scale,
              static_cast<float2 *>(a.out));
        rc = e != cudaSuccess ? cuda_fail("k3_fft_x_reg smem", e) : check_launch("k3_fft_x_reg");
        done = true;
      }
    });
    return done;
  };
  if (!fft_x_reg(std::false_type{})) dispatch_len(a.lx, [&]<int LX>() {
    constexpr int NL = 2048 / LX, NT = NL * LX / 8;
    const size_t bytes = size_t(NL) * (LX + 1) * sizeof(C);
    const long rows = long(nb) * 3 * a.nz * a.ny;
    cudaError_t e = allow_smem(k3_fft_x<C, LX>, bytes);
    if (e == cudaSuccess)
      k3_fft_x<C, LX><<<unsigned((rows + NL - 1) / NL), NT, bytes, s>>>(nb, a.nz, a.ny, a.nx, a.ly, a.plist,
                                                                       a.active, tw, T);
    rc = e != cudaSuccess ? cuda_fail("k3_fft_x smem", e) : check_launch("k3_fft_x");
  });
  if (rc) return rc;
  auto fft_y = [&](auto inv_tag) {
    constexpr bool INV = decltype(inv_tag)::value;
    rc = DBI_ERR_UNSUPPORTED;
    dispatch_len(a.ly, [&]<int LY>() {
      if constexpr (sizeof(C) == 8 && LY <= 256) {
        using Y = YRegCfg<LY>;
        cudaError_t e = allow_smem(k3_fft_y_reg<LY, INV>, Y::smem);
        const dim3 grid((a.lx + Y::CC - 1) / Y::CC, nb * 3 * a.nz);
        if (e == cudaSuccess)
          k3_fft_y_reg<LY, INV><<<grid, Y::NT, Y::smem, s>>>(a.nz, a.ny, a.lx, a.plist, a.active,
                                                             reinterpret_cast<const float2 *>(tw),
                                                             reinterpret_cast<float2 *>(T));
        rc = e != cudaSuccess ? cuda_fail("k3_fft_y_reg smem", e) : check_launch("k3_fft_y_reg");
        return;
      }
      constexpr int CC = YCfg<C, LY>::CC, NT = YCfg<C, LY>::NT;
      const size_t bytes = size_t(CC) * (LY + 1) * sizeof(C);
      cudaError_t e = allow_smem(k3_fft_y<C, LY, INV>, bytes);
      const dim3 grid((a.lx + CC - 1) / CC, nb * 3 * a.nz);
      if (e == cudaSuccess) k3_fft_y<C, LY, INV><<<grid, NT, bytes, s>>>(a.nz, a.ny, a.lx, a.plist, a.active, tw, T);
      rc = e != cudaSuccess ? cuda_fail("k3_fft_y smem", e) : check_launch("k3_fft_y");
    });
    return rc;
  };
  if ((rc = fft_y(std::false_type{}))) return rc;
  prof_mark(PROF_COLS, false, s);
  rc = DBI_ERR_UNSUPPORTED;
  dispatch_len(a.lz, [&]<int LZ>() {
    if constexpr (sizeof(C) == 8 && LZ <= 256) {
      using Z = ZRegCfg<LZ>;
      const size_t plane = size_t(a.ly) * a.lx;
      const size_t blocks = (plane + Z::CC - 1) / Z::CC * size_t(nb);
      if (blocks > size_t(INT32_MAX)) {
        set_error("3D z pass: %zu blocks exceed the launch limit", blocks);
        rc = DBI_ERR_UNSUPPORTED;
        return;
      }
      cudaError_t e = allow_smem(k3_fft_z_reg<LZ>, Z::smem);
      if (e == cudaSuccess)
        k3_fft_z_reg<LZ><<<unsigned(blocks), Z::NT, Z::smem, s>>>(
            nb, a.nz, a.nf, plane, a.plist, a.active, a.fidx, static_cast<const float2 *>(a.Ghat),
            reinterpret_cast<const float2 *>(tw), reinterpret_cast<float2 *>(T));
      rc = e != cudaSuccess ? cuda_fail("k3_fft_z_reg smem", e) : check_launch("k3_fft_z_reg");
      return;
    }
    using Z = ZCfg<C, LZ>;
    const size_t bytes = size_t(Z::NL) * Z::LS * sizeof(C);
    const size_t plane = size_t(a.ly) * a.lx;
    cudaError_t e = allow_smem(k3_fft_z_mul<C, LZ>, bytes);
    const size_t blocks = (plane + Z::CC - 1) / Z::CC * size_t(nb);
    if (blocks > size_t(INT32_MAX)) {
      set_error("3D z pass: %zu blocks exceed the launch limit", blocks);
      rc = DBI_ERR_UNSUPPORTED;
      return;
    }
    if (e == cudaSuccess)
      k3_fft_z_mul<C, LZ><<<unsigned(blocks), Z::NT, bytes, s>>>(nb, a.nz, a.nf, plane, a.plist, a.active, a.fidx,
                                                     static_cast<const C *>(a.Ghat), tw, T);
    rc = e != cudaSuccess ? cuda_fail("k3_fft_z_mul smem", e) : check_launch("k3_fft_z_mul");
  });
  prof_mark(PROF_COLS, true, s);
  if (rc) return rc;
  if ((rc = fft_y(std::true_type{}))) return rc;
  rc = DBI_ERR_UNSUPPORTED;
  if (!fft_x_reg(std::true_type{})) dispatch_len(a.lx, [&]<int LX>() {
    constexpr int NL = 2048 / LX, NT = NL * LX / 8;
    const size_t bytes = size_t(NL) * (LX + 1) * sizeof(C);
    const long rows = long(nb) * 3 * a.nz * a.ny;
    cudaError_t e = allow_smem(k3_fft_x_epi<C, LX>, bytes);
    if (e == cudaSuccess)
      k3_fft_x_epi<C, LX><<<unsigned((rows + NL - 1) / NL), NT, bytes, s>>>(
          nb, a.nz, a.ny, a.nx, a.ly, a.plist, a.active, tw, T, static_cast<const C *>(a.ident), a.out_scale,
          static_cast<C *>(a.out));
    rc = e != cudaSuccess ? cuda_fail("k3_fft_x_epi smem", e) : check_launch("k3_fft_x_epi");
  });
  prof_mark(PROF_OPERATOR, true, s);
  return rc;
}

int run_operator_3d(const OpArgs &a, cudaStream_t s) {
  if (a.epi != 0) {
    set_error("the 3D operator has no fused inner products (use GMRES)");
    return DBI_ERR_UNSUPPORTED;
  }
  return a.precision == DBI_C64 ? run3_typed<float2>(a, s) : run3_typed<double2>(a, s);
}

}  // namespace dbi

// ---------------------------------------------------------------------------------------------
// 3D Green's tables and incident fields
// ---------------------------------------------------------------------------------------------
namespace dbi {

// G_ij at offset y != 0 (components 11, 12, 13, 22, 23, 33): with g = y / r,
// D_c = exp(-i k_c r) / (4 pi rho c^2 r), Q_c = q + q^2, q = 1 / (i k_c r),
// G = D_p [g g^T + (3 g g^T - I) Q_p] - D_s [(g g^T - I) + (3 g g^T - I) Q_s].
__device__ void green3_offset(double y1, double y2, double y3, double w, double alpha, double beta, double rho,
                              double2 g[6]) {
  const double r = sqrt(y1 * y1 + y2 * y2 + y3 * y3);
  const double gm[3] = {y1 / r, y2 / r, y3 / r};
  double2 Dc[2], Qc[2];
  const double cs[2] = {alpha, beta};
  for (int m = 0; m < 2; ++m) {
    const double k = w / cs[m], kr = k * r, f = 1.0 / (4.0 * M_PI * rho * cs[m] * cs[m] * r);
    double sn, cn;
    sincos(kr, &sn, &cn);
    Dc[m] = make_double2(cn * f, -sn * f);
    Qc[m] = make_double2(-1.0 / (kr * kr), -1.0 / kr);  // -i / (k r) - 1 / (k r)^2
  }
  const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {0, 1, 2, 1, 2, 2};
  for (int e = 0; e < 6; ++e) {
    const double gg = gm[I[e]] * gm[J[e]], d = I[e] == J[e] ? 1.0 : 0.0, t3 = 3.0 * gg - d;
    // P-part: Dp (gg + t3 Qp); S-part: Ds ((gg - d) + t3 Qs)
    const double2 ap = make_double2(gg + t3 * Qc[0].x, t3 * Qc[0].y);
    const double2 as = make_double2(gg - d + t3 * Qc[1].x, t3 * Qc[1].y);
    const double2 p = make_double2(Dc[0].x * ap.x - Dc[0].y * ap.y, Dc[0].x * ap.y + Dc[0].y * ap.x);
    const double2 q = make_double2(Dc[1].x * as.x - Dc[1].y * as.y, Dc[1].x * as.y + Dc[1].y * as.x);
    g[e] = make_double2(p.x - q.x, p.y - q.y);
  }
}

// Mean of G over the ball of volume h^3: delta_ij (2 k_s^2 <g_s> + k_p^2 <g_p>) / (3 rho w^2),
// <g_c> = 3 (exp(-i k a)(1 + i k a) - 1) / (4 pi a^3 k^2), a = h (3 / (4 pi))^(1/3).
__device__ double2 green3_self(double h, double w, double alpha, double beta, double rho) {
  const double a = h * cbrt(3.0 / (4.0 * M_PI));
  double2 tot = make_double2(0.0, 0.0);
  const double cs[2] = {alpha, beta}, wt[2] = {1.0, 2.0};
  for (int m = 0; m < 2; ++m) {
    const double k = w / cs[m], ka = k * a;
    double sn, cn;
    sincos(ka, &sn, &cn);
    // exp(-i k a)(1 + i k a) - 1 = (cos ka + ka sin ka - 1) + i (ka cos ka - sin ka)
    const double f = 3.0 / (4.0 * M_PI * a * a * a * k * k) * wt[m] * k * k;
    tot.x += f * (cn + ka * sn - 1.0);
    tot.y += f * (ka * cn - sn);
  }
  const double d = 1.0 / (3.0 * rho * w * w);
  return make_double2(tot.x * d, tot.y * d);
}

// One thread per offset (dz, dy, dx) >= 0, mirrored into the octant slots: the diagonal
// components are even in every coordinate, G_12 odd in x and y, G_13 in x and z, G_23 in y and z.
template <typename C>
__global__ void k3_green_space(int nz, int ny, int nx, int lz, int ly, int lx, double h, const double *omega,
                               double rho, double alpha, double beta, double2 *W, C *Gspace) {
  using R = typename RealOf<C>::type;
  const int dx = blockIdx.x * blockDim.x + threadIdx.x;
  const int dzy = blockIdx.y, dz = dzy / ny, dy = dzy - dz * ny, f = blockIdx.z;
  if (dx >= nx) return;
  double2 g[6];
  if (dz == 0 && dy == 0 && dx == 0) {
    const double2 sv = green3_self(h, omega[f], alpha, beta, rho);
    for (int e = 0; e < 6; ++e) g[e] = (e == 0 || e == 3 || e == 5) ? sv : make_double2(0.0, 0.0);
  } else {
    green3_offset(dx * h, dy * h, dz * h, omega[f], alpha, beta, rho, g);
  }
  const size_t vol = size_t(lz) * ly * lx;
  for (int sz = 0; sz < 2; ++sz) {
    if (sz && dz == 0) continue;
    for (int sy = 0; sy < 2; ++sy) {
      if (sy && dy == 0) continue;
      for (int sx = 0; sx < 2; ++sx) {
        if (sx && dx == 0) continue;
        const size_t cell = (size_t(sz ? lz - dz : dz) * ly + (sy ? ly - dy : dy)) * lx + (sx ? lx - dx : dx);
        const int sg[6] = {1, (sx ^ sy) ? -1 : 1, (sx ^ sz) ? -1 : 1, 1, (sy ^ sz) ? -1 : 1, 1};
        for (int e = 0; e < 6; ++e) {
          const double2 v = make_double2(sg[e] * g[e].x, sg[e] * g[e].y);
          W[(size_t(f) * 6 + e) * vol + cell] = v;
          if (Gspace) Gspace[(size_t(f) * 6 + e) * vol + cell] = mk<C>(R(v.x), R(v.y));
        }
      }
    }
  }
}

template <typename C>
__global__ void k3_scale_cast(const double2 *W, C *Ghat, size_t n, double scale) {
  using R = typename RealOf<C>::type;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    Ghat[i] = mk<C>(R(W[i].x * scale), R(W[i].y * scale));
}

// u0[b][i] = sum_j G_ij(x - x_s) f_j; problems with an out-of-range source or frequency get 0.
template <typename C>
__global__ void k3_incident(int nf, int nz, int ny, int nx, int lz, int ly, int lx, const int *fidx,
                            const C *Gspace, const int *src, const double *forces, C *u0) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int zy = blockIdx.y, z = zy / ny, y = zy - z * ny, b = blockIdx.z;
  if (x >= nx) return;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(z) * ny + y) * nx + x;
  C *o = u0 + size_t(b) * 3 * cells + cell;
  const int zs = src[3 * b], ys = src[3 * b + 1], xs = src[3 * b + 2];
  if (zs < 0 || zs >= nz || ys < 0 || ys >= ny || xs < 0 || xs >= nx || unsigned(fidx[b]) >= unsigned(nf)) {
    for (int c = 0; c < 3; ++c) o[c * cells] = czero<C>();
    return;
  }
  const int dz = (z - zs + lz) % lz, dy = (y - ys + ly) % ly, dx = (x - xs + lx) % lx;
  const size_t vol = size_t(lz) * ly * lx, slot = (size_t(dz) * ly + dy) * lx + dx;
  const C *G = Gspace + size_t(fidx[b]) * 6 * vol + slot;
  const C g[6] = {G[0], G[vol], G[2 * vol], G[3 * vol], G[4 * vol], G[5 * vol]};
  const R f1 = R(forces[3 * b]), f2 = R(forces[3 * b + 1]), f3 = R(forces[3 * b + 2]);
  o[0] = cadd(cadd(cscale(g[0], f1), cscale(g[1], f2)), cscale(g[2], f3));
  o[cells] = cadd(cadd(cscale(g[1], f1), cscale(g[3], f2)), cscale(g[4], f3));
  o[2 * cells] = cadd(cadd(cscale(g[2], f1), cscale(g[4], f2)), cscale(g[5], f3));
}

static bool len_ok(int L) { return L >= 16 && L <= 1024 && (L & (L - 1)) == 0; }

static int check_grid3(const dbi_grid3 *g) {
  if (!g) { set_error("grid is NULL"); return DBI_ERR_ARG; }
  if (g->nz < 1 || g->ny < 1 || g->nx < 1 || !(g->h > 0) || size_t(g->nz) * g->ny > 65535) {
    set_error("3D grid needs nz, ny, nx >= 1, nz ny <= 65535 and h > 0");
    return DBI_ERR_ARG;
  }
  if (!len_ok(g->lz) || !len_ok(g->ly) || !len_ok(g->lx)) {
    set_error("FFT grid %d x %d x %d: each side must be a power of two in [16, 1024]", g->lz, g->ly, g->lx);
    return DBI_ERR_UNSUPPORTED;
  }
  if (g->lz < 2 * g->nz - 1 || g->ly < 2 * g->ny - 1 || g->lx < 2 * g->nx - 1) {
    set_error("FFT grid too small for the cells (need >= 2n - 1 on every side)");
    return DBI_ERR_ARG;
  }
  return DBI_OK;
}

static size_t csize3(int precision) { return precision == DBI_C64 ? sizeof(float2) : sizeof(double2); }
static size_t bytes_field3(const dbi_grid3 *g, int B, int precision) {
  return align256(size_t(B) * 3 * g->nz * g->ny * g->nx * csize3(precision));
}
static size_t bytes_spec3(const dbi_grid3 *g, int B, int precision) {
  return align256(size_t(B) * 3 * g->nz * g->ly * g->lx * csize3(precision));
}
static size_t bytes_sig3(const dbi_grid3 *g, int B, int precision) {
  return align256(size_t(B) * 6 * g->nz * g->ny * g->nx * csize3(precision));
}

}  // namespace dbi

using namespace dbi;

extern "C" size_t dbi_workspace_bytes_3d(const dbi_grid3 *g, int B, int precision, int op, int restart) {
  if (check_grid3(g) || check_precision(precision) || B < 0) return 0;
  const size_t tw = bytes_twiddles(precision);
  switch (op) {
    case DBI_OP_GREENS:  // B counts frequencies
      return bytes_twiddles(DBI_C128) +
             align256(size_t(B) * 6 * g->lz * g->ly * g->lx * sizeof(double2));
    case DBI_OP_APPLY:
      return tw + bytes_spec3(g, B, precision) + bytes_sig3(g, B, precision) + bytes_scales(B);
    case DBI_OP_SOLVE:
      if (restart < 1 || restart > kGmresMaxRestart) return 0;
      return tw + bytes_spec3(g, B, precision) + bytes_sig3(g, B, precision) +
             gmres_bytes_fields(bytes_field3(g, B, precision), B, restart);
    default:
      return 0;
  }
}

extern "C" int greens_tabulate_3d(const dbi_grid3 *g, const dbi_medium *ref, const double *omega, int nf,
                                  int precision, void *Ghat, void *Gspace, void *work, size_t work_bytes,
                                  dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid3(g)) || (rc = check_precision(precision))) return rc;
  if (!ref || reference_is_vti(*ref) || !(ref->rho0 > 0) || !(ref->alpha0 > ref->beta0) || !(ref->beta0 > 0)) {
    set_error("the 3D reference must be isotropic with rho0 > 0 and alpha0 > beta0 > 0");
    return DBI_ERR_ARG;
  }
  if (nf < 1 || !omega || !Ghat) { set_error("need nf >= 1, omega and Ghat"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes_3d(g, nf, precision, DBI_OP_GREENS, 1);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  double2 *tw = static_cast<double2 *>(ar.take(bytes_twiddles(DBI_C128)));
  const size_t vol = size_t(g->lz) * g->ly * g->lx, tab = size_t(nf) * 6 * vol;
  double2 *W = static_cast<double2 *>(ar.take(tab * sizeof(double2)));
  if ((rc = ar.check("greens_tabulate_3d"))) return rc;
  if ((rc = launch_twiddles(tw, DBI_C128, s))) return rc;
  cudaError_t e = cudaMemsetAsync(W, 0, tab * sizeof(double2), s);
  if (e == cudaSuccess && Gspace) e = cudaMemsetAsync(Gspace, 0, tab * csize3(precision), s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(3D Green table)", e);
  const dim3 grid((g->nx + 127) / 128, g->nz * g->ny, nf);
  if (precision == DBI_C64)
    k3_green_space<float2><<<grid, 128, 0, s>>>(g->nz, g->ny, g->nx, g->lz, g->ly, g->lx, g->h, omega, ref->rho0,
                                                ref->alpha0, ref->beta0, W, static_cast<float2 *>(Gspace));
  else
    k3_green_space<double2><<<grid, 128, 0, s>>>(g->nz, g->ny, g->nx, g->lz, g->ly, g->lx, g->h, omega,
                                                 ref->rho0, ref->alpha0, ref->beta0, W,
                                                 static_cast<double2 *>(Gspace));
  if ((rc = check_launch("k3_green_space"))) return rc;
  // FP64 3D FFT: x (rows), y (columns of the [ly][lx] planes), z (columns of [lz][ly lx])
  if ((rc = fft_rows_fp64(W, long(nf) * 6 * g->lz * g->ly, g->lx, tw, s))) return rc;
  if ((rc = fft_cols_fp64(W, nf * 6 * g->lz, g->ly, g->lx, tw, s))) return rc;
  if ((rc = fft_cols_fp64(W, nf * 6, g->lz, g->ly * g->lx, tw, s))) return rc;
  const double scale = g->h * g->h * g->h / (double(g->lz) * g->ly * g->lx);
  const int blocks = int(std::min<size_t>((tab + 255) / 256, 8192));
  if (precision == DBI_C64) k3_scale_cast<float2><<<blocks, 256, 0, s>>>(W, static_cast<float2 *>(Ghat), tab, scale);
  else k3_scale_cast<double2><<<blocks, 256, 0, s>>>(W, static_cast<double2 *>(Ghat), tab, scale);
  return check_launch("k3_scale_cast");
}

extern "C" int incident_field_3d(const dbi_grid3 *g, const dbi_batch *batch, const void *Gspace,
                                 const int *src_cells, const double *forces, void *u0, int precision,
                                 dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid3(g)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (batch->B == 0) return DBI_OK;
  if (!Gspace || !src_cells || !forces || !u0) { set_error("NULL Gspace, sources, forces or u0"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const dim3 grid((g->nx + 127) / 128, g->nz * g->ny, batch->B);
  if (precision == DBI_C64)
    k3_incident<float2><<<grid, 128, 0, s>>>(batch->nf, g->nz, g->ny, g->nx, g->lz, g->ly, g->lx, batch->fidx,
                                             static_cast<const float2 *>(Gspace), src_cells, forces,
                                             static_cast<float2 *>(u0));
  else
    k3_incident<double2><<<grid, 128, 0, s>>>(batch->nf, g->nz, g->ny, g->nx, g->lz, g->ly, g->lx, batch->fidx,
                                              static_cast<const double2 *>(Gspace), src_cells, forces,
                                              static_cast<double2 *>(u0));
  return check_launch("k3_incident");
}

static int check_model3(const dbi_model3 *model, const dbi_batch *batch, int precision) {
  int rc;
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  if ((rc = check_grid3(&model->grid)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (size_t(batch->B) * 3 * model->grid.nz > 65535) {  // grid.y of the y-line pass: (problem, component, z)
    set_error("3D batch too large: B * 3 * nz = %zu exceeds 65535 (split the batch)",
              size_t(batch->B) * 3 * model->grid.nz);
    return DBI_ERR_UNSUPPORTED;
  }
  if (reference_is_vti(model->ref)) {
    set_error("the 3D reference must be isotropic");
    return DBI_ERR_ARG;
  }
  return DBI_OK;
}

static OpArgs args3(const dbi_model3 *model, const dbi_batch *batch, const void *Ghat, int precision, void *T,
                    void *T2, void *tw) {
  const dbi_grid3 *g = &model->grid;
  OpArgs a{};
  a.precision = precision;
  a.nz = g->nz; a.ny = g->ny; a.nx = g->nx; a.lz = g->lz; a.ly = g->ly; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.m = model->m;
  reference_values(model->ref, a.ref);
  a.ref[5] = model->ref.rho0 * model->ref.beta0 * model->ref.beta0;  // C66
  a.stencil = true; a.T = T; a.T2 = T2; a.Ghat = Ghat; a.tw = tw;
  return a;
}

extern "C" int ls_apply_3d(const dbi_model3 *model, const dbi_batch *batch, const void *Ghat, const void *u,
                           void *out, int precision, void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_model3(model, batch, precision);
  if (rc || batch->B == 0) return rc;
  if (!Ghat || !u || !out || !model->m) { set_error("NULL model->m, Ghat, input or output"); return DBI_ERR_ARG; }
  if (u == out) { set_error("input and output must be distinct buffers"); return DBI_ERR_ARG; }
  const dbi_grid3 *g = &model->grid;
  const size_t need = dbi_workspace_bytes_3d(g, batch->B, precision, DBI_OP_APPLY, 1);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spec3(g, batch->B, precision));
  void *T2 = ar.take(bytes_sig3(g, batch->B, precision));
  Scales sc = carve_scales(ar, batch->B);
  if ((rc = ar.check("ls_apply_3d"))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  const size_t n = size_t(3) * g->nz * g->ny * g->nx;
  if ((rc = pow2_scales(u, precision, false, batch->B, n, sc.part, sc.scale, sc.inv, nullptr, s))) return rc;
  OpArgs a = args3(model, batch, Ghat, precision, T, T2, tw);
  a.in = u; a.ident = u; a.out = out;
  a.in_scale = sc.scale; a.out_scale = sc.inv;
  return run_operator(a, s);
}

extern "C" int ls_solve_3d(const dbi_model3 *model, const dbi_batch *batch, const void *Ghat, const void *rhs,
                           void *u, const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                           void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_model3(model, batch, precision);
  if (rc || (rc = check_krylov(opts))) return rc;
  if (restart < 1 || restart > kGmresMaxRestart) {
    set_error("restart length %d outside [1, %d]", restart, kGmresMaxRestart);
    return DBI_ERR_ARG;
  }
  if (batch->B == 0) return DBI_OK;
  if (!Ghat || !rhs || !u || !model->m) { set_error("NULL model->m, Ghat, rhs or u"); return DBI_ERR_ARG; }
  if (rhs == u) { set_error("rhs and u must be distinct buffers"); return DBI_ERR_ARG; }
  const dbi_grid3 *g = &model->grid;
  const size_t need = dbi_workspace_bytes_3d(g, batch->B, precision, DBI_OP_SOLVE, restart);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spec3(g, batch->B, precision));
  void *T2 = ar.take(bytes_sig3(g, batch->B, precision));
  if ((rc = ar.check("ls_solve_3d"))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  OpArgs a = args3(model, batch, Ghat, precision, T, T2, tw);
  return run_gmres(a, ar, bytes_field3(g, batch->B, precision), restart, rhs, u, opts->zero_guess != 0, *opts,
                   status, s);
}

// ---------------------------------------------------------------------------------------------
// Distorted-Born products in 3D (Eq. 20, 25-35 with the 3D VTI stiffness)
// ---------------------------------------------------------------------------------------------
namespace dbi {

// d[b][r][c] = u[b][c] at receiver cell r (P u); out-of-range receivers give 0.
template <typename C>
__global__ void k3_sample(int B, int nz, int ny, int nx, int n_rec, const int *rec, const C *u, C *d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * n_rec) return;
  const int b = i / n_rec, r = i - b * n_rec;
  const int iz = rec[3 * r], iy = rec[3 * r + 1], ix = rec[3 * r + 2];
  const bool in = iz >= 0 && iz < nz && iy >= 0 && iy < ny && ix >= 0 && ix < nx;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(iz) * ny + iy) * nx + ix;
  for (int c = 0; c < 3; ++c)
    d[size_t(i) * 3 + c] = in ? u[size_t(b) * 3 * cells + c * cells + cell] : czero<C>();
}

// q[b] = P^T conj(r[b]): conj(r) added at the receiver cells of a zeroed field (receivers that
// share a cell are summed).
template <typename C>
__global__ void k3_inject_conj(int B, int nz, int ny, int nx, int n_rec, const int *rec, const C *r, C *q) {
  using R = typename RealOf<C>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * n_rec) return;
  const int b = i / n_rec, k = i - b * n_rec;
  const int iz = rec[3 * k], iy = rec[3 * k + 1], ix = rec[3 * k + 2];
  if (iz < 0 || iz >= nz || iy < 0 || iy >= ny || ix < 0 || ix >= nx) return;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(iz) * ny + iy) * nx + ix;
  for (int c = 0; c < 3; ++c) {
    const C v = r[size_t(i) * 3 + c];
    R *o = reinterpret_cast<R *>(q + size_t(b) * 3 * cells + c * cells + cell);
    atomicAdd(o, v.x);
    atomicAdd(o + 1, -v.y);
  }
}

// g[p][cell] = sum_b imaging of problem b (FP64 accumulation in problem order): rho:
// Re(w^2 u_a . u_b); C_p: -Re(eps(u_a)^T B_p eps(u_b)), B_C11 = E11 + E22 + E12 + E21,
// B_C13 = E13 + E31 + E23 + E32, B_C33 = E33, B_C55 = E44 + E55, B_C66 = E66 - 2 (E12 + E21).
template <typename C, typename GOut>
__global__ void __launch_bounds__(128) k3_imaging(int B, int nf, int nz, int ny, int nx, double h, const double *omega,
                                                  const int *fidx, const C *ua, const C *ub, GOut *g) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int zy = blockIdx.y, z = zy / ny, y = zy - z * ny;
  if (x >= nx) return;
  const size_t cells = size_t(nz) * ny * nx, cell = (size_t(z) * ny + y) * nx + x;
  const R inv2h = R(1.0 / (2.0 * h));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int b = 0; b < B; ++b) {
    if (unsigned(fidx[b]) >= unsigned(nf)) continue;
    const double w = omega[fidx[b]];
    C ea[6], eb[6];
    for (int side = 0; side < 2; ++side) {
      const C *u = (side ? ub : ua) + size_t(b) * 3 * cells;
      auto U = [&](int c, int dz, int dy, int dx) -> C {
        const int zz = z + dz, yy = y + dy, xx = x + dx;
        if (zz < 0 || zz >= nz || yy < 0 || yy >= ny || xx < 0 || xx >= nx) return czero<C>();
        return u[c * cells + (size_t(zz) * ny + yy) * nx + xx];
      };
      auto D = [&](int c, int k) -> C {
        return cscale(csub(U(c, k == 2, k == 1, k == 0), U(c, -(k == 2), -(k == 1), -(k == 0))), inv2h);
      };
      C *e = side ? eb : ea;
      e[0] = D(0, 0); e[1] = D(1, 1); e[2] = D(2, 2);
      e[3] = cadd(D(1, 2), D(2, 1)); e[4] = cadd(D(0, 2), D(2, 0)); e[5] = cadd(D(0, 1), D(1, 0));
    }
    auto re = [](C a, C b) { return double(a.x) * double(b.x) - double(a.y) * double(b.y); };  // Re(a b)
    const C *pa = ua + size_t(b) * 3 * cells + cell, *pb = ub + size_t(b) * 3 * cells + cell;
    acc[0] += w * w * (re(pa[0], pb[0]) + re(pa[cells], pb[cells]) + re(pa[2 * cells], pb[2 * cells]));
    const C a12 = cadd(ea[0], ea[1]), b12 = cadd(eb[0], eb[1]);
    acc[1] -= re(a12, b12);
    acc[2] -= re(a12, eb[2]) + re(ea[2], b12);
    acc[3] -= re(ea[2], eb[2]);
    acc[4] -= re(ea[3], eb[3]) + re(ea[4], eb[4]);
    acc[5] -= re(ea[5], eb[5]) - 2.0 * (re(ea[0], eb[1]) + re(ea[1], eb[0]));
  }
  for (int p = 0; p < 6; ++p) g[p * cells + cell] = GOut(acc[p]);
}

}  // namespace dbi

static size_t bytes_products3(const dbi_grid3 *g, int B, int precision, int restart) {
  return bytes_twiddles(precision) + bytes_spec3(g, B, precision) + bytes_sig3(g, B, precision) +
         bytes_scales(B) + 2 * bytes_field3(g, B, precision) + gmres_bytes_fields(bytes_field3(g, B, precision), B, restart);
}

extern "C" size_t dbi_products_workspace_bytes_3d(const dbi_grid3 *g, int B, int precision, int restart) {
  if (check_grid3(g) || check_precision(precision) || B < 0 || restart < 1 || restart > kGmresMaxRestart) return 0;
  return bytes_products3(g, B, precision, restart);
}

namespace dbi {

// Everything the 3D products share: the background operator, two field buffers, scales, and the
// region the GMRES solves carve their basis from (afresh for every solve).
struct Ctx3 {
  OpArgs op;
  const dbi_grid3 *g;
  const dbi_batch *batch;
  void *src, *sol;
  Scales sc;
  void *gm_base;
  size_t gm_bytes, fbytes;
  int restart, precision;
  dbi_krylov_opts opts;
  const dbi_status *status;
  cudaStream_t s;
};

static int solve3(const Ctx3 &c, const void *rhs, void *x) {
  Arena ar(c.gm_base, c.gm_bytes);
  return run_gmres(c.op, ar, c.fbytes, c.restart, rhs, x, true, c.opts, c.status, c.s);
}

// d = P A_b^-1 G (w^2 dm_rho u_b + div(dC(dm) : eps(u_b)))
static int frechet3(const Ctx3 &c, const void *u_b, const int *rec, int n_rec, const void *dm, void *d) {
  const dbi_grid3 *g = c.g;
  const int B = c.batch->B;
  const size_t n = size_t(3) * g->nz * g->ny * g->nx;
  int rc;
  if ((rc = pow2_scales(u_b, c.precision, false, B, n, c.sc.part, c.sc.scale, c.sc.inv, nullptr, c.s))) return rc;
  OpArgs a = c.op;  // the perturbation as the model, a zero reference, no identity term
  a.m = dm;
  for (int i = 0; i < 6; ++i) a.ref[i] = 0.0;
  a.in = u_b; a.ident = nullptr; a.out = c.src;
  a.in_scale = c.sc.scale; a.out_scale = c.sc.inv;
  if ((rc = run_operator(a, c.s)) || (rc = solve3(c, c.src, c.sol))) return rc;
  const int tot = B * n_rec;
  if (c.precision == DBI_C64)
    k3_sample<float2><<<(tot + 127) / 128, 128, 0, c.s>>>(B, g->nz, g->ny, g->nx, n_rec, rec,
                                                          static_cast<const float2 *>(c.sol), static_cast<float2 *>(d));
  else
    k3_sample<double2><<<(tot + 127) / 128, 128, 0, c.s>>>(B, g->nz, g->ny, g->nx, n_rec, rec,
                                                           static_cast<const double2 *>(c.sol),
                                                           static_cast<double2 *>(d));
  return check_launch("k3_sample");
}

// g = Re J^H r (GOut: the precision's real type, or double for the normal equation)
template <typename GOut>
static int adjoint3(const Ctx3 &c, const void *u_b, const int *rec, int n_rec, const void *r, GOut *gout) {
  const dbi_grid3 *g = c.g;
  const int B = c.batch->B;
  const size_t n = size_t(3) * g->nz * g->ny * g->nx;
  const int tot = B * n_rec;
  int rc;
  cudaError_t e = cudaMemsetAsync(c.sol, 0, c.fbytes, c.s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(adjoint source)", e);
  if (c.precision == DBI_C64)
    k3_inject_conj<float2><<<(tot + 127) / 128, 128, 0, c.s>>>(B, g->nz, g->ny, g->nx, n_rec, rec,
                                                               static_cast<const float2 *>(r),
                                                               static_cast<float2 *>(c.sol));
  else
    k3_inject_conj<double2><<<(tot + 127) / 128, 128, 0, c.s>>>(B, g->nz, g->ny, g->nx, n_rec, rec,
                                                                static_cast<const double2 *>(r),
                                                                static_cast<double2 *>(c.sol));
  if ((rc = check_launch("k3_inject_conj"))) return rc;
  if ((rc = pow2_scales(c.sol, c.precision, false, B, n, c.sc.part, c.sc.scale, c.sc.inv, nullptr, c.s))) return rc;
  OpArgs a = c.op;  // plain convolution of the injected residual
  a.stencil = false;
  a.in = c.sol; a.ident = nullptr; a.out = c.src;
  a.in_scale = c.sc.scale; a.out_scale = c.sc.inv;
  if ((rc = run_operator(a, c.s)) || (rc = solve3(c, c.src, c.sol))) return rc;
  const dim3 grid((g->nx + 127) / 128, g->nz * g->ny);
  if (c.precision == DBI_C64)
    k3_imaging<float2, GOut><<<grid, 128, 0, c.s>>>(B, c.batch->nf, g->nz, g->ny, g->nx, g->h, c.batch->omega,
                                                    c.batch->fidx, static_cast<const float2 *>(c.sol),
                                                    static_cast<const float2 *>(u_b), gout);
  else
    k3_imaging<double2, GOut><<<grid, 128, 0, c.s>>>(B, c.batch->nf, g->nz, g->ny, g->nx, g->h, c.batch->omega,
                                                     c.batch->fidx, static_cast<const double2 *>(c.sol),
                                                     static_cast<const double2 *>(u_b), gout);
  return check_launch("k3_imaging");
}

// Validation and carving common to the 3D products (extra_bytes: what the caller carves after).
static int prepare3(const dbi_model3 *bg, const dbi_batch *batch, const void *Ghat, const void *u_b,
                    const int *rec, int n_rec, const dbi_krylov_opts *opts, int restart, const dbi_status *status,
                    int precision, void *work, size_t work_bytes, size_t extra_bytes, dbi_stream stream, Arena &ar,
                    Ctx3 &c) {
  int rc = check_model3(bg, batch, precision);
  if (rc || (rc = check_krylov(opts))) return rc;
  if (restart < 1 || restart > kGmresMaxRestart) {
    set_error("restart length %d outside [1, %d]", restart, kGmresMaxRestart);
    return DBI_ERR_ARG;
  }
  if (batch->B > 0 && (!Ghat || !u_b || !bg->m || !rec || n_rec < 1)) {
    set_error("NULL model->m, Ghat, background fields or receivers");
    return DBI_ERR_ARG;
  }
  const dbi_grid3 *g = &bg->grid;
  const size_t need = bytes_products3(g, batch->B, precision, restart) + extra_bytes;
  if (batch->B > 0 && (!work || work_bytes < need)) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  if (batch->B == 0) return DBI_OK;
  c.g = g;
  c.batch = batch;
  c.precision = precision;
  c.restart = restart;
  c.opts = *opts;
  c.status = status;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spec3(g, batch->B, precision));
  void *T2 = ar.take(bytes_sig3(g, batch->B, precision));
  c.sc = carve_scales(ar, batch->B);
  c.fbytes = bytes_field3(g, batch->B, precision);
  c.src = ar.take(c.fbytes);
  c.sol = ar.take(c.fbytes);
  c.gm_bytes = gmres_bytes_fields(c.fbytes, batch->B, restart);
  c.gm_base = ar.take(c.gm_bytes);
  if ((rc = ar.check("3D products"))) return rc;
  if ((rc = launch_twiddles(tw, precision, c.s))) return rc;
  c.op = args3(bg, batch, Ghat, precision, T, T2, tw);
  return DBI_OK;
}

}  // namespace dbi

extern "C" int frechet_apply_3d(const dbi_model3 *background, const dbi_batch *batch, const void *Ghat,
                                const void *u_b, const int *rec_cells, int n_rec, const void *dm, void *d,
                                const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                                void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  Arena ar(work, work_bytes);
  Ctx3 c{};
  int rc = prepare3(background, batch, Ghat, u_b, rec_cells, n_rec, opts, restart, status, precision, work,
                    work_bytes, 0, stream, ar, c);
  if (rc || batch->B == 0) return rc;
  if (!dm || !d) { set_error("NULL dm or d"); return DBI_ERR_ARG; }
  return frechet3(c, u_b, rec_cells, n_rec, dm, d);
}

extern "C" int adjoint_apply_3d(const dbi_model3 *background, const dbi_batch *batch, const void *Ghat,
                                const void *u_b, const int *rec_cells, int n_rec, const void *r, void *g_out,
                                const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                                void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  Arena ar(work, work_bytes);
  Ctx3 c{};
  int rc = prepare3(background, batch, Ghat, u_b, rec_cells, n_rec, opts, restart, status, precision, work,
                    work_bytes, 0, stream, ar, c);
  if (rc || batch->B == 0) return rc;
  if (!r || !g_out) { set_error("NULL r or g"); return DBI_ERR_ARG; }
  if (precision == DBI_C64) return adjoint3(c, u_b, rec_cells, n_rec, r, static_cast<float *>(g_out));
  return adjoint3(c, u_b, rec_cells, n_rec, r, static_cast<double *>(g_out));
}

namespace dbi {
// y = s_p x (scale = sc[S_INV]) or y = s_p x / sc[S_INV] (invert): the normal operator is applied to
// p / ||p|| and its result multiplied by ||p||, so that the single-precision fields of the Frechet
// and adjoint solves stay far from underflow whatever the size of the CG vectors
template <typename TO>
static __global__ void k3_mscale_norm(int np, size_t plane, const double *x, TO *y, MScale s, const double *sc,
                                      int invert) {
  const double f = invert ? (sc[S_INV] > 0.0 ? 1.0 / sc[S_INV] : 0.0) : sc[S_INV];
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < np * plane; i += size_t(gridDim.x) * blockDim.x)
    y[i] = TO(x[i] * s.s[i / plane] * f);
}
}  // namespace dbi

// ---------------------------------------------------------------------------------------------
// Tikhonov normal equation in 3D (Eq. 23, 24): (Re J~^H J~ + lambda I) x = Re J~^H dd on the
// relative unknowns x_p = dm_p / s_p, s = (rho0, C11_0 for C11 and C13, C33_0, C55_0, C66_0)
// ---------------------------------------------------------------------------------------------
static size_t bytes_ncg3(const dbi_grid3 *g, int B, int precision, int n_rec, int iters) {
  const size_t nm = size_t(6) * g->nz * g->ny * g->nx;
  return 5 * align256(nm * sizeof(double)) + align256(nm * sizeof(double)) + align256(kMBlocks * sizeof(double)) +
         256 + align256(size_t(iters + 1) * sizeof(double)) +
         align256(size_t(B) * n_rec * 3 * (precision == DBI_C64 ? sizeof(float2) : sizeof(double2)));
}

extern "C" size_t dbi_normal_cg_workspace_bytes_3d(const dbi_grid3 *g, int B, int precision, int restart, int n_rec,
                                                  int iters) {
  if (check_grid3(g) || check_precision(precision) || B < 1 || restart < 1 || restart > kGmresMaxRestart ||
      n_rec < 1 || iters < 0)
    return 0;
  return bytes_products3(g, B, precision, restart) + bytes_ncg3(g, B, precision, n_rec, iters);
}

extern "C" int normal_cg_3d(const dbi_model3 *background, const dbi_batch *batch, const void *Ghat, const void *u_b,
                            const int *rec_cells, int n_rec, const void *dd, const dbi_cg_opts *cg,
                            const void *power_start, void *dm, double *lambda_out, double *hist_out,
                            const dbi_krylov_opts *opts, int restart, const dbi_status *status, int precision,
                            void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  if (!cg || cg->iters < 0 || cg->iters > 4096 ||
      (!(cg->lambda > 0) && (cg->power_iters < 1 || !power_start || !(cg->lambda_rel > 0)))) {
    set_error("CG options need 0 <= iters <= 4096 and lambda > 0, or lambda_rel > 0, power_iters >= 1 and a start vector");
    return DBI_ERR_ARG;
  }
  if (!batch || batch->B < 1) { set_error("normal_cg_3d needs at least one problem"); return DBI_ERR_ARG; }
  if (!dd || !dm) { set_error("NULL dd or dm"); return DBI_ERR_ARG; }
  Arena ar(work, work_bytes);
  Ctx3 c{};
  const size_t extra = background ? bytes_ncg3(&background->grid, batch->B, precision, n_rec, cg->iters) : 0;
  int rc = prepare3(background, batch, Ghat, u_b, rec_cells, n_rec, opts, restart, status, precision, work,
                    work_bytes, extra, stream, ar, c);
  if (rc) return rc;
  const dbi_grid3 *g = c.g;
  const size_t plane = size_t(g->nz) * g->ny * g->nx, nm = 6 * plane, mb = nm * sizeof(double);
  double *x = static_cast<double *>(ar.take(mb));
  double *r = static_cast<double *>(ar.take(mb));
  double *p = static_cast<double *>(ar.take(mb));
  double *q = static_cast<double *>(ar.take(mb));
  double *gd = static_cast<double *>(ar.take(mb));
  void *dmt = ar.take(mb);  // the precision's real type
  double *part = static_cast<double *>(ar.take(kMBlocks * sizeof(double)));
  double *sc = static_cast<double *>(ar.take(16 * sizeof(double)));
  double *hist = static_cast<double *>(ar.take(size_t(cg->iters + 1) * sizeof(double)));
  void *dvec = ar.take(size_t(batch->B) * n_rec * 3 * (precision == DBI_C64 ? sizeof(float2) : sizeof(double2)));
  if ((rc = ar.check("normal_cg_3d"))) return rc;
  cudaStream_t s = c.s;
  const dbi_medium &m0 = background->ref;
  const double a2 = m0.rho0 * m0.alpha0 * m0.alpha0, b2 = m0.rho0 * m0.beta0 * m0.beta0;
  const MScale MS{{m0.rho0, a2, a2, a2, b2, b2}};
  const MScale one{{1, 1, 1, 1, 1, 1}};
  const int mblocks = int(std::min<size_t>((nm + 255) / 256, 4096));
  auto dot = [&](const double *a, const double *b) -> int {
    k_mdot<<<kMBlocks, kMThreads, 0, s>>>(nm, a, b, part);
    return check_launch("k_mdot");
  };
  auto scal = [&](int what, int k) -> int {
    k_scalar<<<1, 32, 0, s>>>(what, part, sc, hist, k);
    return check_launch("k_scalar");
  };
  auto H = [&](const double *pin, double *qout) -> int {  // S Re J^H J S p, applied to p / ||p||
    int e;
    if ((e = dot(pin, pin)) || (e = scal(3, 0))) return e;  // sc[S_INV] = 1 / ||p||
    if (precision == DBI_C64)
      k3_mscale_norm<float><<<mblocks, 256, 0, s>>>(6, plane, pin, static_cast<float *>(dmt), MS, sc, 0);
    else k3_mscale_norm<double><<<mblocks, 256, 0, s>>>(6, plane, pin, static_cast<double *>(dmt), MS, sc, 0);
    if ((e = check_launch("k3_mscale_norm"))) return e;
    if ((e = frechet3(c, u_b, rec_cells, n_rec, dmt, dvec))) return e;
    if ((e = adjoint3<double>(c, u_b, rec_cells, n_rec, dvec, gd))) return e;
    k3_mscale_norm<double><<<mblocks, 256, 0, s>>>(6, plane, gd, qout, MS, sc, 1);
    return check_launch("k3_mscale_norm");
  };
  auto axpy = [&](int mode, const double *xx, double *yy, const double *qq, double *rr) -> int {
    k_maxpy<<<mblocks, 256, 0, s>>>(nm, mode, sc, xx, yy, qq, rr);
    return check_launch("k_maxpy");
  };
  double init_sc[16] = {0};
  init_sc[S_LAMBDA] = cg->lambda;
  init_sc[S_LREL] = cg->lambda_rel;
  cudaError_t e = cudaMemcpyAsync(sc, init_sc, sizeof(init_sc), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail("cudaMemcpyAsync(scalars)", e);
  if (!(cg->lambda > 0)) {  // lambda = lambda_rel x the Rayleigh quotient after power steps
    if (precision == DBI_C64) k_mscale<float, double><<<mblocks, 256, 0, s>>>(6, plane, static_cast<const float *>(power_start), p, one);
    else k_mscale<double, double><<<mblocks, 256, 0, s>>>(6, plane, static_cast<const double *>(power_start), p, one);
    if ((rc = check_launch("k_mscale"))) return rc;
    if ((rc = dot(p, p)) || (rc = scal(3, 0)) || (rc = axpy(2, p, p, nullptr, nullptr))) return rc;
    for (int it = 0; it < cg->power_iters; ++it)
      if ((rc = H(p, q)) || (rc = dot(q, q)) || (rc = scal(3, 0)) || (rc = axpy(2, q, p, nullptr, nullptr))) return rc;
    if ((rc = H(p, q)) || (rc = dot(p, q)) || (rc = scal(4, 0))) return rc;
  }
  if ((rc = adjoint3<double>(c, u_b, rec_cells, n_rec, dd, gd))) return rc;  // r = p = S Re J^H dd, x = 0
  k_mscale<double, double><<<mblocks, 256, 0, s>>>(6, plane, gd, r, MS);
  if ((rc = check_launch("k_mscale"))) return rc;
  e = cudaMemsetAsync(x, 0, mb, s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(x)", e);
  if ((rc = axpy(4, r, p, nullptr, nullptr)) || (rc = dot(r, r)) || (rc = scal(0, 0))) return rc;
  for (int k = 0; k < cg->iters; ++k) {
    if ((rc = H(p, q)) || (rc = axpy(3, p, q, nullptr, nullptr))) return rc;  // q = H p + lambda p
    if ((rc = dot(p, q)) || (rc = scal(1, 0))) return rc;
    if ((rc = axpy(0, p, x, q, r))) return rc;
    if ((rc = dot(r, r)) || (rc = scal(2, k + 1))) return rc;
    if ((rc = axpy(1, r, p, nullptr, nullptr))) return rc;
  }
  if (precision == DBI_C64) k_mscale<double, float><<<mblocks, 256, 0, s>>>(6, plane, x, static_cast<float *>(dm), MS);
  else k_mscale<double, double><<<mblocks, 256, 0, s>>>(6, plane, x, static_cast<double *>(dm), MS);
  if ((rc = check_launch("k_mscale"))) return rc;
  double lam = 0.0;
  std::vector<double> h(size_t(cg->iters) + 1);
  e = cudaMemcpyAsync(&lam, sc + S_LAMBDA, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail("reading the CG results", e);
  if (lambda_out) *lambda_out = lam;
  if (hist_out) for (size_t i = 0; i < h.size(); ++i) hist_out[i] = h[i];
  return DBI_OK;
}

extern "C" int sample_3d(const dbi_grid3 *g, int B, const int *rec_cells, int n_rec, const void *u, void *d,
                         int precision, dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid3(g)) || (rc = check_precision(precision))) return rc;
  if (B < 0 || n_rec < 0) { set_error("need B >= 0 and n_rec >= 0"); return DBI_ERR_ARG; }
  if (B == 0 || n_rec == 0) return DBI_OK;
  if (!rec_cells || !u || !d) { set_error("NULL receivers, u or d"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int tot = B * n_rec;
  if (precision == DBI_C64)
    k3_sample<float2><<<(tot + 127) / 128, 128, 0, s>>>(B, g->nz, g->ny, g->nx, n_rec, rec_cells,
                                                        static_cast<const float2 *>(u), static_cast<float2 *>(d));
  else
    k3_sample<double2><<<(tot + 127) / 128, 128, 0, s>>>(B, g->nz, g->ny, g->nx, n_rec, rec_cells,
                                                         static_cast<const double2 *>(u), static_cast<double2 *>(d));
  return check_launch("k3_sample");
}

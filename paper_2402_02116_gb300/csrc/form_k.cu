// The paper-literal LS operator (Eq. 9): the stress term with the derivative on the Green's tensor,
//   A u = u - [ w^2 G * (drho u) + (grad G) * sigma ],  sigma = dC : eps(u),
//   (grad G * sigma)_i = sum_jk (D_k G_ij) * sigma_jk,
// with D_k G the central differences of the lattice G_h (greens_tabulate_k) and eps the central
// differences of u (fields zero outside D). Over the five sources (w^2 drho u1, w^2 drho u3,
// sigma1, sigma5, sigma3) the kernel is the 2 x 5 matrix
//   [ G11  G13  D1G11  D3G11 + D1G13  D3G13 ]
//   [ G13  G33  D1G13  D3G13 + D1G33  D3G33 ],
// applied by Eq. 12 on the zero-padded grid. Three kernels per batch:
//   kk_rows_forward : the five source rows of a row tile, forward FFT along x of each -> T5
//   kk_cols         : per column, forward FFT along z of each source, accumulate the 2 x 5 product,
//                     inverse FFT of the two sums -> T2
//   kk_rows_inverse : the inverse row pass and epilogue of the divergence form (op_tiles.cuh)
#include <algorithm>

#include "krylov.cuh"
#include "op_tiles.cuh"
#include "operator.cuh"

namespace dbi {

template <typename C> struct KP {
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
  C *T5;  // [slot][5][lx][nz] source spectra (column-major)
  C *T2;  // [slot][2][lx][nz] output spectra
  const C *Ghat;  // [nf][3][lx][lz]
  const C *Dhat;  // [nf][6][lx][lz]
  const C *tw;
  const int *active;
  const int *plist;
  int s0;
  const double *in_scale, *m_scale, *out_scale;
  const C *krhat;
  double *part_out;
  int part_count;
};

template <typename C> __device__ __forceinline__ int kproblem(const KP<C> &p) {
  const int sl = p.s0 + int(blockIdx.y);
  return p.plist ? p.plist[sl] : sl;
}

// Accessor of the inverse-row tile body (op_tiles.cuh) over the output spectra T2.
template <typename C> struct KTile {
  using Rl = typename RealOf<C>::type;
  KP<C> p;
  int b, slot, f;
  __device__ __forceinline__ size_t fld() const { return size_t(b) * 2 * p.nz * p.nx; }
  __device__ __forceinline__ int nz() const { return p.nz; }
  __device__ __forceinline__ int nx() const { return p.nx; }
  __device__ __forceinline__ int lx() const { return p.lx; }
  __device__ __forceinline__ Rl inv2h() const { return p.inv2h; }
  __device__ __forceinline__ Rl ref(int i) const { return p.ref[i]; }
  __device__ __forceinline__ const Rl *m() const { return p.m; }
  __device__ __forceinline__ const C *in() const { return p.in + fld(); }
  __device__ __forceinline__ const C *ident() const { return p.ident ? p.ident + fld() : nullptr; }
  __device__ __forceinline__ C *out() const { return p.out + fld(); }
  __device__ __forceinline__ C *T() const { return p.T2 + size_t(slot) * 2 * p.lx * p.nz; }
  __device__ __forceinline__ const C *G() const { return p.Ghat + size_t(f) * 3 * p.lx * p.lz; }
  __device__ __forceinline__ const C *tw() const { return p.tw; }
  __device__ __forceinline__ const C *krhat() const { return p.krhat + fld(); }
  __device__ __forceinline__ double *part() const { return p.part_out + size_t(b) * p.part_count * kRedSlots; }
  __device__ __forceinline__ Rl w2() const {
    const double om = p.omega[f];
    return Rl(om * om);
  }
  __device__ __forceinline__ Rl isc() const { return p.in_scale ? Rl(p.in_scale[b]) : Rl(1); }
  __device__ __forceinline__ Rl osc() const { return p.out_scale ? Rl(p.out_scale[b]) : Rl(1); }
  __device__ __forceinline__ Rl ms() const { return p.m_scale ? Rl(p.m_scale[0]) : Rl(1); }
};

// Shared memory of kk_rows_forward: staged u [2][ROWS + 2][nx + 2], then one region that holds
// the FFT lines of two sources [2][ROWS][LP] and, after the transform, their transposition tile
// [2][LX][ROWS + 1].
template <typename C, int LX> inline size_t kk_rows_forward_smem(int nx) {
  using RC = RowCfg<C, LX>;
  const size_t region = std::max(size_t(2) * RC::ROWS * RC::LP, size_t(2) * LX * (RC::ROWS + 1));
  return (size_t(2) * (RC::ROWS + 2) * (nx + 2) + region) * sizeof(C);
}

// The five sources of ROWS rows (w^2 drho u1, w^2 drho u3, sigma1, sigma5, sigma3 with
// sigma = dC : eps(u)), two at a time ((s1, s3), (sigma1, sigma5), sigma3): zero-padded to LX,
// forward FFT along x, transposed into T5[slot][c][kx][z].
template <typename C, int LX>
__global__ void __launch_bounds__(kTileThreads) kk_rows_forward(KP<C> p) {
  using Rl = typename RealOf<C>::type;
  using RC = RowCfg<C, LX>;
  constexpr int ROWS = RC::ROWS, T = RC::T, LP = RC::LP, RG = ROWS + 2, RP = ROWS + 1;
  const int b = kproblem(p), f = p.fidx[b], slot = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  const int z0 = blockIdx.x * ROWS, nz = p.nz, nx = p.nx, W = nx + 2;
  const int rr = threadIdx.x / T, t = threadIdx.x - rr * T, z = z0 + rr;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *su = reinterpret_cast<C *>(smem_raw);  // [2][RG][W]: u at rows z0 - 1 .. z0 + ROWS
  C *R = su + size_t(2) * RG * W;           // FFT lines, then the transposition tile
  const size_t plane = size_t(nz) * nx;
  const C *u = p.in + size_t(b) * 2 * plane;
  const Rl isc = p.in_scale ? Rl(p.in_scale[b]) : Rl(1);
  for (int i = threadIdx.x; i < 2 * RG * W; i += kTileThreads) {
    const int c = i / (RG * W), rem = i - c * RG * W, r = rem / W, xx = rem - r * W - 1, zz = z0 - 1 + r;
    const bool in = zz >= 0 && zz < nz && xx >= 0 && xx < nx;
    su[i] = in ? cscale(__ldg(u + c * plane + size_t(zz) * nx + xx), isc) : czero<C>();
  }
  __syncthreads();
  const Rl ms = p.m_scale ? Rl(p.m_scale[0]) : Rl(1), fh = p.inv2h;
  const double om = p.omega[f];
  const Rl w2 = Rl(om * om);
  auto U = [&](int c, int dz, int dx, int x) { return su[(c * RG + rr + 1 + dz) * W + x + 1 + dx]; };
  auto dm = [&](int q, size_t cell) { return (__ldg(p.m + q * plane + cell) - p.ref[q]) * ms; };
  // source c at column x of this thread's row (inside D)
  auto source = [&](int c, int x) -> C {
    const size_t cell = size_t(z) * nx + x;
    if (c < 2) return cscale(U(c, 0, 0, x), w2 * dm(0, cell));
    if (c == 3) {
      const C e5 = cadd(csub(U(0, 1, 0, x), U(0, -1, 0, x)), csub(U(1, 0, 1, x), U(1, 0, -1, x)));
      return cscale(e5, fh * dm(4, cell));
    }
    const C e1 = cscale(csub(U(0, 0, 1, x), U(0, 0, -1, x)), fh);
    const C e3 = cscale(csub(U(1, 1, 0, x), U(1, -1, 0, x)), fh);
    const Rl d13 = dm(2, cell);
    return c == 2 ? cadd(cscale(e1, dm(1, cell)), cscale(e3, d13)) : cadd(cscale(e1, d13), cscale(e3, dm(3, cell)));
  };
  const TwReg<C, LX> tr(t, p.tw);
  C *Tb = p.T5 + size_t(slot) * 5 * LX * nz;
  auto pass = [&]<int NL>(int c0) {
    C v[NL][8];
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) {
        const int x = t + mm * T;
        v[l][mm] = (mm < kHalf && z < nz && x < nx) ? source(c0 + l, x) : czero<C>();
      }
    C *ln[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) ln[l] = R + size_t(l * ROWS + rr) * LP;
    RegPlan<LX>::template run<C, NL, false, true>(v, reinterpret_cast<C *const(&)[NL]>(ln), t, tr,
                                                  RowSync<T>{1 + rr});
    __syncthreads();  // every row is done with its lines: the region becomes the tile
#pragma unroll
    for (int l = 0; l < NL; ++l)
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) R[(size_t(l) * LX + t + mm * T) * RP + rr] = v[l][mm];
    __syncthreads();
    C *Tc = Tb + size_t(c0) * LX * nz;
    for (int idx = threadIdx.x; idx < NL * LX * ROWS; idx += kTileThreads) {
      const int r = idx % ROWS, ck = idx / ROWS;  // ck = l * LX + kx
      if (z0 + r < nz) Tc[size_t(ck) * nz + z0 + r] = R[size_t(ck) * RP + r];
    }
    __syncthreads();  // the tile has been stored before the next lines overwrite it
  };
  pass.template operator()<2>(0);
  pass.template operator()<2>(2);
  pass.template operator()<1>(4);
}

// For CC columns kx: the sources' columns (two at a time in complex64), forward FFT along z, times their two
// kernel entries, summed into the two outputs; inverse FFT of the sums; keep z < nz ->
// T2[slot][i][kx][z].
// Lines per forward column FFT: complex64 may pair the sources (two CTAs per SM either way);
// complex128 transforms one line at a time (two would not fit in the register file).
#ifndef DBI_KCOLS_LINES
#define DBI_KCOLS_LINES 2
#endif
template <typename C> constexpr int kKColsLines = sizeof(C) == 8 ? DBI_KCOLS_LINES : 1;

template <typename C, int LZ>
__global__ void __launch_bounds__(kTileThreads, sizeof(C) == 8 ? 2 : 1) kk_cols(KP<C> p) {
  using CF = ColCfg<C, LZ>;
  constexpr int CC = CF::CC, T = CF::T, LP = CF::LP;
  const int b = kproblem(p), f = p.fidx[b], slot = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  const int col = threadIdx.x / T, t = threadIdx.x - col * T;
  const int kx = blockIdx.x * CC + col, nz = p.nz, lx = p.lx;
  const bool live = kx < lx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *smem = reinterpret_cast<C *>(smem_raw);
  const TwReg<C, LZ> tr(t, p.tw);
  const size_t plane = size_t(lx) * LZ;
  const C *G = p.Ghat + size_t(f) * 3 * plane + size_t(kx) * LZ;
  const C *D = p.Dhat + size_t(f) * 6 * plane + size_t(kx) * LZ;
  // kernel entries (first row, second row) of each source
  const C *e0[5] = {G, G + plane, D, D + 2 * plane, D + 4 * plane};
  const C *e1[5] = {G + plane, G + 2 * plane, D + plane, D + 3 * plane, D + 5 * plane};
  C acc[2][8];
#pragma unroll
  for (int mm = 0; mm < 8; ++mm) acc[0][mm] = acc[1][mm] = czero<C>();
  const C *Tb = p.T5 + size_t(slot) * 5 * lx * nz;
  C *const lines[2] = {smem + size_t(col) * LP, smem + size_t(CC + col) * LP};
  auto pass = [&]<int NL>(int c0) {
    C v[NL][8];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const C *src = Tb + (size_t(c0 + l) * lx + kx) * nz;
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) {
        const int z = t + mm * T;
        v[l][mm] = (mm < kHalf && live && z < nz) ? src[z] : czero<C>();
      }
    }
    RegPlan<LZ>::template run<C, NL, false, true>(v, reinterpret_cast<C *const(&)[NL]>(lines), t, tr,
                                                  RowSync<T>{1 + col});
    if (live) {
#pragma unroll
      for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int mm = 0; mm < 8; ++mm) {
          const int kz = t + mm * T;
          acc[0][mm] = cadd(acc[0][mm], cmul(__ldg(e0[c0 + l] + kz), v[l][mm]));
          acc[1][mm] = cadd(acc[1][mm], cmul(__ldg(e1[c0 + l] + kz), v[l][mm]));
        }
    }
  };
  if constexpr (kKColsLines<C> == 2) {
    pass.template operator()<2>(0);
    pass.template operator()<2>(2);
    pass.template operator()<1>(4);
  } else {
#pragma unroll 1
    for (int c = 0; c < 5; ++c) {
      const C *src = Tb + (size_t(c) * lx + kx) * nz;
      C v[1][8];
#pragma unroll
      for (int mm = 0; mm < 8; ++mm) {
        const int z = t + mm * T;
        v[0][mm] = (mm < kHalf && live && z < nz) ? src[z] : czero<C>();
      }
      C *const ln[1] = {lines[0]};
      RegPlan<LZ>::template run<C, 1, false, true>(v, ln, t, tr, RowSync<T>{1 + col});
      if (live) {
#pragma unroll
        for (int mm = 0; mm < 8; ++mm) {
          const int kz = t + mm * T;
          acc[0][mm] = cadd(acc[0][mm], cmul(__ldg(e0[c] + kz), v[0][mm]));
          acc[1][mm] = cadd(acc[1][mm], cmul(__ldg(e1[c] + kz), v[0][mm]));
        }
      }
    }
  }
  RegPlan<LZ>::template run<C, 2, true>(acc, lines, t, tr, RowSync<T>{1 + col});
  if (live) {
    C *o = p.T2 + size_t(slot) * 2 * lx * nz;
#pragma unroll
    for (int mm = 0; mm < kHalf; ++mm) {
      const int z = t + mm * T;
      if (z < nz) {
        o[size_t(kx) * nz + z] = acc[0][mm];
        o[(size_t(lx) + kx) * nz + z] = acc[1][mm];
      }
    }
  }
}

template <typename C, int LX, int EPI>
__global__ void __launch_bounds__(kTileThreads) kk_rows_inverse(KP<C> p) {
  const int b = kproblem(p), f = p.fidx[b];
  if ((p.active && !p.active[b]) || unsigned(f) >= unsigned(p.nf)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_inverse_tile<C, LX, EPI, 0>(KTile<C>{p, b, int(blockIdx.y), f}, blockIdx.x, reinterpret_cast<C *>(smem_raw));
}

template <typename C> static int run_k_typed(const OpArgs &a, cudaStream_t s) {
  using Rl = typename RealOf<C>::type;
  const int nb = a.plist ? a.nb : a.B;
  if (nb <= 0) return DBI_OK;
  KP<C> p;
  p.nz = a.nz; p.nx = a.nx; p.lz = a.lz; p.lx = a.lx; p.nf = a.nf;
  p.inv2h = Rl(1.0 / (2.0 * a.h));
  p.omega = a.omega; p.fidx = a.fidx;
  p.m = static_cast<const Rl *>(a.m);
  for (int i = 0; i < 5; ++i) p.ref[i] = Rl(a.ref[i]);
  p.in = static_cast<const C *>(a.in);
  p.ident = static_cast<const C *>(a.ident);
  p.out = static_cast<C *>(a.out);
  p.T5 = static_cast<C *>(a.T);
  p.T2 = p.T5 + size_t(a.B) * 5 * a.lx * a.nz;
  p.Ghat = static_cast<const C *>(a.Ghat);
  p.Dhat = static_cast<const C *>(a.Dhat);
  p.tw = static_cast<const C *>(a.tw);
  p.active = a.active;
  p.plist = a.plist;
  p.s0 = 0;
  p.in_scale = a.in_scale; p.m_scale = a.m_scale; p.out_scale = a.out_scale;
  p.krhat = static_cast<const C *>(a.krhat);
  p.part_out = a.part_out;
  p.part_count = operator_parts_k(a.nz, a.lx, a.precision);
  int rc = DBI_OK;
  prof_mark(PROF_OPERATOR, false, s);
  prof_mark(PROF_ROWS_FORWARD, false, s);
  dispatch_len(a.lx, [&]<int LX>() {
    using RC = RowCfg<C, LX>;
    const size_t bytes = kk_rows_forward_smem<C, LX>(a.nx);
    const dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, nb);
    cudaError_t e = allow_smem(kk_rows_forward<C, LX>, bytes);
    if (e == cudaSuccess) kk_rows_forward<C, LX><<<grid, kTileThreads, bytes, s>>>(p);
    rc = e != cudaSuccess ? cuda_fail("kk_rows_forward smem", e) : check_launch("kk_rows_forward");
  });
  prof_mark(PROF_ROWS_FORWARD, true, s);
  if (rc) return rc;
  prof_mark(PROF_COLS, false, s);
  dispatch_len(a.lz, [&]<int LZ>() {
    using CF = ColCfg<C, LZ>;
    const size_t bytes = cols_smem<C, LZ>();
    const dim3 grid((a.lx + CF::CC - 1) / CF::CC, nb);
    cudaError_t e = allow_smem(kk_cols<C, LZ>, bytes);
    if (e == cudaSuccess) kk_cols<C, LZ><<<grid, kTileThreads, bytes, s>>>(p);
    rc = e != cudaSuccess ? cuda_fail("kk_cols smem", e) : check_launch("kk_cols");
  });
  prof_mark(PROF_COLS, true, s);
  if (rc) return rc;
  prof_mark(PROF_ROWS_INVERSE, false, s);
  dispatch_len(a.lx, [&]<int LX>() {
    using RC = RowCfg<C, LX>;
    const size_t bytes = rows_inverse_smem<C, LX>();
    const dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, nb);
    cudaError_t e;
    auto launch = [&](auto kernel) {
      e = allow_smem(kernel, bytes);
      if (e == cudaSuccess) kernel<<<grid, kTileThreads, bytes, s>>>(p);
    };
    if (a.epi == 1) launch(kk_rows_inverse<C, LX, 1>);
    else if (a.epi == 2) launch(kk_rows_inverse<C, LX, 2>);
    else launch(kk_rows_inverse<C, LX, 0>);
    rc = e != cudaSuccess ? cuda_fail("kk_rows_inverse smem", e) : check_launch("kk_rows_inverse");
  });
  prof_mark(PROF_ROWS_INVERSE, true, s);
  prof_mark(PROF_OPERATOR, true, s);
  return rc;
}

int run_form_k(const OpArgs &a, cudaStream_t s) {
  return a.precision == DBI_C64 ? run_k_typed<float2>(a, s) : run_k_typed<double2>(a, s);
}

}  // namespace dbi

using namespace dbi;

static int check_k(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *Dhat,
                   const void *in, const void *out, int precision, void *work, size_t work_bytes, int op) {
  int rc;
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  if ((rc = check_grid(&model->grid)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (batch->B > 0 && (!Ghat || !Dhat || !in || !out || !model->m)) {
    set_error("NULL model->m, Ghat, Dhat, input or output");
    return DBI_ERR_ARG;
  }
  if (in == out && batch->B > 0) { set_error("input and output must be distinct buffers"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes(&model->grid, batch->B, precision, op);
  if (batch->B > 0 && (!work || work_bytes < need)) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  return DBI_OK;
}

static OpArgs k_args(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *Dhat,
                     int precision, void *T, void *tw) {
  const dbi_grid *g = &model->grid;
  OpArgs a{};
  a.precision = precision; a.nz = g->nz; a.nx = g->nx; a.lz = g->lz; a.lx = g->lx; a.h = g->h;
  a.B = batch->B; a.nf = batch->nf; a.omega = batch->omega; a.fidx = batch->fidx;
  a.m = model->m; reference_values(model->ref, a.ref);
  a.stencil = true; a.T = T; a.Ghat = Ghat; a.Dhat = Dhat; a.tw = tw;
  return a;
}

extern "C" int ls_apply_k(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *Dhat,
                          const void *u, void *out, int precision, void *work, size_t work_bytes,
                          dbi_stream stream) {
  clear_error();
  int rc = check_k(model, batch, Ghat, Dhat, u, out, precision, work, work_bytes, DBI_OP_APPLY_K);
  if (rc || batch->B == 0) return rc;
  const dbi_grid *g = &model->grid;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral_k(g, batch->B, precision));
  Scales sc = carve_scales(ar, batch->B);
  if ((rc = ar.check("ls_apply_k"))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  if ((rc = pow2_scales(u, precision, false, batch->B, size_t(2) * g->nz * g->nx, sc.part, sc.scale, sc.inv,
                        nullptr, s)))
    return rc;
  OpArgs a = k_args(model, batch, Ghat, Dhat, precision, T, tw);
  a.in = u; a.ident = u; a.out = out;
  a.in_scale = sc.scale; a.out_scale = sc.inv;
  return run_operator(a, s);
}

extern "C" int ls_solve_k(const dbi_model *model, const dbi_batch *batch, const void *Ghat, const void *Dhat,
                          const void *rhs, void *u, const dbi_krylov_opts *opts, const dbi_status *status,
                          int precision, void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_k(model, batch, Ghat, Dhat, rhs, u, precision, work, work_bytes, DBI_OP_SOLVE_K);
  if (rc || (rc = check_krylov(opts)) || batch->B == 0) return rc;
  const dbi_grid *g = &model->grid;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  void *tw = ar.take(bytes_twiddles(precision));
  void *T = ar.take(bytes_spectral_k(g, batch->B, precision));
  SolverBufs sb = carve_solver(ar, g, batch->B, precision);
  if ((rc = ar.check("ls_solve_k"))) return rc;
  if ((rc = launch_twiddles(tw, precision, s))) return rc;
  OpArgs a = k_args(model, batch, Ghat, Dhat, precision, T, tw);
  return run_bicgstab(a, sb, rhs, u, opts->zero_guess != 0, *opts, status, s, true);
}

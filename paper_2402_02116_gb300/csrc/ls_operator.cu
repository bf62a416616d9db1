// The batched LS operator A u = u - h^2 G * (w^2 drho u + div(dC : eps(u))) (Eq. 6, 10) and the
// plain Green's convolution, both evaluated by Eq. 12 on the zero-padded lz x lx grid as three
// kernels per batch:
//   k_rows_forward : contrast source by central differences (fields zero outside D) for a few rows,
//                    zero-pad each row to lx, forward FFT along x  -> T[b][c][z][kx]   (z < nz)
//   k_cols         : for a tile of kx columns, forward FFT along z of the nz non-zero rows padded
//                    to lz, 2x2 multiply by Ghat(kz, kx), inverse FFT along z, keep z < nz -> T
//   k_rows_inverse : inverse FFT along x, keep x < nx, out = ident - result (or the result).
// Ghat already carries h^2 / (lz lx), so no other scaling is applied.
#include "fft.cuh"
#include "operator.cuh"

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
  const double *in_scale, *m_scale, *out_scale;
};

// Elements of one CTA's line buffer and values per thread in the FFT passes.
template <typename C> struct Cfg;
template <> struct Cfg<float2> { static constexpr int rowElems = 4096, colElems = 8192, vpt = 16; };
template <> struct Cfg<double2> { static constexpr int rowElems = 2048, colElems = 4096, vpt = 8; };

template <typename C, int LX> struct RowCfg {
  static constexpr int ROWS = Cfg<C>::rowElems / (2 * LX) > 0 ? Cfg<C>::rowElems / (2 * LX) : 1;
  static constexpr int NT = 2 * ROWS * LX / Cfg<C>::vpt;
  static constexpr int LS = LX + 1;
};
template <typename C, int LZ> struct ColCfg {
  static constexpr int CCr = Cfg<C>::colElems / (2 * LZ);
  static constexpr int CC = CCr > 64 ? 64 : (CCr > 0 ? CCr : 1);
  static constexpr int NT = 2 * CC * LZ / Cfg<C>::vpt;
  static constexpr int LS = LZ + 1;
};

// Stress sigma = dC eps at cell (z, x) of D from the staged u; zero outside D.
template <typename C>
__device__ __forceinline__ void stress_at(const OpP<C> &p, const C *su, int W, int RS, int z0, int z,
                                          int x, typename RealOf<C>::type ms, C &s1, C &s3, C &s5) {
  using Rl = typename RealOf<C>::type;
  if (z < 0 || z >= p.nz || x < 0 || x >= p.nx) {
    s1 = s3 = s5 = czero<C>();
    return;
  }
  // su[c][rr][xx]: rr = z - (z0 - 2), xx = x + 1
  auto U = [&](int c, int zz, int xx) { return su[(c * RS + (zz - z0 + 2)) * W + xx + 1]; };
  const C e1 = cscale(csub(U(0, z, x + 1), U(0, z, x - 1)), p.inv2h);
  const C e3 = cscale(csub(U(1, z + 1, x), U(1, z - 1, x)), p.inv2h);
  const C e5 = cscale(cadd(csub(U(0, z + 1, x), U(0, z - 1, x)), csub(U(1, z, x + 1), U(1, z, x - 1))), p.inv2h);
  const size_t cell = size_t(z) * p.nx + x, plane = size_t(p.nz) * p.nx;
  const Rl d11 = (p.m[1 * plane + cell] - p.ref[1]) * ms;
  const Rl d13 = (p.m[2 * plane + cell] - p.ref[2]) * ms;
  const Rl d33 = (p.m[3 * plane + cell] - p.ref[3]) * ms;
  const Rl d55 = (p.m[4 * plane + cell] - p.ref[4]) * ms;
  s1 = cadd(cscale(e1, d11), cscale(e3, d13));
  s3 = cadd(cscale(e1, d13), cscale(e3, d33));
  s5 = cscale(e5, d55);
}

template <typename C, int LX, bool STENCIL>
__global__ void __launch_bounds__(RowCfg<C, LX>::NT) k_rows_forward(OpP<C> p) {
  using Rl = typename RealOf<C>::type;
  constexpr int ROWS = RowCfg<C, LX>::ROWS, NT = RowCfg<C, LX>::NT, LS = RowCfg<C, LX>::LS;
  const int b = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(p.fidx[b]) >= unsigned(p.nf)) return;
  const int z0 = blockIdx.x * ROWS;
  const int nz = p.nz, nx = p.nx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *lines = reinterpret_cast<C *>(smem_raw);  // [2 ROWS][LS], line = c * ROWS + rr
  const C *in = p.in + size_t(b) * 2 * nz * nx;
  const Rl isc = p.in_scale ? Rl(p.in_scale[b]) : Rl(1);

  if constexpr (STENCIL) {
    constexpr int RS = ROWS + 4;
    const int W = nx + 2;
    C *su = lines + 2 * ROWS * LS;  // [2][ROWS + 4][nx + 2]
    for (int idx = threadIdx.x; idx < 2 * RS * W; idx += NT) {
      const int c = idx / (RS * W), rem = idx - c * RS * W;
      const int rr = rem / W, xx = rem - rr * W - 1, z = z0 - 2 + rr;
      su[idx] = (z >= 0 && z < nz && xx >= 0 && xx < nx) ? cscale(in[(size_t(c) * nz + z) * nx + xx], isc)
                                                          : czero<C>();
    }
    __syncthreads();
    const double om = p.omega[p.fidx[b]];
    const Rl ms = p.m_scale ? Rl(p.m_scale[0]) : Rl(1);
    const Rl w2 = Rl(om * om);
    for (int idx = threadIdx.x; idx < ROWS * LX; idx += NT) {
      const int rr = idx / LX, x = idx - rr * LX, z = z0 + rr;
      C o1 = czero<C>(), o3 = czero<C>();
      if (z < nz && x < nx) {
        C a1, a3, a5, b1, b3, b5;
        const size_t cell = size_t(z) * nx + x;
        const Rl drho = (p.m[cell] - p.ref[0]) * ms;
        const C u1 = su[(0 * RS + rr + 2) * W + x + 1];
        const C u3 = su[(1 * RS + rr + 2) * W + x + 1];
        // d/dx1 terms: sigma at (z, x +- 1)
        stress_at(p, su, W, RS, z0, z, x + 1, ms, a1, a3, a5);
        stress_at(p, su, W, RS, z0, z, x - 1, ms, b1, b3, b5);
        o1 = cscale(csub(a1, b1), p.inv2h);  // d1 sigma1
        o3 = cscale(csub(a5, b5), p.inv2h);  // d1 sigma5
        // d/dx3 terms: sigma at (z +- 1, x)
        stress_at(p, su, W, RS, z0, z + 1, x, ms, a1, a3, a5);
        stress_at(p, su, W, RS, z0, z - 1, x, ms, b1, b3, b5);
        o1 = cadd(o1, cscale(csub(a5, b5), p.inv2h));  // d3 sigma5
        o3 = cadd(o3, cscale(csub(a3, b3), p.inv2h));  // d3 sigma3
        o1 = cadd(o1, cscale(u1, w2 * drho));
        o3 = cadd(o3, cscale(u3, w2 * drho));
      }
      lines[rr * LS + x] = o1;
      lines[(ROWS + rr) * LS + x] = o3;
    }
  } else {
    for (int idx = threadIdx.x; idx < 2 * ROWS * LX; idx += NT) {
      const int c = idx / (ROWS * LX), rem = idx - c * ROWS * LX;
      const int rr = rem / LX, x = rem - rr * LX, z = z0 + rr;
      lines[(c * ROWS + rr) * LS + x] =
          (z < nz && x < nx) ? cscale(in[(size_t(c) * nz + z) * nx + x], isc) : czero<C>();
    }
  }
  __syncthreads();
  Plan<LX>::template run<C, 2 * ROWS, LS, NT, false>(lines, p.tw);
  C *T = p.T + size_t(b) * 2 * nz * LX;
  for (int idx = threadIdx.x; idx < 2 * ROWS * LX; idx += NT) {
    const int c = idx / (ROWS * LX), rem = idx - c * ROWS * LX;
    const int rr = rem / LX, x = rem - rr * LX, z = z0 + rr;
    if (z < nz) T[(size_t(c) * nz + z) * LX + x] = lines[(c * ROWS + rr) * LS + x];
  }
}

template <typename C, int LZ>
__global__ void __launch_bounds__(ColCfg<C, LZ>::NT) k_cols(OpP<C> p) {
  constexpr int CC = ColCfg<C, LZ>::CC, NT = ColCfg<C, LZ>::NT, LS = ColCfg<C, LZ>::LS;
  const int b = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(p.fidx[b]) >= unsigned(p.nf)) return;
  const int kx0 = blockIdx.x * CC;
  const int nz = p.nz, lx = p.lx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *lines = reinterpret_cast<C *>(smem_raw);  // [2 CC][LS], line = c * CC + j
  C *T = p.T + size_t(b) * 2 * nz * lx;
  for (int idx = threadIdx.x; idx < 2 * CC * LZ; idx += NT) {
    const int c = idx / (CC * LZ), rem = idx - c * CC * LZ;
    const int z = rem / CC, j = rem - z * CC, kx = kx0 + j;
    lines[(c * CC + j) * LS + z] = (z < nz && kx < lx) ? T[(size_t(c) * nz + z) * lx + kx] : czero<C>();
  }
  __syncthreads();
  Plan<LZ>::template run<C, 2 * CC, LS, NT, false>(lines, p.tw);
  const C *G = p.Ghat + size_t(p.fidx[b]) * 3 * LZ * lx;
  for (int idx = threadIdx.x; idx < CC * LZ; idx += NT) {
    const int kz = idx / CC, j = idx - kz * CC, kx = kx0 + j;
    if (kx < lx) {
      const C g11 = G[(size_t(0) * LZ + kz) * lx + kx];
      const C g13 = G[(size_t(1) * LZ + kz) * lx + kx];
      const C g33 = G[(size_t(2) * LZ + kz) * lx + kx];
      const C s1 = lines[j * LS + kz], s3 = lines[(CC + j) * LS + kz];
      lines[j * LS + kz] = cadd(cmul(g11, s1), cmul(g13, s3));
      lines[(CC + j) * LS + kz] = cadd(cmul(g13, s1), cmul(g33, s3));
    }
  }
  __syncthreads();
  Plan<LZ>::template run<C, 2 * CC, LS, NT, true>(lines, p.tw);
  for (int idx = threadIdx.x; idx < 2 * CC * LZ; idx += NT) {
    const int c = idx / (CC * LZ), rem = idx - c * CC * LZ;
    const int z = rem / CC, j = rem - z * CC, kx = kx0 + j;
    if (z < nz && kx < lx) T[(size_t(c) * nz + z) * lx + kx] = lines[(c * CC + j) * LS + z];
  }
}

template <typename C, int LX>
__global__ void __launch_bounds__(RowCfg<C, LX>::NT) k_rows_inverse(OpP<C> p) {
  constexpr int ROWS = RowCfg<C, LX>::ROWS, NT = RowCfg<C, LX>::NT, LS = RowCfg<C, LX>::LS;
  const int b = blockIdx.y;
  if ((p.active && !p.active[b]) || unsigned(p.fidx[b]) >= unsigned(p.nf)) return;
  const int z0 = blockIdx.x * ROWS;
  const int nz = p.nz, nx = p.nx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *lines = reinterpret_cast<C *>(smem_raw);
  const C *T = p.T + size_t(b) * 2 * nz * LX;
  for (int idx = threadIdx.x; idx < 2 * ROWS * LX; idx += NT) {
    const int c = idx / (ROWS * LX), rem = idx - c * ROWS * LX;
    const int rr = rem / LX, x = rem - rr * LX, z = z0 + rr;
    lines[(c * ROWS + rr) * LS + x] = z < nz ? T[(size_t(c) * nz + z) * LX + x] : czero<C>();
  }
  __syncthreads();
  Plan<LX>::template run<C, 2 * ROWS, LS, NT, true>(lines, p.tw);
  const size_t base = size_t(b) * 2 * nz * nx;
  using Rl = typename RealOf<C>::type;
  const Rl osc = p.out_scale ? Rl(p.out_scale[b]) : Rl(1);
  for (int idx = threadIdx.x; idx < 2 * ROWS * nx; idx += NT) {
    const int c = idx / (ROWS * nx), rem = idx - c * ROWS * nx;
    const int rr = rem / nx, x = rem - rr * nx, z = z0 + rr;
    if (z < nz) {
      const size_t o = base + (size_t(c) * nz + z) * nx + x;
      const C v = cscale(lines[(c * ROWS + rr) * LS + x], osc);
      p.out[o] = p.ident ? csub(p.ident[o], v) : v;
    }
  }
}

// Opt a kernel into more than 48 KB of dynamic shared memory once per device.
template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

template <typename C> static int run_typed(const OpArgs &a, cudaStream_t s) {
  using Rl = typename RealOf<C>::type;
  if (a.B == 0) return DBI_OK;
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
  p.in_scale = a.in_scale; p.m_scale = a.m_scale; p.out_scale = a.out_scale;
  int rc = DBI_OK;
  const bool stencil = a.stencil;
  prof_mark(PROF_OPERATOR, false, s);
  prof_mark(PROF_ROWS_FORWARD, false, s);
  dispatch_len(a.lx, [&]<int LX>() {
    using RC = RowCfg<C, LX>;
    const size_t lines = size_t(2) * RC::ROWS * RC::LS * sizeof(C);
    const size_t su = stencil ? size_t(2) * (RC::ROWS + 4) * (a.nx + 2) * sizeof(C) : 0;
    dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, a.B);
    cudaError_t e;
    if (stencil) {
      e = allow_smem(k_rows_forward<C, LX, true>, lines + su);
      if (e == cudaSuccess) k_rows_forward<C, LX, true><<<grid, RC::NT, lines + su, s>>>(p);
    } else {
      e = allow_smem(k_rows_forward<C, LX, false>, lines);
      if (e == cudaSuccess) k_rows_forward<C, LX, false><<<grid, RC::NT, lines, s>>>(p);
    }
    rc = e != cudaSuccess ? cuda_fail("k_rows_forward smem", e) : check_launch("k_rows_forward");
  });
  prof_mark(PROF_ROWS_FORWARD, true, s);
  if (rc) return rc;
  prof_mark(PROF_COLS, false, s);
  dispatch_len(a.lz, [&]<int LZ>() {
    using CCfg = ColCfg<C, LZ>;
    const size_t bytes = size_t(2) * CCfg::CC * CCfg::LS * sizeof(C);
    dim3 grid((a.lx + CCfg::CC - 1) / CCfg::CC, a.B);
    cudaError_t e = allow_smem(k_cols<C, LZ>, bytes);
    if (e == cudaSuccess) k_cols<C, LZ><<<grid, CCfg::NT, bytes, s>>>(p);
    rc = e != cudaSuccess ? cuda_fail("k_cols smem", e) : check_launch("k_cols");
  });
  prof_mark(PROF_COLS, true, s);
  if (rc) return rc;
  prof_mark(PROF_ROWS_INVERSE, false, s);
  dispatch_len(a.lx, [&]<int LX>() {
    using RC = RowCfg<C, LX>;
    const size_t bytes = size_t(2) * RC::ROWS * RC::LS * sizeof(C);
    dim3 grid((a.nz + RC::ROWS - 1) / RC::ROWS, a.B);
    cudaError_t e = allow_smem(k_rows_inverse<C, LX>, bytes);
    if (e == cudaSuccess) k_rows_inverse<C, LX><<<grid, RC::NT, bytes, s>>>(p);
    rc = e != cudaSuccess ? cuda_fail("k_rows_inverse smem", e) : check_launch("k_rows_inverse");
  });
  prof_mark(PROF_ROWS_INVERSE, true, s);
  prof_mark(PROF_OPERATOR, true, s);
  return rc;
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

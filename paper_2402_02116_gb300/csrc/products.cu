// Matrix-free distorted-Born products (Eq. 20, 25-35), the L2 data residual and the Tikhonov
// normal-equation CG (Eq. 23, 24).
//
// Frechet:  d = P A_b^{-1} K s_dm,  s_dm = w^2 dm_rho u_b + div(dC(dm) : eps(u_b))
//           (the operator's stencil with dm as the contrast and no identity term; Y and M of
//           Eq. 26 in one source by linearity), then one background solve and receiver sampling.
// Adjoint:  u_a = A_b^{-1} K P^T conj(r)  (conj(r) injected at the receivers, Eq. 33-35), then
//           g_rho = sum_b Re(w^2 u_a . u_b), g_p = -sum_b Re(eps(u_a)^T B_p eps(u_b)) with the
//           Appendix C matrices restricted to Voigt {1, 3, 5}: B11 = e1 e1^T, B33 = e3 e3^T,
//           B55 = e5 e5^T, B13 = e1 e3^T + e3 e1^T (B66 has no 2D part).
#include <algorithm>
#include <cmath>
#include <vector>

#include "krylov.cuh"
#include "mspace.cuh"

namespace dbi {


// ----------------------------------------------------------------------------------------------
// receivers
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ bool rec_ok(const int *cells, int k, int nz, int nx, int &iz, int &ix) {
  iz = cells[2 * k];
  ix = cells[2 * k + 1];
  return iz >= 0 && iz < nz && ix >= 0 && ix < nx;
}

// d = fac[b] * P u, the factor applied in FP64
template <typename C>
__global__ void k_sample(int B, int nrec, int nz, int nx, const int *cells, const C *u, const double *fac, C *d) {
  using R = typename RealOf<C>::type;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (k >= nrec) return;
  int iz, ix;
  const bool ok = rec_ok(cells, k, nz, nx, iz, ix);
  const size_t base = size_t(b) * 2 * nz * nx;
  const double f = fac[b];
  for (int c = 0; c < 2; ++c) {
    const C v = ok ? u[base + (size_t(c) * nz + iz) * nx + ix] : czero<C>();
    d[(size_t(b) * nrec + k) * 2 + c] = mk<C>(R(double(v.x) * f), R(double(v.y) * f));
  }
}

template <typename C>
__global__ void k_zero(size_t n, C *x) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    x[i] = czero<C>();
}

// q = P^T conj(r): one thread per (problem, component) adds the receivers in order.
template <typename C>
__global__ void k_inject_conj(int B, int nrec, int nz, int nx, const int *cells, const C *r, C *q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * B) return;
  const int b = t >> 1, c = t & 1;
  C *qb = q + size_t(b) * 2 * nz * nx + size_t(c) * nz * nx;
  for (int k = 0; k < nrec; ++k) {
    int iz, ix;
    if (!rec_ok(cells, k, nz, nx, iz, ix)) continue;
    const C v = r[(size_t(b) * nrec + k) * 2 + c];
    qb[size_t(iz) * nx + ix] = cadd(qb[size_t(iz) * nx + ix], cconj(v));
  }
}

// ----------------------------------------------------------------------------------------------
// imaging condition (Eq. 32, real part), FP64 accumulation over the problems
// ----------------------------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ C at(const C *u, int nz, int nx, int z, int x) {
  return (z >= 0 && z < nz && x >= 0 && x < nx) ? u[size_t(z) * nx + x] : czero<C>();
}

template <typename C>
__device__ __forceinline__ void strain(const C *u1, const C *u3, int nz, int nx, int z, int x,
                                       typename RealOf<C>::type inv2h, C &e1, C &e3, C &e5) {
  e1 = cscale(csub(at(u1, nz, nx, z, x + 1), at(u1, nz, nx, z, x - 1)), inv2h);
  e3 = cscale(csub(at(u3, nz, nx, z + 1, x), at(u3, nz, nx, z - 1, x)), inv2h);
  e5 = cscale(cadd(csub(at(u1, nz, nx, z + 1, x), at(u1, nz, nx, z - 1, x)),
                   csub(at(u3, nz, nx, z, x + 1), at(u3, nz, nx, z, x - 1))), inv2h);
}

// Partial images of the problems [c * pb, min(B, (c + 1) * pb)) for chunk c = blockIdx.z, FP64.
// u_a is stored as src_scale[b] * st[b].scale * (the back-propagated field) and u_b is read times
// ub_scale[b] (powers of two bringing both near unit norm), so the strain products are formed in
// FP32 without underflow and accumulated in FP64 with the exact factor 1 / (all three scales).
template <typename C>
__global__ void k_imaging_part(int B, int pb, int nf, int nz, int nx, double h, const double *omega,
                               const int *fidx, const C *ua, const C *ub, const double *src_scale,
                               const KState *st, const double *ub_scale, double *part) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  if (x >= nx) return;
  const R inv2h = R(1.0 / (2.0 * h));
  const size_t plane = size_t(nz) * nx, cell = size_t(z) * nx + x;
  double g0 = 0, g1 = 0, g2 = 0, g3 = 0, g4 = 0;
  const int b1e = min(B, (int(blockIdx.z) + 1) * pb);
  for (int b = blockIdx.z * pb; b < b1e; ++b) {
    if (unsigned(fidx[b]) >= unsigned(nf)) continue;
    const C *a1 = ua + size_t(b) * 2 * plane, *a3 = a1 + plane;
    const C *c1 = ub + size_t(b) * 2 * plane, *c3 = c1 + plane;
    const R us = R(ub_scale[b]);
    const double w = omega[fidx[b]];
    const double f = 1.0 / (src_scale[b] * st[b].scale * ub_scale[b]);
    C ea1, ea3, ea5, eb1, eb3, eb5;
    strain(a1, a3, nz, nx, z, x, inv2h, ea1, ea3, ea5);
    strain(c1, c3, nz, nx, z, x, R(inv2h * us), eb1, eb3, eb5);
    const C pa1 = a1[cell], pa3 = a3[cell], pb1 = cscale(c1[cell], us), pb3 = cscale(c3[cell], us);
    const R rho_t = cmul(pa1, pb1).x + cmul(pa3, pb3).x;
    const R t11 = cmul(ea1, eb1).x;
    const R t13 = cmul(ea1, eb3).x + cmul(ea3, eb1).x;
    const R t33 = cmul(ea3, eb3).x;
    const R t55 = cmul(ea5, eb5).x;
    g0 += f * w * w * double(rho_t);
    g1 -= f * double(t11);
    g2 -= f * double(t13);
    g3 -= f * double(t33);
    g4 -= f * double(t55);
  }
  double *o = part + size_t(blockIdx.z) * 5 * plane + cell;
  o[0] = g0;
  o[plane] = g1;
  o[2 * plane] = g2;
  o[3 * plane] = g3;
  o[4 * plane] = g4;
}

// g = sum of the chunks' partial images, in chunk order.
template <typename GOut>
__global__ void k_imaging_sum(size_t n, int nch, const double *part, GOut *g) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    double a = 0.0;
    for (int c = 0; c < nch; ++c) a += part[size_t(c) * n + i];
    g[i] = GOut(a);
  }
}

// ----------------------------------------------------------------------------------------------
// data residual r = P u - d_obs and phi = 1/2 sum |r|^2 (one CTA, fixed summation order)
// ----------------------------------------------------------------------------------------------
template <typename C>
__global__ void k_residual(int B, int nrec, int nz, int nx, const int *cells, const C *u, const C *dobs,
                           C *r, double *phi) {
  __shared__ double sh[32];
  double acc = 0.0;
  const int total = B * nrec;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = t / nrec, k = t - b * nrec;
    int iz, ix;
    const bool ok = rec_ok(cells, k, nz, nx, iz, ix);
    for (int c = 0; c < 2; ++c) {
      const size_t o = (size_t(b) * nrec + k) * 2 + c;
      const C uv = ok ? u[size_t(b) * 2 * nz * nx + (size_t(c) * nz + iz) * nx + ix] : czero<C>();
      const C rv = csub(uv, dobs[o]);
      r[o] = rv;
      acc += double(rv.x) * double(rv.x) + double(rv.y) * double(rv.y);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && phi) {
    double s = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += sh[w];
    *phi = 0.5 * s;
  }
}

// ----------------------------------------------------------------------------------------------
// internal drivers
// ----------------------------------------------------------------------------------------------
struct ProdCtx {
  int precision;
  const dbi_grid *g;
  const dbi_batch *batch;
  const void *m_b;
  double ref[5];
  const void *Ghat;
  const void *tw;
  void *T;
  SolverBufs sb;
  void *f1, *f2;  // two fields [B][2][nz][nx]
  Scales sc;      // power-of-two normalisers of the convolution inputs
  double *img;    // [imaging_chunks(B)][5][nz][nx] FP64 partial images
  dbi_krylov_opts opts;
  const dbi_status *status;
  cudaStream_t s;
};

static OpArgs base_op(const ProdCtx &c) {
  OpArgs a{};
  a.precision = c.precision; a.nz = c.g->nz; a.nx = c.g->nx; a.lz = c.g->lz; a.lx = c.g->lx;
  a.h = c.g->h; a.B = c.batch->B; a.nf = c.batch->nf; a.omega = c.batch->omega; a.fidx = c.batch->fidx;
  a.T = c.T; a.Ghat = c.Ghat; a.tw = c.tw;
  return a;
}

static int solve_background(const ProdCtx &c, const void *rhs, void *x, bool unscale) {
  OpArgs a = base_op(c);
  a.m = c.m_b;
  for (int i = 0; i < 5; ++i) a.ref[i] = c.ref[i];
  return run_bicgstab(a, c.sb, rhs, x, true, c.opts, c.status, c.s, unscale);
}

// d = J dm (dm in the precision's real type). The source is built from u_b scaled by 2^k_b per
// problem and dm scaled by 2^k_m so that FP32 intermediates stay in range; the sampled data are
// multiplied back by 2^-(k_b + k_m) in FP64.
static int frechet_internal(const ProdCtx &c, const void *u_b, const dbi_receivers *rec, const void *dm, void *d) {
  int rc;
  const int B = c.batch->B;
  const size_t plane = size_t(c.g->nz) * c.g->nx;
  if ((rc = pow2_scales(dm, c.precision, true, 1, 5 * plane, c.sc.part, c.sc.mscale, nullptr, nullptr, c.s)))
    return rc;
  if ((rc = pow2_scales(u_b, c.precision, false, B, 2 * plane, c.sc.part, c.sc.scale, c.sc.inv, c.sc.mscale, c.s)))
    return rc;
  OpArgs a = base_op(c);
  a.m = dm;  // the perturbation plays the contrast; nothing to subtract
  a.stencil = true; a.in = u_b; a.ident = nullptr; a.out = c.f1;
  a.in_scale = c.sc.scale; a.m_scale = c.sc.mscale;
  if ((rc = run_operator(a, c.s))) return rc;
  if ((rc = solve_background(c, c.f1, c.f2, true))) return rc;
  dim3 grid((rec->n + 127) / 128, B);
  if (c.precision == DBI_C64)
    k_sample<float2><<<grid, 128, 0, c.s>>>(B, rec->n, c.g->nz, c.g->nx, rec->cells,
                                            static_cast<const float2 *>(c.f2), c.sc.inv, static_cast<float2 *>(d));
  else
    k_sample<double2><<<grid, 128, 0, c.s>>>(B, rec->n, c.g->nz, c.g->nx, rec->cells,
                                             static_cast<const double2 *>(c.f2), c.sc.inv, static_cast<double2 *>(d));
  return check_launch("k_sample");
}

// g = Re J^H r summed over problems; GOut = double (internal) or the precision's real type
template <typename GOut>
static int adjoint_internal(const ProdCtx &c, const void *u_b, const dbi_receivers *rec, const void *r, GOut *g) {
  int rc;
  const int B = c.batch->B, nz = c.g->nz, nx = c.g->nx;
  const size_t n = size_t(B) * 2 * nz * nx;
  const int zb = int(std::min<size_t>((n + 255) / 256, 8192));
  // q = P^T conj(r) in f2, then f1 = K q, then f2 = A_b^{-1} f1
  if (c.precision == DBI_C64) {
    k_zero<float2><<<zb, 256, 0, c.s>>>(n, static_cast<float2 *>(c.f2));
    if ((rc = check_launch("k_zero"))) return rc;
    k_inject_conj<float2><<<(2 * B + 127) / 128, 128, 0, c.s>>>(B, rec->n, nz, nx, rec->cells,
                                                                static_cast<const float2 *>(r), static_cast<float2 *>(c.f2));
  } else {
    k_zero<double2><<<zb, 256, 0, c.s>>>(n, static_cast<double2 *>(c.f2));
    if ((rc = check_launch("k_zero"))) return rc;
    k_inject_conj<double2><<<(2 * B + 127) / 128, 128, 0, c.s>>>(B, rec->n, nz, nx, rec->cells,
                                                                 static_cast<const double2 *>(r), static_cast<double2 *>(c.f2));
  }
  if ((rc = check_launch("k_inject_conj"))) return rc;
  // scale q by 2^k_b per problem; the solver keeps its own power-of-two scale on the solution,
  // and the imaging multiplies both back in FP64
  if ((rc = pow2_scales(c.f2, c.precision, false, B, size_t(2) * nz * nx, c.sc.part, c.sc.scale, nullptr,
                        nullptr, c.s)))
    return rc;
  OpArgs a = base_op(c);
  a.stencil = false; a.in = c.f2; a.ident = nullptr; a.out = c.f1;
  a.in_scale = c.sc.scale;
  if ((rc = run_operator(a, c.s))) return rc;
  if ((rc = solve_background(c, c.f1, c.f2, false))) return rc;
  // u_b normalised per problem for the FP32 strain products
  if ((rc = pow2_scales(u_b, c.precision, false, B, size_t(2) * nz * nx, c.sc.part, c.sc.aux, nullptr,
                        nullptr, c.s)))
    return rc;
  const int nch = imaging_chunks(B), pb = (B + nch - 1) / nch;
  dim3 grid((nx + 127) / 128, nz, nch);
  if (c.precision == DBI_C64)
    k_imaging_part<float2><<<grid, 128, 0, c.s>>>(B, pb, c.batch->nf, nz, nx, c.g->h, c.batch->omega,
                                                  c.batch->fidx, static_cast<const float2 *>(c.f2),
                                                  static_cast<const float2 *>(u_b), c.sc.scale, c.sb.st,
                                                  c.sc.aux, c.img);
  else
    k_imaging_part<double2><<<grid, 128, 0, c.s>>>(B, pb, c.batch->nf, nz, nx, c.g->h, c.batch->omega,
                                                   c.batch->fidx, static_cast<const double2 *>(c.f2),
                                                   static_cast<const double2 *>(u_b), c.sc.scale, c.sb.st,
                                                   c.sc.aux, c.img);
  if ((rc = check_launch("k_imaging_part"))) return rc;
  const size_t nm = size_t(5) * nz * nx;
  k_imaging_sum<GOut><<<int(std::min<size_t>((nm + 255) / 256, 4096)), 256, 0, c.s>>>(nm, nch, c.img, g);
  return check_launch("k_imaging_sum");
}

static int prepare(ProdCtx &c, Arena &ar, const dbi_model *bg, const dbi_batch *batch, const void *Ghat,
                   const dbi_krylov_opts *opts, const dbi_status *status, int precision, dbi_stream stream) {
  c.precision = precision;
  c.g = &bg->grid;
  c.batch = batch;
  c.m_b = bg->m;
  reference_values(bg->ref, c.ref);
  c.Ghat = Ghat;
  c.s = reinterpret_cast<cudaStream_t>(stream);
  c.tw = ar.take(bytes_twiddles(precision));
  c.T = ar.take(bytes_spectral(c.g, batch->B, precision));
  c.sb = carve_solver(ar, c.g, batch->B, precision);
  c.f1 = ar.take(bytes_field(c.g, batch->B, precision));
  c.f2 = ar.take(bytes_field(c.g, batch->B, precision));
  c.sc = carve_scales(ar, batch->B);
  c.img = static_cast<double *>(ar.take(size_t(imaging_chunks(batch->B)) * 5 * c.g->nz * c.g->nx * sizeof(double)));
  c.opts = *opts;
  c.status = status;
  if (const int rc = ar.check("distorted-Born products")) return rc;
  return launch_twiddles(const_cast<void *>(c.tw), precision, c.s);
}

static int check_products(const dbi_model *bg, const dbi_batch *batch, const void *Ghat, const void *u_b,
                          const dbi_receivers *rec, const void *in, const void *out,
                          const dbi_krylov_opts *opts, int precision, void *work, size_t work_bytes, int op) {
  int rc;
  if (!bg) { set_error("background model is NULL"); return DBI_ERR_ARG; }
  if ((rc = check_grid(&bg->grid, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision)) ||
      (rc = check_krylov(opts)))
    return rc;
  if (!rec || rec->n < 0 || (rec->n > 0 && !rec->cells)) { set_error("bad receivers"); return DBI_ERR_ARG; }
  if (batch->B > 0 && (!bg->m || !Ghat || !u_b || !in || !out)) {
    set_error("NULL background model, Ghat, u_b, input or output");
    return DBI_ERR_ARG;
  }
  const size_t need = dbi_workspace_bytes(&bg->grid, batch->B, precision, op);
  if (batch->B > 0 && (!work || work_bytes < need)) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  return DBI_OK;
}

}  // namespace dbi

using namespace dbi;

extern "C" int frechet_apply(const dbi_model *background, const dbi_batch *batch, const void *Ghat,
                             const void *u_b, const dbi_receivers *rec, const void *dm, void *d,
                             const dbi_krylov_opts *opts, const dbi_status *status, int precision,
                             void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_products(background, batch, Ghat, u_b, rec, dm, d, opts, precision, work, work_bytes,
                          DBI_OP_FRECHET);
  if (rc || batch->B == 0 || rec->n == 0) return rc;
  Arena ar(work, work_bytes);
  ProdCtx c;
  if ((rc = prepare(c, ar, background, batch, Ghat, opts, status, precision, stream))) return rc;
  return frechet_internal(c, u_b, rec, dm, d);
}

extern "C" int adjoint_apply(const dbi_model *background, const dbi_batch *batch, const void *Ghat,
                             const void *u_b, const dbi_receivers *rec, const void *r, void *g,
                             const dbi_krylov_opts *opts, const dbi_status *status, int precision,
                             void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_products(background, batch, Ghat, u_b, rec, r, g, opts, precision, work, work_bytes,
                          DBI_OP_ADJOINT);
  if (rc) return rc;
  if (batch->B == 0 || rec->n == 0) {
    const size_t bytes = size_t(5) * background->grid.nz * background->grid.nx *
                         (precision == DBI_C64 ? sizeof(float) : sizeof(double));
    cudaError_t e = cudaMemsetAsync(g, 0, bytes, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DBI_OK : cuda_fail("cudaMemsetAsync(g)", e);
  }
  Arena ar(work, work_bytes);
  ProdCtx c;
  if ((rc = prepare(c, ar, background, batch, Ghat, opts, status, precision, stream))) return rc;
  if (precision == DBI_C64) return adjoint_internal<float>(c, u_b, rec, r, static_cast<float *>(g));
  return adjoint_internal<double>(c, u_b, rec, r, static_cast<double *>(g));
}

extern "C" int data_residual(const dbi_grid *g, const dbi_batch *batch, const dbi_receivers *rec,
                             const void *u, const void *d_obs, void *r, double *phi, int precision,
                             dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid(g, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (!rec || rec->n < 0 || (rec->n > 0 && !rec->cells)) { set_error("bad receivers"); return DBI_ERR_ARG; }
  if (batch->B > 0 && rec->n > 0 && (!u || !d_obs || !r)) { set_error("NULL u, d_obs or r"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == DBI_C64)
    k_residual<float2><<<1, 1024, 0, s>>>(batch->B, rec->n, g->nz, g->nx, rec->cells,
                                          static_cast<const float2 *>(u), static_cast<const float2 *>(d_obs),
                                          static_cast<float2 *>(r), phi);
  else
    k_residual<double2><<<1, 1024, 0, s>>>(batch->B, rec->n, g->nz, g->nx, rec->cells,
                                           static_cast<const double2 *>(u), static_cast<const double2 *>(d_obs),
                                           static_cast<double2 *>(r), phi);
  return check_launch("k_residual");
}

extern "C" int normal_cg(const dbi_model *background, const dbi_batch *batch, const void *Ghat,
                         const void *u_b, const dbi_receivers *rec, const void *dd,
                         const dbi_cg_opts *cg, const void *power_start, void *dm, double *lambda_out,
                         double *hist_out, const dbi_krylov_opts *opts, const dbi_status *status,
                         int precision, void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc = check_products(background, batch, Ghat, u_b, rec, dd, dm, opts, precision, work, work_bytes,
                          DBI_OP_NORMAL_CG);
  if (rc) return rc;
  if (!cg || cg->iters < 0 || cg->iters > 4096 || (!(cg->lambda > 0) && (cg->power_iters < 1 || !power_start || !(cg->lambda_rel > 0)))) {
    set_error("CG options need 0 <= iters <= 4096 and lambda > 0, or lambda_rel > 0, power_iters >= 1 and a start vector");
    return DBI_ERR_ARG;
  }
  const dbi_grid *g = &background->grid;
  if (size_t(rec->n) > size_t(g->nz) * g->nx) { set_error("normal_cg supports at most nz * nx receivers"); return DBI_ERR_ARG; }
  if (batch->B == 0) { set_error("normal_cg needs at least one problem"); return DBI_ERR_ARG; }
  Arena ar(work, work_bytes);
  ProdCtx c;
  if ((rc = prepare(c, ar, background, batch, Ghat, opts, status, precision, stream))) return rc;
  const size_t plane = size_t(g->nz) * g->nx, nm = 5 * plane;
  const size_t mb = nm * sizeof(double);
  double *x = static_cast<double *>(ar.take(mb));
  double *r = static_cast<double *>(ar.take(mb));
  double *p = static_cast<double *>(ar.take(mb));
  double *q = static_cast<double *>(ar.take(mb));
  double *gd = static_cast<double *>(ar.take(mb));
  void *dmt = ar.take(mb);  // the precision's real type
  double *part = static_cast<double *>(ar.take(bytes_partials(1)));
  double *sc = static_cast<double *>(ar.take(16 * sizeof(double)));
  double *hist = static_cast<double *>(ar.take(size_t(cg->iters + 1) * sizeof(double)));
  void *dvec = ar.take(size_t(batch->B) * g->nz * g->nx * 2 * (precision == DBI_C64 ? sizeof(float2) : sizeof(double2)));
  if ((rc = ar.check("normal_cg"))) return rc;
  cudaStream_t s = c.s;
  double rv[5];
  reference_values(background->ref, rv);
  const MScale MS{{rv[0], rv[1], rv[1], rv[3], rv[4], 0.0}};  // C13 takes the scale of C11
  const int mblocks = int(std::min<size_t>((nm + 255) / 256, 4096));

  // q = S adjoint(frechet(S p)) in FP64 model space
  auto H = [&](const double *pin, double *qout) -> int {
    int e;
    if (precision == DBI_C64) k_mscale<double, float><<<mblocks, 256, 0, s>>>(5, plane, pin, static_cast<float *>(dmt), MS);
    else k_mscale<double, double><<<mblocks, 256, 0, s>>>(5, plane, pin, static_cast<double *>(dmt), MS);
    if ((e = check_launch("k_mscale"))) return e;
    if ((e = frechet_internal(c, u_b, rec, dmt, dvec))) return e;
    if ((e = adjoint_internal<double>(c, u_b, rec, dvec, gd))) return e;
    k_mscale<double, double><<<mblocks, 256, 0, s>>>(5, plane, gd, qout, MS);
    return check_launch("k_mscale");
  };
  auto dot = [&](const double *a, const double *b) -> int {
    k_mdot<<<kMBlocks, kMThreads, 0, s>>>(nm, a, b, part);
    return check_launch("k_mdot");
  };
  auto scal = [&](int what, int k) -> int {
    k_scalar<<<1, 32, 0, s>>>(what, part, sc, hist, k);
    return check_launch("k_scalar");
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

  if (!(cg->lambda > 0)) {  // power iteration on Re J~^H J~
    const MScale one{{1, 1, 1, 1, 1, 1}};
    if (precision == DBI_C64) k_mscale<float, double><<<mblocks, 256, 0, s>>>(5, plane, static_cast<const float *>(power_start), p, one);
    else k_mscale<double, double><<<mblocks, 256, 0, s>>>(5, plane, static_cast<const double *>(power_start), p, one);
    if ((rc = check_launch("k_mscale"))) return rc;
    if ((rc = dot(p, p)) || (rc = scal(3, 0)) || (rc = axpy(2, p, p, nullptr, nullptr))) return rc;
    for (int it = 0; it < cg->power_iters; ++it) {
      if ((rc = H(p, q)) || (rc = dot(q, q)) || (rc = scal(3, 0)) || (rc = axpy(2, q, p, nullptr, nullptr))) return rc;
    }
    if ((rc = H(p, q)) || (rc = dot(p, q)) || (rc = scal(4, 0))) return rc;
  }
  // CG from x = 0: r = p = S Re J^H dd
  if ((rc = adjoint_internal<double>(c, u_b, rec, dd, gd))) return rc;
  k_mscale<double, double><<<mblocks, 256, 0, s>>>(5, plane, gd, r, MS);
  if ((rc = check_launch("k_mscale"))) return rc;
  e = cudaMemsetAsync(x, 0, mb, s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(x)", e);
  if ((rc = axpy(4, r, p, nullptr, nullptr)) || (rc = dot(r, r)) || (rc = scal(0, 0))) return rc;
  for (int k = 0; k < cg->iters; ++k) {
    if ((rc = H(p, q)) || (rc = axpy(3, p, q, nullptr, nullptr))) return rc;  // q = H p + lambda p
    if ((rc = dot(p, q)) || (rc = scal(1, 0))) return rc;                      // alpha
    if ((rc = axpy(0, p, x, q, r))) return rc;                                 // x, r
    if ((rc = dot(r, r)) || (rc = scal(2, k + 1))) return rc;                  // beta, hist
    if ((rc = axpy(1, r, p, nullptr, nullptr))) return rc;                     // p
  }
  if (precision == DBI_C64) k_mscale<double, float><<<mblocks, 256, 0, s>>>(5, plane, x, static_cast<float *>(dm), MS);
  else k_mscale<double, double><<<mblocks, 256, 0, s>>>(5, plane, x, static_cast<double *>(dm), MS);
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

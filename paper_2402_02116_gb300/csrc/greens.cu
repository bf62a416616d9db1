// Green's tensor tables (Appendix A, Eq. A-3, A-4) and the incident field (Eq. 7).
//
// greens_tabulate evaluates the 2D isotropic Green's tensor
//   G_ij(y) = 1/(8 i rho) [A delta_ij - B (2 g_i g_j - delta_ij)],
//   A = H0(w r/alpha)/alpha^2 + H0(w r/beta)/beta^2,  B = H2(w r/alpha)/alpha^2 - H2(w r/beta)/beta^2,
// H_n = J_n - i Y_n (second kind, outgoing for exp(+i w t)), in FP64 at the cell-centre offsets
// (dx h, dz h), |dz| < nz, |dx| < nx, placed at slot (dz mod lz, dx mod lx). The self cell takes
// the mean of G over the disk of radius h / sqrt(pi): only A survives the angular mean, and
// the disk mean of H0(k r) is 2 H1(k a)/(k a) - 4i/(pi k^2 a^2). The table is then transformed by
// an FP64 2D FFT (rows, then columns), scaled by h^2 / (lz lx), which folds the quadrature
// weight and the inverse-FFT normalisation of Eq. 12 into it, and stored column-major.
#include <cmath>

#include "fft.cuh"
#include "operator.cuh"

namespace dbi {

// H_n^(2)(z) = J_n(z) - i Y_n(z), n = 0, 1, 2 (n = 2 by the recurrence H2 = (2/z) H1 - H0).
__device__ __forceinline__ void hankel2_012(double z, double2 &h0, double2 &h1, double2 &h2) {
  h0 = make_double2(j0(z), -y0(z));
  h1 = make_double2(j1(z), -y1(z));
  h2 = make_double2(2.0 * h1.x / z - h0.x, 2.0 * h1.y / z - h0.y);
}

__device__ __forceinline__ double2 times_inv_8i_rho(double2 v, double rho) {
  // v / (8 i rho) = -i v / (8 rho)
  const double s = 1.0 / (8.0 * rho);
  return make_double2(v.y * s, -v.x * s);
}

__device__ void green_offset(double y1, double y3, double omega, double alpha, double beta,
                             double rho, double2 &g11, double2 &g13, double2 &g33) {
  const double r = hypot(y1, y3);
  const double c1 = y1 / r, c3 = y3 / r;
  double2 h0a, h1a, h2a, h0b, h1b, h2b;
  hankel2_012(omega * r / alpha, h0a, h1a, h2a);
  hankel2_012(omega * r / beta, h0b, h1b, h2b);
  const double ia2 = 1.0 / (alpha * alpha), ib2 = 1.0 / (beta * beta);
  const double2 A = make_double2(h0a.x * ia2 + h0b.x * ib2, h0a.y * ia2 + h0b.y * ib2);
  const double2 B = make_double2(h2a.x * ia2 - h2b.x * ib2, h2a.y * ia2 - h2b.y * ib2);
  const double q11 = 2.0 * c1 * c1 - 1.0, q33 = 2.0 * c3 * c3 - 1.0, q13 = 2.0 * c1 * c3;
  g11 = times_inv_8i_rho(make_double2(A.x - B.x * q11, A.y - B.y * q11), rho);
  g33 = times_inv_8i_rho(make_double2(A.x - B.x * q33, A.y - B.y * q33), rho);
  g13 = times_inv_8i_rho(make_double2(-B.x * q13, -B.y * q13), rho);
}

__device__ double2 green_self(double h, double omega, double alpha, double beta, double rho) {
  const double a = h / sqrt(M_PI);
  double2 tot = make_double2(0.0, 0.0);
  const double cs[2] = {alpha, beta};
  for (int i = 0; i < 2; ++i) {
    const double k = omega / cs[i], ka = k * a;
    const double2 h1 = make_double2(j1(ka), -y1(ka));
    // 2 H1(ka)/(ka) - 4 i / (pi k^2 a^2)
    const double2 mean = make_double2(2.0 * h1.x / ka, 2.0 * h1.y / ka - 4.0 / (M_PI * ka * ka));
    const double ic2 = 1.0 / (cs[i] * cs[i]);
    tot.x += mean.x * ic2;
    tot.y += mean.y * ic2;
  }
  return times_inv_8i_rho(tot, rho);
}

// One thread per offset (dz, dx) with dz, dx >= 0: G11 and G33 are even and G13 odd in each
// offset coordinate (Eq. A-3), so the four slots (+-dz, +-dx) are filled from one evaluation (the
// mirrored values are bit-identical to direct evaluations). Gap slots are zeroed beforehand.
template <typename C>
__global__ void k_green_space(int nz, int nx, int lz, int lx, double h, const double *omega,
                              double rho, double alpha, double beta, double2 *W, C *Gspace) {
  const int dx = blockIdx.x * blockDim.x + threadIdx.x;
  const int dz = blockIdx.y;
  const int f = blockIdx.z;
  if (dx >= nx) return;
  double2 g11, g13 = make_double2(0, 0), g33;
  const double w = omega[f];
  if (dz == 0 && dx == 0) {
    g11 = g33 = green_self(h, w, alpha, beta, rho);
  } else {
    green_offset(dx * h, dz * h, w, alpha, beta, rho, g11, g13, g33);
  }
  const size_t plane = size_t(lz) * lx, base = size_t(f) * 3 * plane;
  using R = typename RealOf<C>::type;
  for (int sz = 0; sz < 2; ++sz) {
    if (sz == 1 && dz == 0) continue;
    const int iz = sz ? lz - dz : dz;
    for (int sx = 0; sx < 2; ++sx) {
      if (sx == 1 && dx == 0) continue;
      const int ix = sx ? lx - dx : dx;
      const double sg = (sz ^ sx) ? -1.0 : 1.0;  // G13 is odd in each coordinate
      const double2 q13 = make_double2(sg * g13.x, sg * g13.y);
      const size_t cell = size_t(iz) * lx + ix;
      W[base + cell] = g11;
      W[base + plane + cell] = q13;
      W[base + 2 * plane + cell] = g33;
      if (Gspace) {
        Gspace[base + cell] = mk<C>(R(g11.x), R(g11.y));
        Gspace[base + plane + cell] = mk<C>(R(q13.x), R(q13.y));
        Gspace[base + 2 * plane + cell] = mk<C>(R(g33.x), R(g33.y));
      }
    }
  }
}

// In-place FP64 FFT of NL contiguous lines of length L per block.
template <int L>
__global__ void __launch_bounds__(256) k_fft_rows64(double2 *data, long nlines, const double2 *tw) {
  constexpr int NL = 2048 / L > 0 ? 2048 / L : 1, LS = L + 1, NT = NL * L / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *s = reinterpret_cast<double2 *>(smem_raw);
  const long l0 = long(blockIdx.x) * NL;
  for (int idx = threadIdx.x; idx < NL * L; idx += NT) {
    const int l = idx / L, k = idx - l * L;
    s[l * LS + k] = (l0 + l < nlines) ? data[(l0 + l) * L + k] : make_double2(0, 0);
  }
  __syncthreads();
  Plan<L>::template run<double2, NL, LS, NT, false>(s, tw);
  for (int idx = threadIdx.x; idx < NL * L; idx += NT) {
    const int l = idx / L, k = idx - l * L;
    if (l0 + l < nlines) data[(l0 + l) * L + k] = s[l * LS + k];
  }
}

// In-place FP64 FFT along the columns of row-major [L][width] matrices; CC columns per block,
// matrix blockIdx.y.
template <int L>
__global__ void __launch_bounds__(256) k_fft_cols64(double2 *data, int width, const double2 *tw) {
  constexpr int CC = 2048 / L > 0 ? 2048 / L : 1, LS = L + 1, NT = CC * L / 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *s = reinterpret_cast<double2 *>(smem_raw);
  double2 *M = data + size_t(blockIdx.y) * L * width;
  const int c0 = blockIdx.x * CC;
  for (int idx = threadIdx.x; idx < CC * L; idx += NT) {
    const int z = idx / CC, j = idx - z * CC;
    s[j * LS + z] = (c0 + j < width) ? M[size_t(z) * width + c0 + j] : make_double2(0, 0);
  }
  __syncthreads();
  Plan<L>::template run<double2, CC, LS, NT, false>(s, tw);
  for (int idx = threadIdx.x; idx < CC * L; idx += NT) {
    const int z = idx / CC, j = idx - z * CC;
    if (c0 + j < width) M[size_t(z) * width + c0 + j] = s[j * LS + z];
  }
}

// FP64 FFT of length 768 = 3 x 256 by one decimation-in-frequency step: with the thirds
// x_p[i] = x[i + 256 p] of a line, X[3m + q] = sum_i W_256^{im} W_768^{iq} sum_p W_3^{pq} x_p[i], i.e.
// the 256-point DFTs of the three folded lines. A block holds NL lines; line l's third p is loaded
// to s[(3 l + p) LS + i], and the fold writes its residue q to the same slots (3 l + q), in place.
constexpr int k768NL = 2, k768LS = 257, k768NT = 3 * k768NL * 256 / 8;

__device__ __forceinline__ void fold768_fp64(double2 *s, const double2 *tw) {
  const double2 w3 = tw[kTwiddleN / 3], w3b = tw[2 * kTwiddleN / 3];  // W_3, W_3^2
  constexpr int TWS = kTwiddleN / 768;
  for (int idx = threadIdx.x; idx < k768NL * 256; idx += k768NT) {
    const int l = idx >> 8, i = idx & 255;
    double2 *p = s + 3 * l * k768LS + i;
    const double2 a0 = p[0], a1 = p[k768LS], a2 = p[2 * k768LS];
    p[0] = cadd(a0, cadd(a1, a2));
    p[k768LS] = cmul(tw[i * TWS], cadd(a0, cadd(cmul(w3, a1), cmul(w3b, a2))));
    p[2 * k768LS] = cmul(tw[2 * i * TWS], cadd(a0, cadd(cmul(w3b, a1), cmul(w3, a2))));
  }
}

__global__ void __launch_bounds__(k768NT) k_fft_rows64_768(double2 *data, long nlines, const double2 *tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *s = reinterpret_cast<double2 *>(smem_raw);
  const long l0 = long(blockIdx.x) * k768NL;
  for (int idx = threadIdx.x; idx < k768NL * 768; idx += k768NT) {
    const int l = idx / 768, k = idx - l * 768;
    s[(3 * l + (k >> 8)) * k768LS + (k & 255)] = l0 + l < nlines ? data[(l0 + l) * 768 + k] : make_double2(0, 0);
  }
  __syncthreads();
  fold768_fp64(s, tw);
  __syncthreads();
  Plan<256>::template run<double2, 3 * k768NL, k768LS, k768NT, false>(s, tw);
  for (int idx = threadIdx.x; idx < k768NL * 768; idx += k768NT) {
    const int l = idx / 768, k = idx - l * 768, m = k / 3, q = k - 3 * m;
    if (l0 + l < nlines) data[(l0 + l) * 768 + k] = s[(3 * l + q) * k768LS + m];
  }
}

// The same along the columns of row-major [768][width] matrices (matrix blockIdx.y).
__global__ void __launch_bounds__(k768NT) k_fft_cols64_768(double2 *data, int width, const double2 *tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2 *s = reinterpret_cast<double2 *>(smem_raw);
  double2 *M = data + size_t(blockIdx.y) * 768 * width;
  const int c0 = blockIdx.x * k768NL;
  for (int idx = threadIdx.x; idx < k768NL * 768; idx += k768NT) {
    const int z = idx / k768NL, j = idx - z * k768NL;
    s[(3 * j + (z >> 8)) * k768LS + (z & 255)] = c0 + j < width ? M[size_t(z) * width + c0 + j] : make_double2(0, 0);
  }
  __syncthreads();
  fold768_fp64(s, tw);
  __syncthreads();
  Plan<256>::template run<double2, 3 * k768NL, k768LS, k768NT, false>(s, tw);
  for (int idx = threadIdx.x; idx < k768NL * 768; idx += k768NT) {
    const int z = idx / k768NL, j = idx - z * k768NL, m = z / 3, q = z - 3 * m;
    if (c0 + j < width) M[size_t(z) * width + c0 + j] = s[(3 * j + q) * k768LS + m];
  }
}

// Ghat[f][c][kx][kz] = scale * W[f][c][kz][kx]: scaled, rounded and stored column-major (kz
// contiguous) for the column pass. One 32 x 32 tile per block, transposed through shared memory.
// At lz = 768 the kz slots are residue-major: slot (kz mod 3) 256 + kz / 3 (the order in which the
// column stage's three 256-point transforms consume them).
template <typename C>
__global__ void k_scale_cast_t(const double2 *W, C *Ghat, int lz, int lx, double scale) {
  using R = typename RealOf<C>::type;
  __shared__ double2 tile[32][33];
  const size_t plane = size_t(lz) * lx;
  const double2 *Wm = W + size_t(blockIdx.z) * plane;
  C *Gm = Ghat + size_t(blockIdx.z) * plane;
  const int kx0 = blockIdx.x * 32, kz0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int kz = kz0 + i, kx = kx0 + threadIdx.x;
    if (kz < lz && kx < lx) tile[i][threadIdx.x] = Wm[size_t(kz) * lx + kx];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int kx = kx0 + i, kz = kz0 + threadIdx.x;
    if (kz < lz && kx < lx) {
      const double2 w = tile[threadIdx.x][i];
      const int slot = lz == 768 ? (kz % 3) * 256 + kz / 3 : kz;
      Gm[size_t(kx) * lz + slot] = mk<C>(R(w.x * scale), R(w.y * scale));
    }
  }
}


int fft_rows_fp64(double2 *W, long nlines, int L, const double2 *tw, cudaStream_t s) {
  if (L == 768) {
    const size_t bytes = size_t(3 * k768NL) * k768LS * sizeof(double2);
    k_fft_rows64_768<<<unsigned((nlines + k768NL - 1) / k768NL), k768NT, bytes, s>>>(W, nlines, tw);
    return check_launch("k_fft_rows64_768");
  }
  int rc = DBI_ERR_UNSUPPORTED;
  dispatch_len(L, [&]<int LL>() {
    constexpr int NL = 2048 / LL > 0 ? 2048 / LL : 1, LS = LL + 1, NT = NL * LL / 8;
    const size_t bytes = size_t(NL) * LS * sizeof(double2);
    cudaError_t e = allow_smem(k_fft_rows64<LL>, bytes);
    if (e == cudaSuccess) k_fft_rows64<LL><<<unsigned((nlines + NL - 1) / NL), NT, bytes, s>>>(W, nlines, tw);
    rc = e != cudaSuccess ? cuda_fail("k_fft_rows64 smem", e) : check_launch("k_fft_rows64");
  });
  return rc;
}

int fft_cols_fp64(double2 *W, int nmat, int L, int width, const double2 *tw, cudaStream_t s) {
  if (L == 768) {
    const size_t bytes = size_t(3 * k768NL) * k768LS * sizeof(double2);
    k_fft_cols64_768<<<dim3((width + k768NL - 1) / k768NL, nmat), k768NT, bytes, s>>>(W, width, tw);
    return check_launch("k_fft_cols64_768");
  }
  int rc = DBI_ERR_UNSUPPORTED;
  dispatch_len(L, [&]<int LL>() {
    constexpr int CC = 2048 / LL > 0 ? 2048 / LL : 1, LS = LL + 1, NT = CC * LL / 8;
    const size_t bytes = size_t(CC) * LS * sizeof(double2);
    cudaError_t e = allow_smem(k_fft_cols64<LL>, bytes);
    dim3 grid((width + CC - 1) / CC, nmat);
    if (e == cudaSuccess) k_fft_cols64<LL><<<grid, NT, bytes, s>>>(W, width, tw);
    rc = e != cudaSuccess ? cuda_fail("k_fft_cols64 smem", e) : check_launch("k_fft_cols64");
  });
  return rc;
}

static int fft2_fp64(double2 *W, int nmat, int lz, int lx, const double2 *tw, cudaStream_t s) {
  int rc = fft_rows_fp64(W, long(nmat) * lz, lx, tw, s);
  return rc ? rc : fft_cols_fp64(W, nmat, lz, lx, tw, s);
}

// Problems whose source cell or frequency index is out of range get u0 = 0.
template <typename C>
__global__ void k_incident(int B, int nf, int nz, int nx, int lz, int lx, const int *fidx, const C *Gspace,
                           const int *src_cells, const double *forces, C *u0) {
  using R = typename RealOf<C>::type;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  const int b = blockIdx.z;
  if (x >= nx) return;
  const int zs = src_cells[2 * b], xs = src_cells[2 * b + 1];
  const size_t o = size_t(b) * 2 * nz * nx + size_t(z) * nx + x;
  if (zs < 0 || zs >= nz || xs < 0 || xs >= nx || unsigned(fidx[b]) >= unsigned(nf)) {
    u0[o] = czero<C>();
    u0[o + size_t(nz) * nx] = czero<C>();
    return;
  }
  int dz = z - zs, dx = x - xs;
  dz = dz < 0 ? dz + lz : dz;
  dx = dx < 0 ? dx + lx : dx;
  const size_t plane = size_t(lz) * lx, cell = size_t(dz) * lx + dx;
  const C *G = Gspace + size_t(fidx[b]) * 3 * plane;
  const C g11 = G[cell], g13 = G[plane + cell], g33 = G[2 * plane + cell];
  const R f1 = R(forces[2 * b]), f3 = R(forces[2 * b + 1]);
  u0[o] = cadd(cscale(g11, f1), cscale(g13, f3));
  u0[o + size_t(nz) * nx] = cadd(cscale(g13, f1), cscale(g33, f3));
}

// Derivative tables of the paper-literal form (Eq. 9): central differences of the lattice G_h,
// (D_k G)(y) = [G_h(y + h e_k) - G_h(y - h e_k)] / 2h (G_h(0) = the self-cell mean), at every
// offset |dz| < nz, |dx| < nx, combined into the six entries the kernel of Eq. 9 needs over the
// stress components: [f][e][kz slot][kx slot] with e = D1G11, D1G13 (sigma1), D3G11 + D1G13,
// D3G13 + D1G33 (sigma5), D3G13, D3G33 (sigma3). One thread per offset; gap slots zeroed before.
__device__ __forceinline__ void green_at(int dz, int dx, double h, double w, double alpha, double beta,
                                         double rho, double2 &g11, double2 &g13, double2 &g33) {
  if (dz == 0 && dx == 0) {
    g11 = g33 = green_self(h, w, alpha, beta, rho);
    g13 = make_double2(0.0, 0.0);
  } else {
    green_offset(dx * h, dz * h, w, alpha, beta, rho, g11, g13, g33);
  }
}

__global__ void k_green_deriv(int nz, int nx, int lz, int lx, double h, const double *omega, double rho,
                              double alpha, double beta, double2 *W) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;  // dx + nx - 1
  const int dz = int(blockIdx.y) - (nz - 1);
  const int f = blockIdx.z;
  if (ix >= 2 * nx - 1) return;
  const int dx = ix - (nx - 1);
  const double w = omega[f];
  double2 xp[3], xm[3], zp[3], zm[3];
  green_at(dz, dx + 1, h, w, alpha, beta, rho, xp[0], xp[1], xp[2]);
  green_at(dz, dx - 1, h, w, alpha, beta, rho, xm[0], xm[1], xm[2]);
  green_at(dz + 1, dx, h, w, alpha, beta, rho, zp[0], zp[1], zp[2]);
  green_at(dz - 1, dx, h, w, alpha, beta, rho, zm[0], zm[1], zm[2]);
  const double i2h = 1.0 / (2.0 * h);
  double2 d1[3], d3[3];
  for (int c = 0; c < 3; ++c) {
    d1[c] = make_double2((xp[c].x - xm[c].x) * i2h, (xp[c].y - xm[c].y) * i2h);
    d3[c] = make_double2((zp[c].x - zm[c].x) * i2h, (zp[c].y - zm[c].y) * i2h);
  }
  const double2 e[6] = {d1[0], d1[1], make_double2(d3[0].x + d1[1].x, d3[0].y + d1[1].y),
                        make_double2(d3[1].x + d1[2].x, d3[1].y + d1[2].y), d3[1], d3[2]};
  const size_t plane = size_t(lz) * lx;
  const size_t cell = size_t(dz < 0 ? dz + lz : dz) * lx + (dx < 0 ? dx + lx : dx);
  for (int k = 0; k < 6; ++k) W[(size_t(f) * 6 + k) * plane + cell] = e[k];
}

}  // namespace dbi

using namespace dbi;

extern "C" int greens_tabulate_k(const dbi_grid *g, const dbi_medium *ref, const double *omega, int nf,
                                 int precision, void *Dhat, void *work, size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid(g)) || (rc = check_precision(precision))) return rc;
  if (ref && reference_is_vti(*ref)) {
    set_error("the derivative tables are tabulated for an isotropic reference only");
    return DBI_ERR_ARG;
  }
  if (!ref || !(ref->rho0 > 0) || !(ref->alpha0 > 0) || !(ref->beta0 > 0) || !(ref->alpha0 > ref->beta0)) {
    set_error("reference medium needs rho0 > 0 and alpha0 > beta0 > 0");
    return DBI_ERR_ARG;
  }
  if (nf < 1 || !omega || !Dhat) { set_error("need nf >= 1, omega and Dhat"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes(g, nf, precision, DBI_OP_GREENS_K);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  double2 *tw = static_cast<double2 *>(ar.take(bytes_twiddles(DBI_C128)));
  const size_t tab = size_t(nf) * 6 * g->lz * g->lx;
  double2 *W = static_cast<double2 *>(ar.take(tab * sizeof(double2)));
  if ((rc = ar.check("greens_tabulate_k"))) return rc;
  if ((rc = launch_twiddles(tw, DBI_C128, s))) return rc;
  cudaError_t e = cudaMemsetAsync(W, 0, tab * sizeof(double2), s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(derivative table)", e);
  dim3 grid((2 * g->nx - 1 + 127) / 128, 2 * g->nz - 1, nf);
  k_green_deriv<<<grid, 128, 0, s>>>(g->nz, g->nx, g->lz, g->lx, g->h, omega, ref->rho0, ref->alpha0,
                                     ref->beta0, W);
  if ((rc = check_launch("k_green_deriv"))) return rc;
  if ((rc = fft2_fp64(W, 6 * nf, g->lz, g->lx, tw, s))) return rc;
  const double scale = g->h * g->h / (double(g->lz) * double(g->lx));
  const dim3 tgrid((g->lx + 31) / 32, (g->lz + 31) / 32, 6 * nf), tblock(32, 8);
  if (precision == DBI_C64)
    k_scale_cast_t<float2><<<tgrid, tblock, 0, s>>>(W, static_cast<float2 *>(Dhat), g->lz, g->lx, scale);
  else
    k_scale_cast_t<double2><<<tgrid, tblock, 0, s>>>(W, static_cast<double2 *>(Dhat), g->lz, g->lx, scale);
  return check_launch("k_scale_cast_t");
}

// A homogeneous VTI reference must be elastically stable: rho, C11, C33, C55 > 0, C11 C33 > C13^2.
static int check_vti(const dbi_medium *r) {
  if (!(r->rho0 > 0) || !(r->c11 > 0) || !(r->c33 > 0) || !(r->c55 > 0) || !(r->c11 * r->c33 > r->c13 * r->c13)) {
    set_error("VTI reference needs rho0, C11, C33, C55 > 0 and C11 C33 > C13^2");
    return DBI_ERR_ARG;
  }
  return DBI_OK;
}

extern "C" int greens_tabulate(const dbi_grid *g, const dbi_medium *ref, const double *omega,
                               int nf, int precision, void *Ghat, void *Gspace, void *work,
                               size_t work_bytes, dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid(g, precision)) || (rc = check_precision(precision))) return rc;
  const bool vti = ref && reference_is_vti(*ref);
  if (vti && (rc = check_vti(ref))) return rc;
  if (!vti && (!ref || !(ref->rho0 > 0) || !(ref->alpha0 > 0) || !(ref->beta0 > 0) || !(ref->alpha0 > ref->beta0))) {
    set_error("reference medium needs rho0 > 0 and alpha0 > beta0 > 0");
    return DBI_ERR_ARG;
  }
  if (nf < 1 || !omega || !Ghat) { set_error("need nf >= 1, omega and Ghat"); return DBI_ERR_ARG; }
  const size_t need = dbi_workspace_bytes(g, nf, precision, DBI_OP_GREENS);
  if (!work || work_bytes < need) {
    set_error("work buffer of %zu bytes, need %zu", work_bytes, need);
    return DBI_ERR_WORKSPACE;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar(work, work_bytes);
  double2 *tw = static_cast<double2 *>(ar.take(bytes_twiddles(DBI_C128)));
  double2 *W = static_cast<double2 *>(ar.take(size_t(nf) * 3 * g->lz * g->lx * sizeof(double2)));
  if ((rc = ar.check("greens_tabulate"))) return rc;
  if ((rc = launch_twiddles(tw, DBI_C128, s))) return rc;
  const size_t tab = size_t(nf) * 3 * g->lz * g->lx;
  cudaError_t e = cudaMemsetAsync(W, 0, tab * sizeof(double2), s);
  if (e == cudaSuccess && Gspace)
    e = cudaMemsetAsync(Gspace, 0, tab * (precision == DBI_C64 ? sizeof(float2) : sizeof(double2)), s);
  if (e != cudaSuccess) return cuda_fail("cudaMemsetAsync(Green table)", e);
  dim3 grid((g->nx + 127) / 128, g->nz, nf);
  if (vti) {
    if ((rc = launch_green_vti(g, *ref, omega, nf, W, Gspace, precision, s))) return rc;
  } else {
    if (precision == DBI_C64)
      k_green_space<float2><<<grid, 128, 0, s>>>(g->nz, g->nx, g->lz, g->lx, g->h, omega, ref->rho0,
                                                 ref->alpha0, ref->beta0, W, static_cast<float2 *>(Gspace));
    else
      k_green_space<double2><<<grid, 128, 0, s>>>(g->nz, g->nx, g->lz, g->lx, g->h, omega, ref->rho0,
                                                  ref->alpha0, ref->beta0, W, static_cast<double2 *>(Gspace));
    if ((rc = check_launch("k_green_space"))) return rc;
  }
  if ((rc = fft2_fp64(W, 3 * nf, g->lz, g->lx, tw, s))) return rc;
  const double scale = g->h * g->h / (double(g->lz) * double(g->lx));
  const dim3 tgrid((g->lx + 31) / 32, (g->lz + 31) / 32, 3 * nf), tblock(32, 8);
  if (precision == DBI_C64)
    k_scale_cast_t<float2><<<tgrid, tblock, 0, s>>>(W, static_cast<float2 *>(Ghat), g->lz, g->lx, scale);
  else
    k_scale_cast_t<double2><<<tgrid, tblock, 0, s>>>(W, static_cast<double2 *>(Ghat), g->lz, g->lx, scale);
  return check_launch("k_scale_cast_t");
}

extern "C" int incident_field(const dbi_grid *g, const dbi_batch *batch, const void *Gspace,
                              const int *src_cells, const double *forces, void *u0, int precision,
                              dbi_stream stream) {
  clear_error();
  int rc;
  if ((rc = check_grid(g, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  if (batch->B == 0) return DBI_OK;
  if (!Gspace || !src_cells || !forces || !u0) { set_error("NULL Gspace, sources, forces or u0"); return DBI_ERR_ARG; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  dim3 grid((g->nx + 127) / 128, g->nz, batch->B);
  if (precision == DBI_C64)
    k_incident<float2><<<grid, 128, 0, s>>>(batch->B, batch->nf, g->nz, g->nx, g->lz, g->lx, batch->fidx,
                                            static_cast<const float2 *>(Gspace), src_cells, forces,
                                            static_cast<float2 *>(u0));
  else
    k_incident<double2><<<grid, 128, 0, s>>>(batch->B, batch->nf, g->nz, g->nx, g->lz, g->lx, batch->fidx,
                                             static_cast<const double2 *>(Gspace), src_cells, forces,
                                             static_cast<double2 *>(u0));
  return check_launch("k_incident");
}

// Plain FP64 C++17 oracle of the 2D elastic Lippmann-Schwinger operator and the misfit gradient of
// the distorted-Born method (arXiv 2402.02116).
//
// TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline and
// reference legs load it (through oracle/cpp_oracle.py). It shares no code with the CUDA library
// and includes nothing from it; it restates the same discrete problem as oracle/dbi_oracle.py:
//   * Green's tensor: the 2D closed form of Appendix A (Eq. A-3, A-4), H^(2) for exp(+i w t),
//     midpoint rule at cell-centre offsets, the disk-averaged self cell (area h^2).
//   * Contrast source (Eq. 6): s = w^2 drho u + div(dC : eps(u)), central differences with fields
//     zero outside the grid, 2D VTI stiffness on Voigt indices {1, 3, 5} (Eq. 39).
//   * LS operator (Eq. 10): A u = u - h^2 G * s, the convolution by Eq. 12 on the zero-padded
//     lz x lx grid with this file's own radix-2 FFT (lz, lx powers of two), or by the direct
//     O(N^4) sum ("tier 1", tiny grids).
//   * Krylov (Eq. 11): BiCGSTAB (van der Vorst), <a, b> = sum conj(a) b, x0 = 0, shadow residual r0.
//   * Gradient (Eq. 23, 25, 32-35): r = P u - d_obs, u_a = A^-1 G P^T conj(r), and
//     Re(w^2 u_a . u_b) for rho, -Re(eps(u_a)^T B_p eps(u_b)) for C11, C13, C33, C55.
// Problems of a batch run in parallel with OpenMP, one problem per thread.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------------
// Green's tensor (Appendix A, Eq. A-3 and A-4)
// ---------------------------------------------------------------------------------------------
cd hankel2(int n, double x) { return cd(std::cyl_bessel_j(double(n), x), -std::cyl_neumann(double(n), x)); }

struct G3 {
  cd g11, g13, g33;
};

// G_ij(y) = 1/(8 i rho) [A d_ij - B (2 g_i g_j - d_ij)], A = H0(w r/a)/a^2 + H0(w r/b)/b^2,
// B = H2(w r/a)/a^2 - H2(w r/b)/b^2, g = y / r, y = (y1, y3) != 0.
G3 green(double y1, double y3, double w, double alpha, double beta, double rho) {
  const double r = std::hypot(y1, y3), g1 = y1 / r, g3 = y3 / r;
  const double za = w * r / alpha, zb = w * r / beta;
  const cd A = hankel2(0, za) / (alpha * alpha) + hankel2(0, zb) / (beta * beta);
  const cd B = hankel2(2, za) / (alpha * alpha) - hankel2(2, zb) / (beta * beta);
  const cd pref = 1.0 / (cd(0.0, 8.0) * rho);
  return {pref * (A - B * (2.0 * g1 * g1 - 1.0)), pref * (-B * 2.0 * g1 * g3), pref * (A - B * (2.0 * g3 * g3 - 1.0))};
}

// Mean of G over the disk of radius a = h / sqrt(pi): the B term has zero angular mean; the disk
// mean of H0(k r) is 2 H1(k a)/(k a) - 4i/(pi k^2 a^2).
G3 green_self(double h, double w, double alpha, double beta, double rho) {
  const double a = h / std::sqrt(kPi);
  cd tot = 0.0;
  for (double c : {alpha, beta}) {
    const double k = w / c;
    tot += (2.0 * hankel2(1, k * a) / (k * a) - cd(0.0, 4.0) / (kPi * k * k * a * a)) / (c * c);
  }
  const cd g = tot / (cd(0.0, 8.0) * rho);
  return {g, 0.0, g};
}

// G_h on the (2nz-1) x (2nx-1) offsets: out[c][dz + nz - 1][dx + nx - 1], y = (dx h, dz h).
void green_lattice(int nz, int nx, double h, double w, double alpha, double beta, double rho, cd *out) {
  const int mz = 2 * nz - 1, mx = 2 * nx - 1;
  for (int iz = 0; iz < mz; ++iz)
    for (int ix = 0; ix < mx; ++ix) {
      const int dz = iz - (nz - 1), dx = ix - (nx - 1);
      const G3 g = (dz == 0 && dx == 0) ? green_self(h, w, alpha, beta, rho) : green(dx * h, dz * h, w, alpha, beta, rho);
      const size_t o = size_t(iz) * mx + ix, plane = size_t(mz) * mx;
      out[o] = g.g11;
      out[plane + o] = g.g13;
      out[2 * plane + o] = g.g33;
    }
}

// ---------------------------------------------------------------------------------------------
// radix-2 FFT (Cooley-Tukey, iterative, in place), unnormalised; sign -1 forward, +1 inverse
// ---------------------------------------------------------------------------------------------
// exp(sign 2 pi i k / n), k < n / 2
void twiddles(int n, int sign, std::vector<cd> &tw) {
  tw.resize(n / 2);
  for (int k = 0; k < n / 2; ++k) tw[k] = std::polar(1.0, sign * 2.0 * kPi * k / n);
}

void fft(cd *x, int n, const std::vector<cd> &tw) {
  for (int i = 1, j = 0; i < n; ++i) {  // bit reversal
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len / 2, step = n / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < half; ++k) {
        const cd a = x[i + k], b = x[i + k + half] * tw[size_t(k) * step];
        x[i + k] = a + b;
        x[i + k + half] = a - b;
      }
  }
}

// 2D FFT of an lz x lx row-major array: every row, then every column (gathered eight at a time
// into contiguous lines).
void fft2(cd *a, int lz, int lx, int sign, std::vector<cd> &col) {
  std::vector<cd> twx, twz;
  twiddles(lx, sign, twx);
  twiddles(lz, sign, twz);
  for (int z = 0; z < lz; ++z) fft(a + size_t(z) * lx, lx, twx);
  constexpr int kG = 8;
  col.resize(size_t(kG) * lz);
  for (int x0 = 0; x0 < lx; x0 += kG) {
    const int g = lx - x0 < kG ? lx - x0 : kG;
    for (int z = 0; z < lz; ++z)
      for (int c = 0; c < g; ++c) col[size_t(c) * lz + z] = a[size_t(z) * lx + x0 + c];
    for (int c = 0; c < g; ++c) fft(col.data() + size_t(c) * lz, lz, twz);
    for (int z = 0; z < lz; ++z)
      for (int c = 0; c < g; ++c) a[size_t(z) * lx + x0 + c] = col[size_t(c) * lz + z];
  }
}

// ---------------------------------------------------------------------------------------------
// one grid and one frequency: tables, contrast source, operator, BiCGSTAB, imaging
// ---------------------------------------------------------------------------------------------
struct Grid {
  int nz, nx, lz, lx;
  double h, rho0, alpha0, beta0;
  double ref[5];  // rho, C11, C13, C33, C55 of the isotropic reference (Eq. 4)
  const double *model;  // [5][nz][nx] absolute
  size_t cells() const { return size_t(nz) * nx; }
};

struct Freq {
  double w;
  std::vector<cd> lat;   // [3][2nz-1][2nx-1]
  std::vector<cd> ghat;  // [3][lz][lx]: FFT of the circulant embedding (Eq. 12)
};

void make_freq(const Grid &g, double w, bool spectrum, Freq &f) {
  f.w = w;
  const int mz = 2 * g.nz - 1, mx = 2 * g.nx - 1;
  f.lat.assign(size_t(3) * mz * mx, 0.0);
  green_lattice(g.nz, g.nx, g.h, w, g.alpha0, g.beta0, g.rho0, f.lat.data());
  if (!spectrum) return;
  const size_t plane = size_t(g.lz) * g.lx;
  f.ghat.assign(3 * plane, 0.0);
  std::vector<cd> col;
  for (int c = 0; c < 3; ++c) {
    cd *P = f.ghat.data() + c * plane;
    for (int iz = 0; iz < mz; ++iz)
      for (int ix = 0; ix < mx; ++ix) {  // offset d goes to slot d mod L
        const int sz = ((iz - (g.nz - 1)) % g.lz + g.lz) % g.lz, sx = ((ix - (g.nx - 1)) % g.lx + g.lx) % g.lx;
        P[size_t(sz) * g.lx + sx] = f.lat[c * size_t(mz) * mx + size_t(iz) * mx + ix];
      }
    fft2(P, g.lz, g.lx, -1, col);
  }
}

// central difference along x1 (last axis) / x3, field zero outside the grid
inline cd d1(const cd *v, int nz, int nx, int z, int x, double inv2h) {
  (void)nz;
  const cd r = x + 1 < nx ? v[size_t(z) * nx + x + 1] : 0.0, l = x > 0 ? v[size_t(z) * nx + x - 1] : 0.0;
  return (r - l) * inv2h;
}
inline cd d3(const cd *v, int nz, int nx, int z, int x, double inv2h) {
  const cd d = z + 1 < nz ? v[size_t(z + 1) * nx + x] : 0.0, u = z > 0 ? v[size_t(z - 1) * nx + x] : 0.0;
  return (d - u) * inv2h;
}

// Voigt strain (eps1, eps3, eps5) of u = (u1, u3): [3][nz][nx]
void strain(const Grid &g, const cd *u, cd *eps) {
  const size_t n = g.cells();
  const double f = 1.0 / (2.0 * g.h);
  const cd *u1 = u, *u3 = u + n;
  for (int z = 0; z < g.nz; ++z)
    for (int x = 0; x < g.nx; ++x) {
      const size_t o = size_t(z) * g.nx + x;
      eps[o] = d1(u1, g.nz, g.nx, z, x, f);
      eps[n + o] = d3(u3, g.nz, g.nx, z, x, f);
      eps[2 * n + o] = d3(u1, g.nz, g.nx, z, x, f) + d1(u3, g.nz, g.nx, z, x, f);
    }
}

// s = w^2 drho u + div(dC : eps(u)) with dC the contrast of the model against the reference
void contrast_source(const Grid &g, double w, const cd *u, cd *s, std::vector<cd> &eps, std::vector<cd> &sig) {
  const size_t n = g.cells();
  eps.resize(3 * n);
  sig.resize(3 * n);
  strain(g, u, eps.data());
  const double *m = g.model;
  for (size_t o = 0; o < n; ++o) {
    const double c11 = m[n + o] - g.ref[1], c13 = m[2 * n + o] - g.ref[2], c33 = m[3 * n + o] - g.ref[3],
                 c55 = m[4 * n + o] - g.ref[4];
    sig[o] = c11 * eps[o] + c13 * eps[n + o];
    sig[n + o] = c13 * eps[o] + c33 * eps[n + o];
    sig[2 * n + o] = c55 * eps[2 * n + o];
  }
  const double f = 1.0 / (2.0 * g.h);
  const cd *s1 = sig.data(), *s3 = s1 + n, *s5 = s1 + 2 * n;
  for (int z = 0; z < g.nz; ++z)
    for (int x = 0; x < g.nx; ++x) {
      const size_t o = size_t(z) * g.nx + x;
      const double wr = w * w * (m[o] - g.ref[0]);
      s[o] = wr * u[o] + d1(s1, g.nz, g.nx, z, x, f) + d3(s5, g.nz, g.nx, z, x, f);
      s[n + o] = wr * u[n + o] + d1(s5, g.nz, g.nx, z, x, f) + d3(s3, g.nz, g.nx, z, x, f);
    }
}

struct Work {
  std::vector<cd> eps, sig, s, S1, S3, col, tmp;
};

// out = h^2 G * src (Eq. 12 with the own FFT, or the direct sum)
void convolve(const Grid &g, const Freq &f, const cd *src, cd *out, bool direct, Work &wk) {
  const size_t n = g.cells();
  if (direct) {
    const int mz = 2 * g.nz - 1, mx = 2 * g.nx - 1;
    const size_t plane = size_t(mz) * mx;
    for (size_t o = 0; o < 2 * n; ++o) out[o] = 0.0;
    for (int zp = 0; zp < g.nz; ++zp)
      for (int xp = 0; xp < g.nx; ++xp) {
        const cd a1 = src[size_t(zp) * g.nx + xp], a3 = src[n + size_t(zp) * g.nx + xp];
        for (int z = 0; z < g.nz; ++z)
          for (int x = 0; x < g.nx; ++x) {
            const size_t l = size_t(z - zp + g.nz - 1) * mx + (x - xp + g.nx - 1), o = size_t(z) * g.nx + x;
            out[o] += f.lat[l] * a1 + f.lat[plane + l] * a3;
            out[n + o] += f.lat[plane + l] * a1 + f.lat[2 * plane + l] * a3;
          }
      }
    for (size_t o = 0; o < 2 * n; ++o) out[o] *= g.h * g.h;
    return;
  }
  const size_t L = size_t(g.lz) * g.lx;
  wk.S1.assign(L, 0.0);
  wk.S3.assign(L, 0.0);
  for (int z = 0; z < g.nz; ++z)
    for (int x = 0; x < g.nx; ++x) {
      wk.S1[size_t(z) * g.lx + x] = src[size_t(z) * g.nx + x];
      wk.S3[size_t(z) * g.lx + x] = src[n + size_t(z) * g.nx + x];
    }
  fft2(wk.S1.data(), g.lz, g.lx, -1, wk.col);
  fft2(wk.S3.data(), g.lz, g.lx, -1, wk.col);
  const cd *G11 = f.ghat.data(), *G13 = G11 + L, *G33 = G11 + 2 * L;
  for (size_t k = 0; k < L; ++k) {
    const cd a = wk.S1[k], b = wk.S3[k];
    wk.S1[k] = G11[k] * a + G13[k] * b;
    wk.S3[k] = G13[k] * a + G33[k] * b;
  }
  fft2(wk.S1.data(), g.lz, g.lx, +1, wk.col);
  fft2(wk.S3.data(), g.lz, g.lx, +1, wk.col);
  const double sc = g.h * g.h / double(L);
  for (int z = 0; z < g.nz; ++z)
    for (int x = 0; x < g.nx; ++x) {
      out[size_t(z) * g.nx + x] = wk.S1[size_t(z) * g.lx + x] * sc;
      out[n + size_t(z) * g.nx + x] = wk.S3[size_t(z) * g.lx + x] * sc;
    }
}

// A u = u - K(s(u))  (Eq. 10)
void apply(const Grid &g, const Freq &f, const cd *u, cd *out, bool direct, Work &wk) {
  const size_t n2 = 2 * g.cells();
  wk.s.resize(n2);
  contrast_source(g, f.w, u, wk.s.data(), wk.eps, wk.sig);
  convolve(g, f, wk.s.data(), out, direct, wk);
  for (size_t o = 0; o < n2; ++o) out[o] = u[o] - out[o];
}

cd vdot(const std::vector<cd> &a, const std::vector<cd> &b) {
  cd s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += std::conj(a[i]) * b[i];
  return s;
}
double norm(const std::vector<cd> &a) { return std::sqrt(std::real(vdot(a, a))); }

// BiCGSTAB for A x = b; returns the operator passes made (the last one checks the true residual).
int bicgstab(const Grid &g, const Freq &f, const std::vector<cd> &b, std::vector<cd> &x, double tol, int max_iter,
             bool direct, Work &wk, double *relres) {
  const size_t n2 = b.size();
  x.assign(n2, 0.0);
  const double bn = norm(b);
  int passes = 0;
  if (bn == 0.0) {
    if (relres) *relres = 0.0;
    return 0;
  }
  std::vector<cd> r = b, rhat = b, p(n2, 0.0), v(n2, 0.0), s(n2), t(n2);
  cd rho_old = 1.0, alpha = 1.0, om = 1.0;
  bool conv = norm(r) / bn <= tol;
  for (int it = 0; !conv && it < max_iter; ++it) {
    cd rho = vdot(rhat, r);
    if (std::abs(rho) < 1e-300 * bn * bn || om == 0.0) {  // breakdown: restart from the iterate
      rhat = r;
      rho = vdot(rhat, r);
      std::fill(p.begin(), p.end(), 0.0);
      std::fill(v.begin(), v.end(), 0.0);
      rho_old = alpha = om = 1.0;
    }
    const cd beta = (rho / rho_old) * (alpha / om);
    for (size_t i = 0; i < n2; ++i) p[i] = r[i] + beta * (p[i] - om * v[i]);
    apply(g, f, p.data(), v.data(), direct, wk);
    ++passes;
    alpha = rho / vdot(rhat, v);
    for (size_t i = 0; i < n2; ++i) s[i] = r[i] - alpha * v[i];
    if (norm(s) / bn <= tol) {
      for (size_t i = 0; i < n2; ++i) x[i] += alpha * p[i];
      r = s;
      conv = true;
      break;
    }
    apply(g, f, s.data(), t.data(), direct, wk);
    ++passes;
    const double tt = std::real(vdot(t, t));
    om = tt != 0.0 ? vdot(t, s) / tt : cd(0.0);
    for (size_t i = 0; i < n2; ++i) {
      x[i] += alpha * p[i] + om * s[i];
      r[i] = s[i] - om * t[i];
    }
    rho_old = rho;
    conv = norm(r) / bn <= tol;
  }
  apply(g, f, x.data(), t.data(), direct, wk);  // true residual
  ++passes;
  for (size_t i = 0; i < n2; ++i) t[i] = b[i] - t[i];
  if (relres) *relres = norm(t) / bn;
  return passes;
}

// Imaging of one problem (Eq. 32, real part): rho: Re(w^2 u_a . u_b); C11, C13, C33, C55:
// -Re(eps(u_a)^T B_p eps(u_b)) with the 2D B matrices (Appendix C restricted to {1, 3, 5}).
void imaging(const Grid &g, double w, const cd *ua, const cd *ub, double *gout, Work &wk) {
  const size_t n = g.cells();
  std::vector<cd> ea(3 * n), eb(3 * n);
  strain(g, ua, ea.data());
  strain(g, ub, eb.data());
  for (size_t o = 0; o < n; ++o) {
    gout[o] += std::real(w * w * (ua[o] * ub[o] + ua[n + o] * ub[n + o]));
    gout[n + o] -= std::real(ea[o] * eb[o]);
    gout[2 * n + o] -= std::real(ea[o] * eb[n + o] + ea[n + o] * eb[o]);
    gout[3 * n + o] -= std::real(ea[n + o] * eb[n + o]);
    gout[4 * n + o] -= std::real(ea[2 * n + o] * eb[2 * n + o]);
  }
  (void)wk;
}

Grid make_grid(int nz, int nx, double h, int lz, int lx, double rho0, double alpha0, double beta0,
               const double *model) {
  Grid g{nz, nx, lz, lx, h, rho0, alpha0, beta0, {}, model};
  const double a2 = alpha0 * alpha0, b2 = beta0 * beta0;
  g.ref[0] = rho0; g.ref[1] = rho0 * a2; g.ref[2] = rho0 * (a2 - 2.0 * b2); g.ref[3] = rho0 * a2; g.ref[4] = rho0 * b2;
  return g;
}

bool pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

// A grid, its model and the tables of its frequencies, shared by the calls below.
struct Ctx {
  Grid g;
  std::vector<double> model;
  std::vector<Freq> F;
};

int nthreads(int threads) {
#ifdef _OPENMP
  return threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

}  // namespace

extern "C" {

int orc_version(void) { return 2; }

int orc_max_threads(void) { return nthreads(0); }

// G_h on the offset lattice: out complex [3][2nz-1][2nx-1] (interleaved re, im).
int orc_green_lattice(int nz, int nx, double h, double omega, double alpha, double beta, double rho, double *out) {
  if (nz < 1 || nx < 1 || !out) return -1;
  green_lattice(nz, nx, h, omega, alpha, beta, rho, reinterpret_cast<cd *>(out));
  return 0;
}

// A context for one grid: the model [5][nz][nx] (copied), the reference medium and the Green's
// lattices and spectra of nf frequencies (built in parallel). NULL on a bad grid (FFT lengths
// must be powers of two >= 2n - 1).
void *orc_create(int nz, int nx, double h, int lz, int lx, double rho0, double alpha0, double beta0,
                 const double *model, int nf, const double *omegas, int threads) {
  if (nz < 1 || nx < 1 || nf < 1 || !pow2(lz) || !pow2(lx) || lz < 2 * nz - 1 || lx < 2 * nx - 1) return nullptr;
  Ctx *c = new Ctx;
  c->model.assign(model, model + size_t(5) * nz * nx);
  c->g = make_grid(nz, nx, h, lz, lx, rho0, alpha0, beta0, c->model.data());
  c->F.resize(nf);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads(threads))
  for (int f = 0; f < nf; ++f) make_freq(c->g, omegas[f], true, c->F[f]);
  return c;
}

void orc_destroy(void *ctx) { delete static_cast<Ctx *>(ctx); }

// A u for B problems: u, out complex [B][2][nz][nx]; problem b at frequency fidx[b]. direct = 1:
// the direct O(N^4) sum instead of the FFT (tiny grids). One problem per OpenMP thread.
int orc_apply(void *ctx, int B, const int *fidx, const double *u, double *out, int direct, int threads) {
  const Ctx *c = static_cast<const Ctx *>(ctx);
  if (!c) return -1;
  const size_t n2 = 2 * c->g.cells();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads(threads))
  for (int b = 0; b < B; ++b) {
    Work wk;
    apply(c->g, c->F[fidx[b]], reinterpret_cast<const cd *>(u) + b * n2, reinterpret_cast<cd *>(out) + b * n2,
          direct != 0, wk);
  }
  return 0;
}

// Misfit gradient of B problems (Eq. 23, 25, 32-35), one problem per OpenMP thread: incident field
// u0 = G_h(x - x_s) f, forward solve, residual r = P u - d_obs at the receivers, adjoint solve of
// A u_a = K P^T conj(r), imaging. src [B][2] cells, forces [B][2]; rec [nrec][2] cells; d_obs
// complex [B][nrec][2]. Outputs: g [5][nz][nx] summed over the problems; u complex [B][2][nz][nx]
// (or NULL); r complex [B][nrec][2] (or NULL); passes [B] operator passes (or NULL); relres [B][2]
// true relative residuals of both solves (or NULL). Returns 0.
int orc_gradient(void *ctx, int B, const int *fidx, const int *src, const double *forces, int nrec, const int *rec,
                 const double *d_obs, double tol, int max_iter, int threads, double *g_out, double *u_out,
                 double *r_out, int *passes_out, double *relres_out) {
  const Ctx *c = static_cast<const Ctx *>(ctx);
  if (!c) return -1;
  const Grid &g = c->g;
  const int nz = g.nz, nx = g.nx;
  const size_t n = g.cells(), n2 = 2 * n;
  std::vector<std::vector<double>> gparts(B);
  const cd *dobs = reinterpret_cast<const cd *>(d_obs);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads(threads))
  for (int b = 0; b < B; ++b) {
    Work wk;
    const Freq &fr = c->F[fidx[b]];
    const int mx = 2 * nx - 1;
    const size_t plane = size_t(2 * nz - 1) * mx;
    std::vector<cd> u0(n2), u, rhs(n2, 0.0), ua;
    const int zs = src[2 * b], xs = src[2 * b + 1];
    const double f1 = forces[2 * b], f3 = forces[2 * b + 1];
    for (int z = 0; z < nz; ++z)
      for (int x = 0; x < nx; ++x) {  // Eq. 7: u0(x) = G_h(x - x_s) f
        const size_t l = size_t(z - zs + nz - 1) * mx + (x - xs + nx - 1), o = size_t(z) * nx + x;
        u0[o] = fr.lat[l] * f1 + fr.lat[plane + l] * f3;
        u0[n + o] = fr.lat[plane + l] * f1 + fr.lat[2 * plane + l] * f3;
      }
    double rr[2] = {0.0, 0.0};
    int passes = bicgstab(g, fr, u0, u, tol, max_iter, false, wk, &rr[0]);
    std::vector<cd> q(n2, 0.0);
    for (int k = 0; k < nrec; ++k) {
      const size_t o = size_t(rec[2 * k]) * nx + rec[2 * k + 1];
      for (int cc = 0; cc < 2; ++cc) {
        const cd res = u[cc * n + o] - dobs[(size_t(b) * nrec + k) * 2 + cc];
        if (r_out) reinterpret_cast<cd *>(r_out)[(size_t(b) * nrec + k) * 2 + cc] = res;
        q[cc * n + o] += std::conj(res);
      }
    }
    convolve(g, fr, q.data(), rhs.data(), false, wk);
    ++passes;
    passes += bicgstab(g, fr, rhs, ua, tol, max_iter, false, wk, &rr[1]);
    gparts[b].assign(5 * n, 0.0);
    imaging(g, fr.w, ua.data(), u.data(), gparts[b].data(), wk);
    if (u_out) std::memcpy(reinterpret_cast<cd *>(u_out) + b * n2, u.data(), n2 * sizeof(cd));
    if (passes_out) passes_out[b] = passes;
    if (relres_out) { relres_out[2 * b] = rr[0]; relres_out[2 * b + 1] = rr[1]; }
  }
  for (size_t o = 0; o < 5 * n; ++o) {  // the sum over problems in problem order
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += gparts[b][o];
    g_out[o] = s;
  }
  return 0;
}

}  // extern "C"

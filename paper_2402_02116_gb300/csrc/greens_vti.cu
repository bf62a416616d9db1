// Green's tensor of a homogeneous VTI reference medium (an extension: the paper's reference is
// isotropic, Appendix A). The 2D P-SV tensor solves (C : grad grad + rho w^2) G = -I delta; in the
// wavenumber domain G^ = (Gamma(k) - rho w^2)^-1 with Gamma_ik = C_ijkl k_j k_l. Writing k = kappa n
// and Gamma(n) = sum_m lambda_m(n) P_m(n) (qP and qSV), the radial integral is exact and the
// plane-wave decomposition over slowness directions remains:
//   G(y) = 1 / (2 pi^2) int_0^pi sum_m P_m(theta) / lambda_m(theta) J(k_m(theta) |n_theta . y|) dtheta,
//   J(x) = -cos x Ci(x) - sin x Si(x) - (i pi / 2) cos x      (outgoing under exp(+i w t)),
//   k_m = w sqrt(rho / lambda_m).
// J is evaluated from the power series of Si and Ci for x < 4 and, above, from the continued
// fraction of e^z E1(z) at z = i x (Abramowitz and Stegun 5.1.22, evaluated by the modified
// Lentz method): Re(e^{ix} E1(ix)) = -cos x Ci(x) - sin x Si(x) + (pi / 2) sin x.
// Quadrature per offset y (r, phi): theta = phi + psi, psi in (-pi/2, pi/2) split at 0; on each half
// u = pi/2 - |psi| in [0, pi/2] with n . y = r sin u. The logarithmic singularity of J at u = 0 is
// integrated by the tanh-sinh rule on [0, u_s] (phase k_max r sin u_s <= 2); the rest by 16-point
// Gauss-Legendre panels over which the phase changes by at most 8 radians. The self cell takes
// the mean over the disk of area h^2: J replaced by its disk mean (tanh-sinh in the distance to
// the diameter), and a 256-point trapezoidal rule over the directions (the integrand is smooth and
// periodic there). Everything is FP64.
#include <cmath>
#include <vector>

#include "operator.cuh"

namespace dbi {

constexpr int kGL = 16;   // Gauss-Legendre points per panel
constexpr int kDE = 49;   // tanh-sinh points on [0, 1] (step 1/8, |t| <= 3)
constexpr int kSelfDirections = 256;

struct VtiQuad {
  double gl_x[kGL], gl_w[kGL];  // Gauss-Legendre on [0, 1]
  double de_x[kDE], de_w[kDE];  // tanh-sinh on [0, 1]
};

struct VtiMedium {
  double rho, c11, c13, c33, c55;
  double lam_min;  // smallest eigenvalue of Gamma(n) over the directions (bounds k_m)
};

__device__ __forceinline__ double2 zmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zinv(double2 a) {
  const double d = 1.0 / (a.x * a.x + a.y * a.y);
  return make_double2(a.x * d, -a.y * d);
}

// J(x) for x > 0 (see the file comment).
__device__ double2 spectral_j(double x) {
  double sx, cx;
  sincos(x, &sx, &cx);
  if (x < 4.0) {
    // Si = sum_k (-1)^k x^(2k+1) / ((2k+1) (2k+1)!), Ci = gamma + ln x + sum_k>=1 (-1)^k x^(2k) / (2k (2k)!)
    const double x2 = x * x;
    double t = x, si = x, u = 1.0, ci = 0.0;
    for (int k = 1; k < 40; ++k) {
      u *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
      t *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
      const double dc = u / (2.0 * k), ds = t / (2.0 * k + 1.0);
      ci += dc;
      si += ds;
      if (fabs(dc) < 1e-18 * fabs(ci) && fabs(ds) < 1e-18 * fabs(si)) break;
    }
    ci += 0.57721566490153286061 + log(x);
    return make_double2(-cx * ci - sx * si, -0.5 * M_PI * cx);
  }
  // e^z E1(z) = 1 / (z + 1 - 1 / (z + 3 - 4 / (z + 5 - 9 / ...))), z = i x
  const double tiny = 1e-300;
  double2 b = make_double2(1.0, x);
  double2 c = make_double2(1.0 / tiny, 0.0);
  double2 d = zinv(b);
  double2 hcf = d;
  for (int i = 1; i < 200; ++i) {
    const double a = -double(i) * double(i);
    b.x += 2.0;
    d = zinv(make_double2(a * d.x + b.x, a * d.y + b.y));
    const double2 ac = zmul2(make_double2(a, 0.0), zinv(c));
    c = make_double2(b.x + ac.x, b.y + ac.y);
    const double2 del = zmul2(c, d);
    hcf = zmul2(hcf, del);
    if (fabs(del.x - 1.0) + fabs(del.y) < 1e-16) break;
  }
  return make_double2(hcf.x - 0.5 * M_PI * sx, -0.5 * M_PI * cx);
}

// Eigen-decomposition of Gamma(n_theta): eigenvalues lam[0] >= lam[1], projectors P[m] as
// (11, 13, 33) entries (P[1] = I - P[0]; both I / 2 where the two eigenvalues meet).
__device__ __forceinline__ void vti_modes(const VtiMedium &M, double theta, double lam[2], double P[2][3]) {
  double s, c;
  sincos(theta, &s, &c);
  const double g11 = M.c11 * c * c + M.c55 * s * s, g33 = M.c55 * c * c + M.c33 * s * s;
  const double g13 = (M.c13 + M.c55) * c * s;
  const double mean = 0.5 * (g11 + g33), half = 0.5 * (g11 - g33), rad = hypot(half, g13);
  lam[0] = mean + rad;
  lam[1] = mean - rad;
  if (rad > 1e-13 * mean) {
    const double id = 0.5 / rad;
    P[0][0] = (g11 - lam[1]) * id;
    P[0][1] = g13 * id;
    P[0][2] = (g33 - lam[1]) * id;
  } else {
    P[0][0] = 0.5; P[0][1] = 0.0; P[0][2] = 0.5;
  }
  P[1][0] = 1.0 - P[0][0];
  P[1][1] = -P[0][1];
  P[1][2] = 1.0 - P[0][2];
}

// acc += wgt * sum_m P_m / lambda_m * J(k_m s) at direction theta.
__device__ __forceinline__ void vti_accumulate(const VtiMedium &M, double omega, double theta, double s, double wgt,
                                               double2 acc[3]) {
  double lam[2], P[2][3];
  vti_modes(M, theta, lam, P);
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const double k = omega * sqrt(M.rho / lam[m]);
    const double2 j = spectral_j(k * s);
    const double f = wgt / lam[m];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc[c].x += f * P[m][c] * j.x;
      acc[c].y += f * P[m][c] * j.y;
    }
  }
}

// G at the offset (y1, y3) != 0.
__device__ void green_vti_offset(const VtiMedium &M, const VtiQuad &Q, double omega, double y1, double y3,
                                 double2 g[3]) {
  const double r = hypot(y1, y3), phi = atan2(y3, y1);
  const double kmax = omega * sqrt(M.rho / M.lam_min);
  const double us = fmin(0.5 * M_PI, 2.0 / (kmax * r));
  double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  // both halves psi = +-(pi/2 - u) share the nodes in u
  auto point = [&](double u, double wgt) {
    const double s = r * sin(u);
    vti_accumulate(M, omega, phi + (0.5 * M_PI - u), s, wgt, acc);
    vti_accumulate(M, omega, phi - (0.5 * M_PI - u), s, wgt, acc);
  };
  for (int i = 0; i < kDE; ++i) point(us * Q.de_x[i], us * Q.de_w[i]);
  if (us < 0.5 * M_PI) {
    const double len = 0.5 * M_PI - us;
    const int np = int(ceil(len * kmax * r / 8.0));
    const double wp = len / np;
    for (int p = 0; p < np; ++p) {
      const double u0 = us + p * wp;
      for (int i = 0; i < kGL; ++i) point(u0 + wp * Q.gl_x[i], wp * Q.gl_w[i]);
    }
  }
  const double norm = 1.0 / (2.0 * M_PI * M_PI);
  for (int c = 0; c < 3; ++c) g[c] = make_double2(acc[c].x * norm, acc[c].y * norm);
}

// One thread per offset (dz, dx) >= 0 except the origin, mirrored into the four quadrant slots
// (G11, G33 even, G13 odd in each coordinate for a VTI medium), as the isotropic tabulation.
template <typename C>
__global__ void __launch_bounds__(128) k_green_vti(int nz, int nx, int lz, int lx, double h, const double *omega,
                                                   VtiMedium M, VtiQuad Q, double2 *W, C *Gspace) {
  const int dx = blockIdx.x * blockDim.x + threadIdx.x;
  const int dz = blockIdx.y, f = blockIdx.z;
  if (dx >= nx || (dz == 0 && dx == 0)) return;
  double2 g[3];
  green_vti_offset(M, Q, omega[f], dx * h, dz * h, g);
  const size_t plane = size_t(lz) * lx, base = size_t(f) * 3 * plane;
  using R = typename RealOf<C>::type;
  for (int sz = 0; sz < 2; ++sz) {
    if (sz == 1 && dz == 0) continue;
    const int iz = sz ? lz - dz : dz;
    for (int sx = 0; sx < 2; ++sx) {
      if (sx == 1 && dx == 0) continue;
      const int ix = sx ? lx - dx : dx;
      const double sg = (sz ^ sx) ? -1.0 : 1.0;
      const double2 v[3] = {g[0], make_double2(sg * g[1].x, sg * g[1].y), g[2]};
      const size_t cell = size_t(iz) * lx + ix;
      for (int c = 0; c < 3; ++c) {
        W[base + c * plane + cell] = v[c];
        if (Gspace) Gspace[base + c * plane + cell] = mk<C>(R(v[c].x), R(v[c].y));
      }
    }
  }
}

// Self cell of every frequency: one CTA of kSelfDirections threads, one direction each; the disk
// mean D(k) = 4 / (pi a^2) int_0^a J(k s) sqrt(a^2 - s^2) ds by tanh-sinh on s = a t.
template <typename C>
__global__ void __launch_bounds__(kSelfDirections) k_green_vti_self(int lz, int lx, double h, const double *omega,
                                                                    VtiMedium M, VtiQuad Q, double2 *W, C *Gspace) {
  __shared__ double sh[6][kSelfDirections];
  const int f = blockIdx.x, t = threadIdx.x;
  const double w = omega[f], a = h / sqrt(M_PI);
  const double theta = M_PI * t / kSelfDirections;
  double lam[2], P[2][3];
  vti_modes(M, theta, lam, P);
  double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int m = 0; m < 2; ++m) {
    const double k = w * sqrt(M.rho / lam[m]);
    double2 dm = make_double2(0, 0);
    for (int i = 0; i < kDE; ++i) {
      const double tt = Q.de_x[i];
      const double2 j = spectral_j(k * a * tt);
      const double wt = Q.de_w[i] * sqrt(1.0 - tt * tt);
      dm.x += wt * j.x;
      dm.y += wt * j.y;
    }
    const double f4 = 4.0 / M_PI / lam[m];
    for (int c = 0; c < 3; ++c) {
      acc[c].x += f4 * P[m][c] * dm.x;
      acc[c].y += f4 * P[m][c] * dm.y;
    }
  }
  for (int c = 0; c < 3; ++c) {
    sh[2 * c][t] = acc[c].x;
    sh[2 * c + 1][t] = acc[c].y;
  }
  __syncthreads();
  if (t < 6) {  // trapezoid over theta in [0, pi): (pi / n) sum, then 1 / (2 pi^2)
    double s = 0.0;
    for (int i = 0; i < kSelfDirections; ++i) s += sh[t][i];
    sh[t][0] = s * (M_PI / kSelfDirections) / (2.0 * M_PI * M_PI);
  }
  __syncthreads();
  if (t < 3) {
    const size_t plane = size_t(lz) * lx, idx = size_t(f) * 3 * plane + t * plane;  // slot (0, 0)
    const double2 v = t == 1 ? make_double2(0.0, 0.0) : make_double2(sh[2 * t][0], sh[2 * t + 1][0]);
    W[idx] = v;
    using R = typename RealOf<C>::type;
    if (Gspace) Gspace[idx] = mk<C>(R(v.x), R(v.y));
  }
}

// Host: quadrature rules from their definitions (Gauss-Legendre nodes by Newton's method on the
// Legendre polynomial, tanh-sinh nodes u = (1 + tanh(pi/2 sinh t)) / 2 written without cancellation).
static VtiQuad make_quad() {
  VtiQuad Q{};
  const int n = kGL;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    Q.gl_x[i] = 0.5 * (1.0 - x);  // [-1, 1] -> [0, 1]
    Q.gl_w[i] = 1.0 / ((1.0 - x * x) * dp * dp);  // (2 / ((1 - x^2) P'^2)) / 2
  }
  const double hstep = 0.125;
  for (int i = 0; i < kDE; ++i) {
    const double t = (i - (kDE - 1) / 2) * hstep;
    const double q = 0.5 * M_PI * std::sinh(t);
    Q.de_x[i] = 1.0 / (1.0 + std::exp(-2.0 * q));
    const double ch = std::cosh(q);
    Q.de_w[i] = hstep * 0.25 * M_PI * std::cosh(t) / (ch * ch);
  }
  return Q;
}

static VtiMedium make_medium(const dbi_medium &r) {
  VtiMedium M{r.rho0, r.c11, r.c13, r.c33, r.c55, 0.0};
  double lmin = 1e300;
  for (int i = 0; i < 3600; ++i) {  // the qSV eigenvalue's minimum over the directions
    const double th = M_PI * i / 3600.0, c = std::cos(th), s = std::sin(th);
    const double g11 = r.c11 * c * c + r.c55 * s * s, g33 = r.c55 * c * c + r.c33 * s * s;
    const double g13 = (r.c13 + r.c55) * c * s;
    lmin = std::fmin(lmin, 0.5 * (g11 + g33) - std::hypot(0.5 * (g11 - g33), g13));
  }
  M.lam_min = 0.98 * lmin;
  return M;
}

int launch_green_vti(const dbi_grid *g, const dbi_medium &ref, const double *omega, int nf, double2 *W,
                     void *Gspace, int precision, cudaStream_t s) {
  static const VtiQuad Q = make_quad();
  const VtiMedium M = make_medium(ref);
  const dim3 grid((g->nx + 127) / 128, g->nz, nf);
  if (precision == DBI_C64) {
    k_green_vti<float2><<<grid, 128, 0, s>>>(g->nz, g->nx, g->lz, g->lx, g->h, omega, M, Q, W,
                                             static_cast<float2 *>(Gspace));
  } else {
    k_green_vti<double2><<<grid, 128, 0, s>>>(g->nz, g->nx, g->lz, g->lx, g->h, omega, M, Q, W,
                                              static_cast<double2 *>(Gspace));
  }
  int rc = check_launch("k_green_vti");
  if (rc) return rc;
  if (precision == DBI_C64)
    k_green_vti_self<float2><<<nf, kSelfDirections, 0, s>>>(g->lz, g->lx, g->h, omega, M, Q, W,
                                                            static_cast<float2 *>(Gspace));
  else
    k_green_vti_self<double2><<<nf, kSelfDirections, 0, s>>>(g->lz, g->lx, g->h, omega, M, Q, W,
                                                             static_cast<double2 *>(Gspace));
  return check_launch("k_green_vti_self");
}

}  // namespace dbi

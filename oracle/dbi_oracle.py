"""Plain, slow, FP64 CPU oracle for the 2D elastic Lippmann-Schwinger (LS) operator and the
matrix-free distorted-Born products built on it (arXiv 2402.02116).

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU-baseline leg
may import this module. The library's CUDA path never imports, links or calls it, and this
module imports nothing from the library: the two share no code.

Everything is complex128 / float64 numpy, written for readability. Library routines used as
single steps: scipy.special.hankel2 (Hankel functions of the second kind) and numpy.fft.fft2/ifft2.

Discrete problem (the paper states the continuous equations; the readings below fill what it
leaves unstated):
  * Reference medium: homogeneous isotropic (rho0, alpha0, beta0); contrast = model - reference
    (Eq. 4). 2D P-SV restriction of the Voigt/VTI stiffness (Eq. 36, 39) to indices {1, 3, 5}.
  * Green's tensor: the 2D closed form of Appendix A (Eq. A-3, A-4), time convention e^{+i w t}
    (H^(2) outgoing). Midpoint quadrature at cell-centre offsets; the self cell uses the average
    of G over the disk of area h^2 (the B term averages to zero there).
  * Derivatives: central differences with the field taken as zero outside the grid, used both
    for the strain of u and for the divergence of the stress (the finite-difference reading of
    Eq. 6 and Eq. 9, Section "Forward modeling").
  * LS operator (Eq. 10, 11): A u = u - h^2 sum_x' G_h(x - x') s(x'),
    s = w^2 drho u + div(dC : eps(u)).
  * Convolution by FFT on a zero-padded lz x lx grid (Eq. 12), lz >= 2 nz - 1, lx >= 2 nx - 1.
  * Krylov: BiCGSTAB with <a, b> = sum conj(a) b, x0 = 0, shadow residual r0; and restarted
    GMRES(m), the solver of the paper's experiments (restart length unstated: m = 30 by default).
  * Frechet (Eq. 20, 26-31): J dm = P A_b^{-1} G (w^2 dm_rho u_b + div(dC(dm) : eps(u_b))), the two
    virtual sources Y and M of Eq. 26 merged into one source by linearity.
  * Adjoint (Eq. 25, 32-35): u_a = A_b^{-1} G P^T conj(r);
    (Re J^H r)_rho = Re(w^2 u_a . u_b), (Re J^H r)_p = -Re(eps(u_a)^T B_p eps(u_b)).
  * Normal equation (Eq. 23, 24): (Re J^H J + lambda I) dm = Re J^H du by CG on relative unknowns.

Pins (tests/test_oracle_pins.py): besides invariants (zero contrast, Born series, reciprocity,
dense solve, finite-difference derivatives), the assembled LS solution is tied to the physics: its
finite-difference residual of the heterogeneous elastic equation falls as O(h^2) under grid
refinement, and the offset lattice's orientation is fixed by the P and S phase rates along each
axis of a non-square lattice. The paper prints no wavefield or data values.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad_vec
from scipy.special import hankel2, sici

# Parameter order: rho, C11, C13, C33, C55.
N_PARAMS = 5


# ---------------------------------------------------------------------------------------------
# Reference medium and contrast (Eq. 4, Eq. 39)
# ---------------------------------------------------------------------------------------------
def reference_params(rho0, alpha0, beta0) -> np.ndarray:
    """(rho, C11, C13, C33, C55) of the homogeneous isotropic reference medium:
    C11 = C33 = rho alpha^2, C13 = rho (alpha^2 - 2 beta^2), C55 = rho beta^2."""
    a2, b2 = alpha0 * alpha0, beta0 * beta0
    return np.array([rho0, rho0 * a2, rho0 * (a2 - 2.0 * b2), rho0 * a2, rho0 * b2])


def contrast(model, rho0, alpha0, beta0) -> np.ndarray:
    """delta rho, delta C of Eq. 4: the model minus the homogeneous reference, per cell."""
    return np.asarray(model, dtype=np.float64) - reference_params(rho0, alpha0, beta0)[:, None, None]


def voigt_2d(c11, c13, c33, c55) -> np.ndarray:
    """The 2D P-SV part (rows/columns 1, 3, 5) of the VTI stiffness matrix of Eq. 39."""
    return np.array([[c11, c13, 0.0], [c13, c33, 0.0], [0.0, 0.0, c55]])


# ---------------------------------------------------------------------------------------------
# Green's tensor (Appendix A, Eq. A-3 and A-4)
# ---------------------------------------------------------------------------------------------
def green_2d(y1, y3, omega, alpha, beta, rho):
    """Closed-form 2D isotropic Green's tensor at offsets y = (y1, y3) != 0.

    G_ij = 1/(8 i rho) [A delta_ij - B (2 g_i g_j - delta_ij)],
    A = H0(w r/alpha)/alpha^2 + H0(w r/beta)/beta^2, B = H2(w r/alpha)/alpha^2 - H2(w r/beta)/beta^2,
    with H_n = H_n^(2) and g = y / r. Returns (G11, G13, G33)."""
    y1 = np.asarray(y1, dtype=np.float64)
    y3 = np.asarray(y3, dtype=np.float64)
    r = np.hypot(y1, y3)
    g1 = y1 / r
    g3 = y3 / r
    za = omega * r / alpha
    zb = omega * r / beta
    A = hankel2(0, za) / alpha ** 2 + hankel2(0, zb) / beta ** 2
    B = hankel2(2, za) / alpha ** 2 - hankel2(2, zb) / beta ** 2
    pref = 1.0 / (8j * rho)
    G11 = pref * (A - B * (2.0 * g1 * g1 - 1.0))
    G33 = pref * (A - B * (2.0 * g3 * g3 - 1.0))
    G13 = pref * (-B * 2.0 * g1 * g3)
    return G11, G13, G33


def green_self_cell(h, omega, alpha, beta, rho):
    """Average of G over the disk of radius a = h / sqrt(pi) centred on the source (the self cell).

    The B term has zero angular mean, so only A contributes. With
    int_0^a H0(k r) r dr = a H1(k a)/k - 2i/(pi k^2), the disk mean of H0(k r) is
    2 H1(k a)/(k a) - 4i/(pi k^2 a^2). Returns (G11, G13, G33) with G13 = 0."""
    a = h / math.sqrt(math.pi)
    total = 0.0 + 0.0j
    for c in (alpha, beta):
        k = omega / c
        mean_h0 = 2.0 * hankel2(1, k * a) / (k * a) - 4.0j / (math.pi * k * k * a * a)
        total += mean_h0 / (c * c)
    g = total / (8j * rho)
    return g, 0.0 + 0.0j, g


def green_lattice(nz, nx, h, omega, alpha, beta, rho) -> np.ndarray:
    """G_h on the (2nz-1) x (2nx-1) lattice of cell-centre offsets; entry [c][dz+nz-1][dx+nx-1]
    holds component c (0: G11, 1: G13, 2: G33) at offset (y1, y3) = (dx h, dz h)."""
    dz = np.arange(-(nz - 1), nz)[:, None] * np.ones((1, 2 * nx - 1))
    dx = np.ones((2 * nz - 1, 1)) * np.arange(-(nx - 1), nx)[None, :]
    y1 = dx * h
    y3 = dz * h
    origin = (dz == 0) & (dx == 0)
    y1s = np.where(origin, 1.0, y1)  # placeholder, overwritten below
    y3s = np.where(origin, 1.0, y3)
    G11, G13, G33 = green_2d(y1s, y3s, omega, alpha, beta, rho)
    s11, s13, s33 = green_self_cell(h, omega, alpha, beta, rho)
    G11 = np.where(origin, s11, G11)
    G13 = np.where(origin, s13, G13)
    G33 = np.where(origin, s33, G33)
    return np.stack([G11, G13, G33]).astype(np.complex128)


# ---------------------------------------------------------------------------------------------
# Homogeneous VTI reference: Green's tensor by its spectral representation (not in the paper)
# ---------------------------------------------------------------------------------------------
def christoffel_2d(n1, n3, c11, c13, c33, c55):
    """Gamma_ik(n) = C_ijkl n_j n_l of the 2D VTI stiffness: entries (11, 13, 33)."""
    return (c11 * n1 * n1 + c55 * n3 * n3, (c13 + c55) * n1 * n3, c55 * n1 * n1 + c33 * n3 * n3)


def spectral_radial(x):
    """J(a, s) = int_0^inf k cos(k s) / (k^2 - a^2) dk for a -> a - i0 (outgoing waves under
    exp(+i w t)), as a function of x = a s > 0: -cos x Ci(x) - sin x Si(x) - (i pi / 2) cos x."""
    si_x, ci_x = sici(x)
    return -np.cos(x) * ci_x - np.sin(x) * si_x - 0.5j * np.pi * np.cos(x)


def _modes(theta, rho, omega, c11, c13, c33, c55):
    """Eigenvalues lambda_m of Gamma(n_theta), their projectors P_m (as 11, 13, 33 entries) and the
    wavenumbers k_m = w sqrt(rho / lambda_m), m = qP, qSV."""
    n1, n3 = np.cos(theta), np.sin(theta)
    g11, g13, g33 = christoffel_2d(n1, n3, c11, c13, c33, c55)
    mean, half = 0.5 * (g11 + g33), 0.5 * (g11 - g33)
    rad = np.hypot(half, g13)
    out = []
    for lam, other in ((mean + rad, mean - rad), (mean - rad, mean + rad)):
        d = lam - other
        P = ((g11 - other) / d, g13 / d, (g33 - other) / d)
        out.append((lam, P, omega * np.sqrt(rho / lam)))
    return out


def green_vti_2d(y1, y3, omega, rho, c11, c13, c33, c55, epsabs=1e-16, epsrel=1e-13):
    """2D Green's tensor of a homogeneous VTI medium at the offset y = (y1, y3) != 0, from
    (Gamma(k) - rho w^2)^-1 inverted over k in polar coordinates (the plane-wave decomposition
    over slowness directions of anisotropic elastodynamics):

        G(y) = 1 / (2 pi^2) int_0^pi sum_m P_m(theta) / lambda_m(theta) J(k_m(theta), |n_theta . y|) dtheta

    with Gamma(n) = sum_m lambda_m P_m. Integrated by scipy's adaptive quadrature over
    psi = theta - phi in (-pi/2, pi/2) (phi the direction of y), so the logarithmic singularity of J
    at n . y = 0 sits at the ends, with breakpoints every few radians of the largest phase k r. The
    integrand is scaled by C55 to order one, so that the absolute tolerance is relative to the
    integral's size; a quadrature that runs out of subdivisions raises. Returns (G11, G13, G33)."""
    r = math.hypot(y1, y3)
    phi = math.atan2(y3, y1)

    def integrand(psi):
        theta = phi + psi
        s = r * math.cos(psi)
        v = np.zeros(6)
        for lam, P, k in _modes(theta, rho, omega, c11, c13, c33, c55):
            j = spectral_radial(k * s) * (c55 / lam)
            for c in range(3):
                v[2 * c] += (P[c] * j).real
                v[2 * c + 1] += (P[c] * j).imag
        return v

    lam_min = min(m[0] for t in np.linspace(0.0, math.pi, 721) for m in _modes(t, rho, omega, c11, c13, c33, c55))
    pieces = max(4, int(math.ceil(omega * math.sqrt(rho / lam_min) * r / 4.0)))
    points = list(np.linspace(-0.5 * math.pi, 0.5 * math.pi, pieces + 1)[1:-1])
    val, _, info = quad_vec(integrand, -0.5 * math.pi, 0.5 * math.pi, epsabs=epsabs, epsrel=epsrel,
                            limit=20000, points=points, full_output=True)
    if info.status == 1:  # subdivision limit (status 2, rounding at the tolerance, is accepted)
        raise RuntimeError(f"VTI Green's tensor quadrature did not converge at y = ({y1}, {y3}): {info.message}")
    g = (val[0::2] + 1j * val[1::2]) / (2.0 * math.pi * math.pi * c55)
    return g[0], g[1], g[2]


def green_vti_self_cell(h, omega, rho, c11, c13, c33, c55):
    """Mean of the VTI Green's tensor over the disk of area h^2 (radius a = h / sqrt(pi)): the
    spectral representation with J replaced by its disk mean
    D(k) = 4 / (pi a^2) int_0^a J(k, s) sqrt(a^2 - s^2) ds (a function of n . y only)."""
    a = h / math.sqrt(math.pi)

    def disk_mean(k):
        def f(t):  # s = a t
            j = spectral_radial(k * a * t) * math.sqrt(1.0 - t * t)
            return np.array([j.real, j.imag])
        v, _ = quad_vec(f, 0.0, 1.0, epsabs=1e-15, epsrel=1e-12, limit=500)
        return (4.0 / math.pi) * (v[0] + 1j * v[1])

    def integrand(theta):
        v = np.zeros(6)
        for lam, P, k in _modes(theta, rho, omega, c11, c13, c33, c55):
            d = disk_mean(k) * (c55 / lam)
            for c in range(3):
                v[2 * c] += (P[c] * d).real
                v[2 * c + 1] += (P[c] * d).imag
        return v

    val, _ = quad_vec(integrand, 0.0, math.pi, epsabs=1e-15, epsrel=1e-11, limit=200)
    g = (val[0::2] + 1j * val[1::2]) / (2.0 * math.pi * math.pi * c55)
    return g[0], g[1], g[2]


def green_lattice_vti(nz, nx, h, omega, rho, c11, c13, c33, c55, epsrel=1e-13) -> np.ndarray:
    """G_h of the VTI reference on the (2nz-1) x (2nx-1) offset lattice ([c][dz+nz-1][dx+nx-1], as
    green_lattice). Only the quadrant dz, dx >= 0 is integrated: the mirror symmetries of a VTI
    medium make G11, G33 even and G13 odd in each of x1 and x3."""
    out = np.zeros((3, 2 * nz - 1, 2 * nx - 1), dtype=np.complex128)
    for dz in range(nz):
        for dx in range(nx):
            if dz == 0 and dx == 0:
                g = green_vti_self_cell(h, omega, rho, c11, c13, c33, c55)
            else:
                g = green_vti_2d(dx * h, dz * h, omega, rho, c11, c13, c33, c55, epsabs=1e-3 * epsrel,
                                 epsrel=epsrel)
            for sz in ((1, -1) if dz else (1,)):
                for sx in ((1, -1) if dx else (1,)):
                    iz, ix = nz - 1 + sz * dz, nx - 1 + sx * dx
                    out[0, iz, ix] = g[0]
                    out[1, iz, ix] = g[1] * sz * sx
                    out[2, iz, ix] = g[2]
    return out


# ---------------------------------------------------------------------------------------------
# Finite-difference strain, stress and divergence (Eq. 6, Eq. 38)
# ---------------------------------------------------------------------------------------------
def d1(v, h):
    """Central difference along x1 (last axis), v taken as zero outside the grid."""
    p = np.zeros(v.shape[:-1] + (v.shape[-1] + 2,), dtype=v.dtype)
    p[..., 1:-1] = v
    return (p[..., 2:] - p[..., :-2]) / (2.0 * h)


def d3(v, h):
    """Central difference along x3 (second-to-last axis), v taken as zero outside the grid."""
    p = np.zeros(v.shape[:-2] + (v.shape[-2] + 2, v.shape[-1]), dtype=v.dtype)
    p[..., 1:-1, :] = v
    return (p[..., 2:, :] - p[..., :-2, :]) / (2.0 * h)


def strain(u, h):
    """Voigt strain (eps1, eps3, eps5) = (du1/dx1, du3/dx3, du1/dx3 + du3/dx1), Eq. 38."""
    u1, u3 = u[0], u[1]
    return np.stack([d1(u1, h), d3(u3, h), d3(u1, h) + d1(u3, h)])


def stress(eps, dmodel):
    """sigma = dC eps with the 2D Voigt dC = [[dC11, dC13, 0], [dC13, dC33, 0], [0, 0, dC55]]."""
    c11, c13, c33, c55 = dmodel[1], dmodel[2], dmodel[3], dmodel[4]
    return np.stack([c11 * eps[0] + c13 * eps[1],
                     c13 * eps[0] + c33 * eps[1],
                     c55 * eps[2]])


def divergence(sig, h):
    """(div sigma)_1 = d1 sig1 + d3 sig5, (div sigma)_3 = d1 sig5 + d3 sig3."""
    return np.stack([d1(sig[0], h) + d3(sig[2], h),
                     d1(sig[2], h) + d3(sig[1], h)])


def contrast_source(u, dmodel, omega, h):
    """s = w^2 drho u + div(dC : grad u), the integrand source of Eq. 6 (dmodel = contrast)."""
    return omega * omega * dmodel[0] * u + divergence(stress(strain(u, h), dmodel), h)


# ---------------------------------------------------------------------------------------------
# Convolution with the Green's tensor (Eq. 6, Eq. 12)
# ---------------------------------------------------------------------------------------------
def convolve_direct(s, G_lat, h):
    """K s (x) = h^2 sum_{x' in D} G_h(x - x') s(x'), summed directly (O(N^4); tiny grids only)."""
    _, nz, nx = s.shape
    out = np.zeros((2, nz, nx), dtype=np.complex128)
    for izp in range(nz):
        for ixp in range(nx):
            win = G_lat[:, nz - 1 - izp: 2 * nz - 1 - izp, nx - 1 - ixp: 2 * nx - 1 - ixp]
            s1, s3 = s[0, izp, ixp], s[1, izp, ixp]
            out[0] += win[0] * s1 + win[1] * s3
            out[1] += win[1] * s1 + win[2] * s3
    return h * h * out


def embed_circulant(G_lat, lz, lx):
    """Place the offset lattice on an lz x lx periodic grid: offset d goes to slot d mod L.
    Needs lz >= 2nz - 1 and lx >= 2nx - 1 so that no two offsets share a slot."""
    _, mz, mx = G_lat.shape
    nz, nx = (mz + 1) // 2, (mx + 1) // 2
    assert lz >= 2 * nz - 1 and lx >= 2 * nx - 1
    P = np.zeros((3, lz, lx), dtype=np.complex128)
    dz = np.arange(-(nz - 1), nz) % lz
    dx = np.arange(-(nx - 1), nx) % lx
    P[:, dz[:, None], dx[None, :]] = G_lat
    return P


def green_spectrum(G_lat, lz, lx):
    """FFT of the circulant embedding (the FFT{G} factor of Eq. 12)."""
    return np.fft.fft2(embed_circulant(G_lat, lz, lx), axes=(-2, -1))


def convolve_fft(s, G_hat, h):
    """K s by Eq. 12: zero-pad s to lz x lx, multiply its FFT by the 2x2 spectrum, invert, crop."""
    _, nz, nx = s.shape
    _, lz, lx = G_hat.shape
    sp = np.zeros((2, lz, lx), dtype=np.complex128)
    sp[:, :nz, :nx] = s
    S = np.fft.fft2(sp, axes=(-2, -1))
    O1 = G_hat[0] * S[0] + G_hat[1] * S[1]
    O3 = G_hat[1] * S[0] + G_hat[2] * S[1]
    o = np.fft.ifft2(np.stack([O1, O3]), axes=(-2, -1))
    return h * h * o[:, :nz, :nx]


# ---------------------------------------------------------------------------------------------
# Paper-literal form: the derivative on the Green's tensor (Eq. 9)
# ---------------------------------------------------------------------------------------------
# Eq. 9 integrates the stress term by parts so that the derivative falls on G: the operator is
#   A u = u - [ w^2 G * (drho u) + (grad G) * sigma ],  (grad G * sigma)_i = sum_jk d_k G_ij sigma_jk,
# sigma = dC : eps(u) (the sign: grad_x' G(x - x') = -(grad G)(x - x')). The derivatives of G are
# the central differences of the lattice G_h, (D_k G)(y) = [G_h(y + h e_k) - G_h(y - h e_k)] / 2h,
# which needs G_h one ring beyond the (2N-1)^2 offsets. For stress that vanishes on the outer ring
# of D this equals the form above term by term (summation by parts); it differs next to the
# boundary of D.
def green_derivative_lattice(nz, nx, h, omega, alpha, beta, rho) -> np.ndarray:
    """(D_k G_h) on the (2nz-1) x (2nx-1) offsets: [6][dz+nz-1][dx+nx-1] holding D1 G11, D1 G13,
    D1 G33, D3 G11, D3 G13, D3 G33 (D1 along x1, the last axis; D3 along x3)."""
    Ge = green_lattice(nz + 1, nx + 1, h, omega, alpha, beta, rho)  # offsets -nz..nz, -nx..nx
    d1g = (Ge[:, 1:-1, 2:] - Ge[:, 1:-1, :-2]) / (2.0 * h)
    d3g = (Ge[:, 2:, 1:-1] - Ge[:, :-2, 1:-1]) / (2.0 * h)
    return np.concatenate([d1g, d3g]).astype(np.complex128)


def form_k_sources(u, dmodel, omega, h):
    """The five fields convolved in Eq. 9: w^2 drho u1, w^2 drho u3, sigma1, sigma5, sigma3."""
    s = omega * omega * dmodel[0] * u
    sig = stress(strain(u, h), dmodel)
    return np.stack([s[0], s[1], sig[0], sig[2], sig[1]])


# Rows of the 2 x 5 kernel of Eq. 9 over the sources (s1, s3, sigma1, sigma5, sigma3), as
# (table, index) pairs summed per entry: table "G" = green_lattice, "D" = green_derivative_lattice.
FORM_K_KERNEL = (
    ((("G", 0),), (("G", 1),), (("D", 0),), (("D", 3), ("D", 1)), (("D", 4),)),
    ((("G", 1),), (("G", 2),), (("D", 1),), (("D", 4), ("D", 2)), (("D", 5),)),
)


def form_k_direct(src, G_lat, DG_lat, h):
    """h^2 sum_{x' in D} K(x - x') src(x') for the 2 x 5 kernel of Eq. 9, summed directly."""
    _, nz, nx = src.shape
    out = np.zeros((2, nz, nx), dtype=np.complex128)
    tables = {"G": G_lat, "D": DG_lat}
    for izp in range(nz):
        for ixp in range(nx):
            sl = (slice(nz - 1 - izp, 2 * nz - 1 - izp), slice(nx - 1 - ixp, 2 * nx - 1 - ixp))
            for i in range(2):
                for c in range(5):
                    ker = sum(tables[t][k][sl] for t, k in FORM_K_KERNEL[i][c])
                    out[i] += ker * src[c, izp, ixp]
    return h * h * out


def form_k_spectra(G_lat, DG_lat, lz, lx):
    """FFTs of the circulant embeddings of the nine distinct kernel entries, as [2][5] spectra."""
    G_hat = green_spectrum(G_lat, lz, lx)
    D_hat = np.concatenate([green_spectrum(DG_lat[0:3], lz, lx), green_spectrum(DG_lat[3:6], lz, lx)])
    tables = {"G": G_hat, "D": D_hat}
    return [[sum(tables[t][k] for t, k in FORM_K_KERNEL[i][c]) for c in range(5)] for i in range(2)]


def form_k_fft(src, K_hat, h):
    """The same convolution by Eq. 12 on the zero-padded grid."""
    _, nz, nx = src.shape
    lz, lx = K_hat[0][0].shape
    sp = np.zeros((5, lz, lx), dtype=np.complex128)
    sp[:, :nz, :nx] = src
    S = np.fft.fft2(sp, axes=(-2, -1))
    O = np.stack([sum(K_hat[i][c] * S[c] for c in range(5)) for i in range(2)])
    o = np.fft.ifft2(O, axes=(-2, -1))
    return h * h * o[:, :nz, :nx]


# ---------------------------------------------------------------------------------------------
# Krylov solver
# ---------------------------------------------------------------------------------------------
def bicgstab(apply, b, tol=1e-12, maxiter=2000, x0=None):
    """BiCGSTAB (van der Vorst 1992) for a complex system, <a, b> = sum conj(a) b.
    Stops when ||b - A x|| / ||b|| <= tol (recursive residual, re-checked on exit).
    Returns (x, info) with info = dict(iters, relres, converged)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, relres=0.0, converged=True)
    r = b - apply(x)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0.0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    converged = np.linalg.norm(r) / bnorm <= tol
    while not converged and it < maxiter:
        it += 1
        rho = np.vdot(rhat, r)
        if abs(rho) < 1e-300 * bnorm * bnorm or omega == 0:
            rhat = r.copy()
            rho = np.vdot(rhat, r)
            p[...] = 0
            v[...] = 0
            rho_old = alpha = omega = 1.0 + 0.0j
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        if np.linalg.norm(s) / bnorm <= tol:
            x = x + alpha * p
            r = s
            converged = True
            break
        t = apply(s)
        tt = np.vdot(t, t)
        omega = np.vdot(t, s) / tt if tt != 0 else 0.0
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        converged = np.linalg.norm(r) / bnorm <= tol
    relres = np.linalg.norm(b - apply(x)) / bnorm
    return x, dict(iters=it, relres=float(relres), converged=bool(converged))


# ---------------------------------------------------------------------------------------------
# The LS problem on one grid with a set of frequencies
def givens(a, b):
    """Complex plane rotation [[c, s], [-conj(s), c]] (c real) that maps (a, b) to (r, 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, np.conj(b) / abs(b), abs(b)
    t = math.hypot(abs(a), abs(b))
    phase = a / abs(a)
    return abs(a) / t, phase * np.conj(b) / t, phase * t


def gmres(apply, b, restart=30, tol=1e-12, maxiter=2000, x0=None):
    """Restarted GMRES(m) (Saad and Schultz 1986), <a, b> = sum conj(a) b.

    One cycle from x0 with r0 = b - A x0, beta = ||r0||: Arnoldi with modified Gram-Schmidt builds
    the orthonormal basis v_1 = r0 / beta, v_2, ... of the Krylov space and the Hessenberg matrix
    H with A V_k = V_(k+1) H_k; the iterate x0 + V_k y minimises ||beta e_1 - H_k y||, which equals
    ||b - A x|| over x0 + span(V_k). Plane rotations reduce H_k to triangular form as it grows, so
    the minimal residual after k steps is the last entry |g_(k+1)| of the rotated right-hand side.
    A cycle stops after `restart` steps, when |g_(k+1)| <= tol ||b||, or when the new basis
    vector vanishes (the solution lies in the space built so far); then y is found by back
    substitution, x = x0 + V_k y, and the next cycle starts from x.

    Returns (x, info): iters = Arnoldi steps (operator applications inside the cycles), relres =
    the true relative residual of the returned x, resvec = the minimal residual after every step
    (relative to ||b||), converged."""
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, relres=0.0, resvec=[], converged=True)
    it = 0
    resvec = []
    converged = False
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            converged = True
            break
        if it >= maxiter:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(restart):
            if it >= maxiter:
                break
            w = apply(V[j])
            it += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):  # earlier rotations on the new column
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            cs[j], sn[j], H[j, j] = givens(H[j, j], H[j + 1, j])
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            resvec.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= tol * bnorm or hn == 0.0:
                break
            V.append(w / hn)
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):  # back substitution with the triangular H
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * V[i]
    relres = np.linalg.norm(b - apply(x)) / bnorm
    return x, dict(iters=it, relres=float(relres), resvec=resvec, converged=bool(converged))


# ---------------------------------------------------------------------------------------------
class LSOracle:
    """Discrete LS operator, forward solves and distorted-Born products for one grid.

    nz, nx, h: grid; lz, lx: FFT grid; rho0, alpha0, beta0: reference medium; omegas: angular
    frequencies (rad/s). method = "fft" (Eq. 12) or "direct" (plain O(N^4) sum)."""

    def __init__(self, nz, nx, h, lz, lx, rho0, alpha0, beta0, omegas, method="fft", ref_vti=None,
                 vti_epsrel=1e-13):
        self.nz, self.nx, self.h, self.lz, self.lx = nz, nx, float(h), lz, lx
        self.rho0, self.alpha0, self.beta0 = float(rho0), float(alpha0), float(beta0)
        self.omegas = np.asarray(omegas, dtype=np.float64)
        self.method = method
        # reference (rho, C11, C13, C33, C55): isotropic from (rho0, alpha0, beta0), or the
        # homogeneous VTI medium ref_vti with its spectral Green's tensor
        if ref_vti is None:
            self.ref = reference_params(rho0, alpha0, beta0)
            self.G_lat = [green_lattice(nz, nx, h, w, alpha0, beta0, rho0) for w in self.omegas]
        else:
            self.ref = np.asarray(ref_vti, dtype=np.float64)
            self.G_lat = [green_lattice_vti(nz, nx, h, w, *self.ref, epsrel=vti_epsrel) for w in self.omegas]
        self.G_hat = [green_spectrum(G, lz, lx) for G in self.G_lat]

    # --- Eq. 6 / Eq. 12 convolution --------------------------------------------------------
    def convolve(self, s, f):
        if self.method == "direct":
            return convolve_direct(s, self.G_lat[f], self.h)
        return convolve_fft(s, self.G_hat[f], self.h)

    # --- Eq. 10: A u = u - K(w^2 drho u + div(dC : grad u)) ------------------------------------
    def apply(self, u, model, f):
        dmod = np.asarray(model, dtype=np.float64) - self.ref[:, None, None]
        return u - self.convolve(contrast_source(u, dmod, self.omegas[f], self.h), f)

    # --- Eq. 9 (derivatives on G): A_K u = u - [w^2 G * (drho u) + (grad G) * sigma] -----------
    def apply_k(self, u, model, f):
        if not hasattr(self, "K_hat"):
            self.K_hat = [form_k_spectra(G, green_derivative_lattice(self.nz, self.nx, self.h, w, self.alpha0,
                                                                     self.beta0, self.rho0), self.lz, self.lx)
                          for G, w in zip(self.G_lat, self.omegas)]
        dmod = contrast(model, self.rho0, self.alpha0, self.beta0)
        return u - form_k_fft(form_k_sources(u, dmod, self.omegas[f], self.h), self.K_hat[f], self.h)

    def solve_k(self, rhs, model, f, tol=1e-12, maxiter=3000):
        shape = rhs.shape
        x, _ = bicgstab(lambda v: self.apply_k(v.reshape(shape), model, f).ravel(), rhs.ravel(), tol=tol,
                        maxiter=maxiter)
        return x.reshape(shape)

    # --- Eq. 7: incident field of a point force f at cell x_s: u0(x) = G_h(x - x_s) f ------------
    def incident(self, f, src_cell, force):
        iz, ix = int(src_cell[0]), int(src_cell[1])
        nz, nx = self.nz, self.nx
        win = self.G_lat[f][:, nz - 1 - iz: 2 * nz - 1 - iz, nx - 1 - ix: 2 * nx - 1 - ix]
        f1, f3 = force
        return np.stack([win[0] * f1 + win[1] * f3, win[1] * f1 + win[2] * f3]).astype(np.complex128)

    # --- Eq. 11 solved by BiCGSTAB -------------------------------------------------------------
    def solve(self, rhs, model, f, tol=1e-12, maxiter=3000):
        shape = rhs.shape
        return bicgstab(lambda v: self.apply(v.reshape(shape), model, f).reshape(-1),
                        rhs.reshape(-1), tol=tol, maxiter=maxiter)[0].reshape(shape)

    def solve_gmres(self, rhs, model, f, restart=30, tol=1e-12, maxiter=3000):
        """A u = rhs by GMRES(restart), the paper's Krylov solver; returns (u, info)."""
        shape = rhs.shape
        x, info = gmres(lambda v: self.apply(v.reshape(shape), model, f).reshape(-1), rhs.reshape(-1),
                        restart=restart, tol=tol, maxiter=maxiter)
        return x.reshape(shape), info

    def solve_info(self, rhs, model, f, tol=1e-12, maxiter=3000):
        shape = rhs.shape
        x, info = bicgstab(lambda v: self.apply(v.reshape(shape), model, f).reshape(-1),
                           rhs.reshape(-1), tol=tol, maxiter=maxiter)
        return x.reshape(shape), info

    def forward(self, model, fidx, src_cells, forces, tol=1e-12):
        """Wavefields u[b] = A^{-1} u0[b] for every problem b (frequency fidx[b], source b's)."""
        U = np.zeros((len(fidx), 2, self.nz, self.nx), dtype=np.complex128)
        for b, f in enumerate(fidx):
            u0 = self.incident(f, src_cells[b], forces[b])
            U[b] = self.solve(u0, model, f, tol=tol)
        return U

    # --- receivers --------------------------------------------------------------------------
    @staticmethod
    def sample(u, rec_cells):
        """P u: both components at the receiver cells, [n_rec][2]."""
        return np.stack([u[:, iz, ix] for iz, ix in rec_cells])

    def inject(self, q, rec_cells):
        """P^T q: a field that holds q[r] at receiver cell r (summed where receivers coincide)."""
        out = np.zeros((2, self.nz, self.nx), dtype=np.complex128)
        for k, (iz, ix) in enumerate(rec_cells):
            out[:, iz, ix] += q[k]
        return out

    # --- Frechet product (Eq. 20, 26-31) ---------------------------------------------------
    def frechet(self, model_b, U_b, fidx, dm, rec_cells, tol=1e-12):
        """J dm for every problem: the virtual source w^2 dm_rho u_b + div(dC(dm) : grad u_b)
        (Y and M of Eq. 26 together), convolved with G, solved in the background, sampled."""
        D = np.zeros((len(fidx), len(rec_cells), 2), dtype=np.complex128)
        for b, f in enumerate(fidx):
            src = contrast_source(U_b[b], dm, self.omegas[f], self.h)
            du = self.solve(self.convolve(src, f), model_b, f, tol=tol)
            D[b] = self.sample(du, rec_cells)
        return D

    # --- adjoint product (Eq. 25, 32-35) ---------------------------------------------------
    @staticmethod
    def imaging(u_a, u_b, omega, h):
        """Pointwise imaging of Eq. 32 (real part): rho: Re(w^2 u_a . u_b);
        C_pq: -Re(eps(u_a)^T B_pq eps(u_b)) with the 2D B matrices of Appendix C."""
        ea = strain(u_a, h)
        eb = strain(u_b, h)
        g = np.empty((N_PARAMS,) + u_a.shape[1:])
        g[0] = np.real(omega * omega * (u_a[0] * u_b[0] + u_a[1] * u_b[1]))
        g[1] = -np.real(ea[0] * eb[0])
        g[2] = -np.real(ea[0] * eb[1] + ea[1] * eb[0])
        g[3] = -np.real(ea[1] * eb[1])
        g[4] = -np.real(ea[2] * eb[2])
        return g

    def adjoint(self, model_b, U_b, fidx, R, rec_cells, tol=1e-12):
        """Re J^H R summed over problems: back-propagate conj(R) from the receivers (Eq. 33-35)
        and apply the imaging condition (Eq. 32)."""
        g = np.zeros((N_PARAMS, self.nz, self.nx))
        for b, f in enumerate(fidx):
            q = self.inject(np.conj(R[b]), rec_cells)
            ua = self.solve(self.convolve(q, f), model_b, f, tol=tol)
            g += self.imaging(ua, U_b[b], self.omegas[f], self.h)
        return g

    # --- misfit -----------------------------------------------------------------------------
    def misfit(self, model, fidx, src_cells, forces, d_obs, rec_cells, tol=1e-12):
        """Phi = 1/2 sum_b ||P u_b(model) - d_obs[b]||^2 and its gradient with respect to the
        per-cell (rho, C11, C13, C33, C55)."""
        U = self.forward(model, fidx, src_cells, forces, tol=tol)
        R = np.stack([self.sample(U[b], rec_cells) for b in range(len(fidx))]) - d_obs
        phi = 0.5 * float(np.sum(np.abs(R) ** 2))
        g = self.adjoint(model, U, fidx, R, rec_cells, tol=tol)
        return phi, g, U

    # --- normal equation (Eq. 23, 24) ------------------------------------------------------
    def param_scale(self):
        """Scale of the relative unknowns: the reference rho, C11 (for C11 and C13), C33, C55 (for an
        isotropic reference: rho0, rho0 alpha0^2 three times, rho0 beta0^2)."""
        r = self.ref
        return np.array([r[0], r[1], r[1], r[3], r[4]])

    def normal_cg(self, model_b, U_b, fidx, dd, rec_cells, iters=30, lam=None, lam_rel=1e-3,
                  power_start=None, power_iters=10, tol=1e-12):
        """Tikhonov normal equation (Re J~^H J~ + lambda I) x = Re J~^H dd on relative unknowns
        x = dm / scale, solved by `iters` CG steps from x = 0; returns (dm, lambda, history of
        ||normal residual||). If lam is None, lambda = lam_rel * (Rayleigh quotient after
        `power_iters` power steps on Re J~^H J~ from `power_start`)."""
        sc = self.param_scale()[:, None, None]

        def H(x):
            return sc * self.adjoint(model_b, U_b, fidx,
                                     self.frechet(model_b, U_b, fidx, sc * x, rec_cells, tol),
                                     rec_cells, tol)

        if lam is None:
            v = np.array(power_start, dtype=np.float64)
            v = v / np.sqrt(np.sum(v * v))
            for _ in range(power_iters):
                w = H(v)
                v = w / np.sqrt(np.sum(w * w))
            lam_max = float(np.sum(v * H(v)))
            lam = lam_rel * lam_max
        rhs = sc * self.adjoint(model_b, U_b, fidx, dd, rec_cells, tol)
        x = np.zeros_like(rhs)
        r = rhs.copy()
        p = r.copy()
        rr = float(np.sum(r * r))
        hist = [math.sqrt(rr)]
        for _ in range(iters):
            q = H(p) + lam * p
            alpha = rr / float(np.sum(p * q))
            x = x + alpha * p
            r = r - alpha * q
            rr_new = float(np.sum(r * r))
            hist.append(math.sqrt(rr_new))
            p = r + (rr_new / rr) * p
            rr = rr_new
        return sc * x, lam, hist


def normalized_error(a, b):
    """||a - b|| / ||b|| (the normalized data / model errors of Eq. 40, 41)."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))

"""Plain FP64 CPU oracle for the 3D elastic Lippmann-Schwinger operator (the paper's 3D extension,
Eq. A-1 and its 3D VTI example).

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's CPU legs may import
this module; the library never imports or calls it, and it imports nothing from the library.

Discrete problem (readings where the paper is silent, as in 2D):
  * Grid [nz][ny][nx] of cubic cells of side h; field components (u1, u2, u3) along (x1, x2, x3),
    x3 the depth; arrays indexed [c][z][y][x].
  * Medium: VTI with vertical symmetry axis, six parameters per cell (rho, C11, C13, C33, C55, C66)
    (C12 = C11 - 2 C66, C44 = C55); the homogeneous reference is isotropic (rho0, alpha0, beta0).
  * Green's tensor: the isotropic 3D tensor of Eq. A-1 written for the time convention of the 2D
    tensor (exp(+i w t), outgoing exp(-i k r)): with g_c(r) = exp(-i k_c r) / (4 pi r),
    G_ij = [k_s^2 g_s delta_ij + d_i d_j (g_s - g_p)] / (rho w^2). The paper prints Eq. A-1 for the
    opposite convention (exp(+i w r / alpha)); this is its complex conjugate.
  * Self cell: the mean of G over the ball of volume h^3 (radius a = h (3 / (4 pi))^(1/3)).
  * Central differences with fields zero outside the grid for the strain and the divergence of the
    stress; quadrature weight h^3; zero-padded FFT convolution on an lz x ly x lx grid (L >= 2N - 1).
  * Krylov: the 2D oracle's BiCGSTAB and GMRES work on flattened fields.
"""
from __future__ import annotations

import math

import numpy as np

from .dbi_oracle import bicgstab, gmres

N_PARAMS_3D = 6  # rho, C11, C13, C33, C55, C66


def reference_params_3d(rho0, alpha0, beta0) -> np.ndarray:
    """(rho, C11, C13, C33, C55, C66) of the isotropic reference."""
    a2, b2 = alpha0 * alpha0, beta0 * beta0
    return np.array([rho0, rho0 * a2, rho0 * (a2 - 2.0 * b2), rho0 * a2, rho0 * b2, rho0 * b2])


# ---------------------------------------------------------------------------------------------
# Green's tensor
# ---------------------------------------------------------------------------------------------
COMPONENTS_3D = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))  # 11, 12, 13, 22, 23, 33


def green_3d(y1, y2, y3, omega, alpha, beta, rho):
    """G_ij at offsets y = (y1, y2, y3) != 0 (arrays), as [6] arrays in COMPONENTS_3D order.

    With the direction cosines g = y / r, D_c = exp(-i k_c r) / (4 pi rho c^2 r) and
    q_c = 1 / (i k_c r) (the conjugate of the paper's -alpha / (i w r)):
    G_ij = D_p [g_i g_j + (3 g_i g_j - delta_ij)(q_p + q_p^2)]
         - D_s [(g_i g_j - delta_ij) + (3 g_i g_j - delta_ij)(q_s + q_s^2)]."""
    y = [np.asarray(v, dtype=np.float64) for v in (y1, y2, y3)]
    r = np.sqrt(y[0] ** 2 + y[1] ** 2 + y[2] ** 2)
    g = [v / r for v in y]
    out = []
    terms = []
    for c in (alpha, beta):
        k = omega / c
        D = np.exp(-1j * k * r) / (4.0 * math.pi * rho * c * c * r)
        q = 1.0 / (1j * k * r)
        terms.append((D, q + q * q))
    (Dp, Qp), (Ds, Qs) = terms
    for i, j in COMPONENTS_3D:
        gg = g[i] * g[j]
        d = 1.0 if i == j else 0.0
        out.append(Dp * (gg + (3 * gg - d) * Qp) - Ds * ((gg - d) + (3 * gg - d) * Qs))
    return out


def green_3d_self_cell(h, omega, alpha, beta, rho):
    """Mean of G over the ball of radius a = h (3 / (4 pi))^(1/3). From
    G = [k_s^2 g_s I + grad grad (g_s - g_p)] / (rho w^2): the ball mean of d_i d_j F for a radial
    F is delta_ij / 3 times the mean of its Laplacian, and Lap (g_s - g_p) = -k_s^2 g_s + k_p^2 g_p
    (the point sources cancel), so <G_ij> = delta_ij (2 k_s^2 <g_s> + k_p^2 <g_p>) / (3 rho w^2) with
    <g_c> = 3 / (4 pi a^3) int_0^a r exp(-i k r) dr = 3 (exp(-i k a)(1 + i k a) - 1) / (4 pi a^3 k^2).
    Returns the diagonal value."""
    a = h * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)

    def mean_g(c):
        k = omega / c
        return 3.0 * (np.exp(-1j * k * a) * (1.0 + 1j * k * a) - 1.0) / (4.0 * math.pi * a ** 3 * k * k)

    ks2, kp2 = (omega / beta) ** 2, (omega / alpha) ** 2
    return (2.0 * ks2 * mean_g(beta) + kp2 * mean_g(alpha)) / (3.0 * rho * omega * omega)


def green_lattice_3d(nz, ny, nx, h, omega, alpha, beta, rho) -> np.ndarray:
    """G_h on the offset lattice: [6][2nz-1][2ny-1][2nx-1], entry [c][dz+nz-1][dy+ny-1][dx+nx-1]."""
    dz = np.arange(-(nz - 1), nz)[:, None, None]
    dy = np.arange(-(ny - 1), ny)[None, :, None]
    dx = np.arange(-(nx - 1), nx)[None, None, :]
    shape = (2 * nz - 1, 2 * ny - 1, 2 * nx - 1)
    Z, Y, X = (np.broadcast_to(v, shape) * h for v in (dz, dy, dx))
    origin = (Z == 0) & (Y == 0) & (X == 0)
    comps = green_3d(np.where(origin, 1.0, X), np.where(origin, 1.0, Y), np.where(origin, 1.0, Z), omega,
                     alpha, beta, rho)
    s = green_3d_self_cell(h, omega, alpha, beta, rho)
    out = []
    for (i, j), G in zip(COMPONENTS_3D, comps):
        out.append(np.where(origin, s if i == j else 0.0, G))
    return np.stack(out).astype(np.complex128)


# ---------------------------------------------------------------------------------------------
# Strain, stress, divergence (central differences, zero outside the grid)
# ---------------------------------------------------------------------------------------------
def diff(v, axis, h):
    """Central difference of v along `axis` (of the [z][y][x] block), zero outside."""
    p = np.pad(v, [(1, 1) if a == axis else (0, 0) for a in range(v.ndim)])
    sl_p = [slice(None)] * v.ndim
    sl_m = [slice(None)] * v.ndim
    sl_p[axis] = slice(2, None)
    sl_m[axis] = slice(None, -2)
    return (p[tuple(sl_p)] - p[tuple(sl_m)]) / (2.0 * h)


AXIS = {0: 2, 1: 1, 2: 0}  # x1 -> x axis (last), x2 -> y axis, x3 -> z axis of [z][y][x]


def strain_3d(u, h):
    """Engineering strain (e11, e22, e33, 2 e23, 2 e13, 2 e12) in Voigt order 1..6."""
    d = lambda c, k: diff(u[c], AXIS[k], h)  # d u_c / d x_k
    return np.stack([d(0, 0), d(1, 1), d(2, 2), d(1, 2) + d(2, 1), d(0, 2) + d(2, 0), d(0, 1) + d(1, 0)])


def stress_3d(eps, dm):
    """sigma = C eps for VTI per cell (Voigt 6 x 6: C11, C12 = C11 - 2 C66, C13, C33, C44 = C55, C66);
    dm = [rho, C11, C13, C33, C55, C66] per cell (only the stiffness is used)."""
    c11, c13, c33, c55, c66 = dm[1], dm[2], dm[3], dm[4], dm[5]
    c12 = c11 - 2.0 * c66
    s1 = c11 * eps[0] + c12 * eps[1] + c13 * eps[2]
    s2 = c12 * eps[0] + c11 * eps[1] + c13 * eps[2]
    s3 = c13 * eps[0] + c13 * eps[1] + c33 * eps[2]
    return np.stack([s1, s2, s3, c55 * eps[3], c55 * eps[4], c66 * eps[5]])


VOIGT = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}


def divergence_3d(sig, h):
    """(div sigma)_i = sum_j d sigma_ij / d x_j."""
    return np.stack([sum(diff(sig[VOIGT[(i, j)]], AXIS[j], h) for j in range(3)) for i in range(3)])


def contrast_source_3d(u, dm, omega, h):
    """w^2 drho u + div(dC : eps(u))."""
    return omega * omega * dm[0] * u + divergence_3d(stress_3d(strain_3d(u, h), dm), h)


# ---------------------------------------------------------------------------------------------
# Convolution (Eq. 6 / Eq. 12 in 3D)
# ---------------------------------------------------------------------------------------------
def _full(Gc):
    """Symmetric 3 x 3 tensor of arrays from the six components."""
    idx = {(i, j): k for k, (i, j) in enumerate(COMPONENTS_3D)}
    return [[Gc[idx[(min(i, j), max(i, j))]] for j in range(3)] for i in range(3)]


def convolve_direct_3d(s, G_lat, h):
    """h^3 sum_x' G(x - x') s(x'), the plain O(N^6) sum (tiny grids only)."""
    _, nz, ny, nx = s.shape
    G = _full(G_lat)
    out = np.zeros_like(s, dtype=np.complex128)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for zp in range(nz):
                    for yp in range(ny):
                        for xp in range(nx):
                            iz, iy, ix = z - zp + nz - 1, y - yp + ny - 1, x - xp + nx - 1
                            for i in range(3):
                                out[i, z, y, x] += sum(G[i][j][iz, iy, ix] * s[j, zp, yp, xp] for j in range(3))
    return h ** 3 * out


def embed_circulant_3d(G_lat, lz, ly, lx):
    _, a, b, c = G_lat.shape
    nz, ny, nx = (a + 1) // 2, (b + 1) // 2, (c + 1) // 2
    E = np.zeros((G_lat.shape[0], lz, ly, lx), dtype=np.complex128)
    for dz in range(-(nz - 1), nz):
        for dy in range(-(ny - 1), ny):
            E[:, dz % lz, dy % ly, np.arange(-(nx - 1), nx) % lx] = G_lat[:, dz + nz - 1, dy + ny - 1, :]
    return E


def green_spectrum_3d(G_lat, lz, ly, lx):
    return np.fft.fftn(embed_circulant_3d(G_lat, lz, ly, lx), axes=(-3, -2, -1))


def convolve_fft_3d(s, G_hat, h):
    _, nz, ny, nx = s.shape
    _, lz, ly, lx = G_hat.shape
    sp = np.zeros((3, lz, ly, lx), dtype=np.complex128)
    sp[:, :nz, :ny, :nx] = s
    S = np.fft.fftn(sp, axes=(-3, -2, -1))
    G = _full(G_hat)
    O = np.stack([sum(G[i][j] * S[j] for j in range(3)) for i in range(3)])
    return h ** 3 * np.fft.ifftn(O, axes=(-3, -2, -1))[:, :nz, :ny, :nx]


class LSOracle3D:
    """3D LS operator A u = u - h^3 G * (w^2 drho u + div(dC : eps(u))) and its solves."""

    def __init__(self, nz, ny, nx, h, lz, ly, lx, rho0, alpha0, beta0, omegas, method="fft"):
        self.nz, self.ny, self.nx, self.h = nz, ny, nx, float(h)
        self.lz, self.ly, self.lx = lz, ly, lx
        self.rho0, self.alpha0, self.beta0 = float(rho0), float(alpha0), float(beta0)
        self.omegas = np.asarray(omegas, dtype=np.float64)
        self.method = method
        self.ref = reference_params_3d(rho0, alpha0, beta0)
        self.G_lat = [green_lattice_3d(nz, ny, nx, h, w, alpha0, beta0, rho0) for w in self.omegas]
        self.G_hat = [green_spectrum_3d(G, lz, ly, lx) for G in self.G_lat] if method == "fft" else None

    def convolve(self, s, f):
        if self.method == "direct":
            return convolve_direct_3d(s, self.G_lat[f], self.h)
        return convolve_fft_3d(s, self.G_hat[f], self.h)

    def apply(self, u, model, f):
        dm = np.asarray(model, dtype=np.float64) - self.ref[:, None, None, None]
        return u - self.convolve(contrast_source_3d(u, dm, self.omegas[f], self.h), f)

    def incident(self, f, src_cell, force):
        """u0(x) = G_h(x - x_s) f for a point force at cell (iz, iy, ix)."""
        iz, iy, ix = (int(v) for v in src_cell)
        nz, ny, nx = self.nz, self.ny, self.nx
        win = self.G_lat[f][:, nz - 1 - iz: 2 * nz - 1 - iz, ny - 1 - iy: 2 * ny - 1 - iy, nx - 1 - ix: 2 * nx - 1 - ix]
        G = _full(win)
        return np.stack([sum(G[i][j] * force[j] for j in range(3)) for i in range(3)]).astype(np.complex128)

    def solve(self, rhs, model, f, tol=1e-12, maxiter=3000, method="gmres", restart=30):
        shape = rhs.shape
        op = lambda v: self.apply(v.reshape(shape), model, f).reshape(-1)
        if method == "gmres":
            x, info = gmres(op, rhs.reshape(-1), restart=restart, tol=tol, maxiter=maxiter)
        else:
            x, info = bicgstab(op, rhs.reshape(-1), tol=tol, maxiter=maxiter)
        return x.reshape(shape), info


# ---------------------------------------------------------------------------------------------
# Distorted-Born products in 3D (Eq. 20, 25-35 with the 3D VTI stiffness)
# ---------------------------------------------------------------------------------------------
def imaging_3d(u_a, u_b, omega, h):
    """Pointwise imaging (real part) for (rho, C11, C13, C33, C55, C66): rho: Re(w^2 u_a . u_b);
    C_p: -Re(eps(u_a)^T B_p eps(u_b)) with B_p = dC/dp of the 3D VTI Voigt matrix (C12 = C11 - 2 C66,
    C44 = C55): B_C11 = E11 + E22 + E12 + E21, B_C13 = E13 + E31 + E23 + E32, B_C33 = E33,
    B_C55 = E44 + E55, B_C66 = E66 - 2 (E12 + E21)."""
    a = strain_3d(u_a, h)
    b = strain_3d(u_b, h)
    g = np.empty((N_PARAMS_3D,) + u_a.shape[1:])
    g[0] = np.real(omega * omega * (u_a[0] * u_b[0] + u_a[1] * u_b[1] + u_a[2] * u_b[2]))
    g[1] = -np.real((a[0] + a[1]) * (b[0] + b[1]))
    g[2] = -np.real((a[0] + a[1]) * b[2] + a[2] * (b[0] + b[1]))
    g[3] = -np.real(a[2] * b[2])
    g[4] = -np.real(a[3] * b[3] + a[4] * b[4])
    g[5] = -np.real(a[5] * b[5] - 2.0 * (a[0] * b[1] + a[1] * b[0]))
    return g


def sample_3d(u, rec_cells):
    """P u: the three components at the receiver cells, [n_rec][3]."""
    return np.stack([u[:, iz, iy, ix] for iz, iy, ix in rec_cells])


def inject_3d(q, rec_cells, shape):
    """P^T q: a field holding q[r] at receiver cell r (summed where receivers coincide)."""
    out = np.zeros((3,) + tuple(shape), dtype=np.complex128)
    for k, (iz, iy, ix) in enumerate(rec_cells):
        out[:, iz, iy, ix] += q[k]
    return out


def frechet_3d(orc, model_b, U_b, fidx, dm, rec_cells, tol=1e-12):
    """J dm for every problem: the virtual source w^2 dm_rho u_b + div(dC(dm) : eps(u_b)) convolved
    with G, solved in the background, sampled at the receivers."""
    D = np.zeros((len(fidx), len(rec_cells), 3), dtype=np.complex128)
    for b, f in enumerate(fidx):
        src = contrast_source_3d(U_b[b], dm, orc.omegas[f], orc.h)
        du, _ = orc.solve(orc.convolve(src, f), model_b, f, tol=tol)
        D[b] = sample_3d(du, rec_cells)
    return D


def adjoint_3d(orc, model_b, U_b, fidx, R, rec_cells, tol=1e-12):
    """Re J^H R summed over the problems: conj(R) injected at the receivers, convolved with G,
    solved in the background (the conjugate-source form of Eq. 33-35) and imaged against u_b."""
    g = np.zeros((N_PARAMS_3D, orc.nz, orc.ny, orc.nx))
    for b, f in enumerate(fidx):
        q = inject_3d(np.conj(R[b]), rec_cells, (orc.nz, orc.ny, orc.nx))
        ua, _ = orc.solve(orc.convolve(q, f), model_b, f, tol=tol)
        g += imaging_3d(ua, U_b[b], orc.omegas[f], orc.h)
    return g


def param_scale_3d(rho0, alpha0, beta0):
    """Scale of the relative unknowns: rho0; rho0 alpha0^2 for C11, C13, C33; rho0 beta0^2 for C55, C66."""
    a2, b2 = rho0 * alpha0 ** 2, rho0 * beta0 ** 2
    return np.array([rho0, a2, a2, a2, b2, b2])


def normal_cg_3d(orc, model_b, U_b, fidx, dd, rec_cells, iters=30, lam=None, lam_rel=1e-3, power_start=None,
                 power_iters=10, tol=1e-12):
    """Tikhonov normal equation (Re J~^H J~ + lambda I) x = Re J~^H dd on relative unknowns, as the
    2D oracle's normal_cg; returns (dm, lambda, history of ||normal residual||)."""
    sc = param_scale_3d(orc.rho0, orc.alpha0, orc.beta0)[:, None, None, None]

    def H(x):
        return sc * adjoint_3d(orc, model_b, U_b, fidx, frechet_3d(orc, model_b, U_b, fidx, sc * x, rec_cells, tol),
                               rec_cells, tol)

    if lam is None:
        v = np.array(power_start, dtype=np.float64)
        v = v / np.sqrt(np.sum(v * v))
        for _ in range(power_iters):
            w = H(v)
            v = w / np.sqrt(np.sum(w * w))
        lam = lam_rel * float(np.sum(v * H(v)))
    r = sc * adjoint_3d(orc, model_b, U_b, fidx, dd, rec_cells, tol)
    x = np.zeros_like(r)
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

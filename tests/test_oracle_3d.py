"""Pins of the 3D oracle (CPU only): the unit point force (traction balance on a small sphere), the
outgoing far field with the point-force radiation amplitudes, the closed-form tensor against its
potential representation
G = [k_s^2 g_s I + grad grad (g_s - g_p)] / (rho w^2) differentiated numerically, the elastic wave
equation by finite differences (residual O(d^2)), the self-cell ball mean against a quadrature of
the closed form, the direct sum against the FFT convolution, zero contrast, the Born series
against the solve, reciprocity of the discrete responses, the 3D Frechet and adjoint products
(the dot test, and the Frechet product against central differences of the forward map), and the
Voigt-form contrast source against the full VTI stiffness tensor, symbolically (sympy)."""
import math

import numpy as np
import pytest

import oracle as O

o3 = O.o3d
RHO, ALPHA, BETA = 2000.0, 2000.0, 1155.0


def G_full(y, w):
    comps = o3.green_3d(y[0], y[1], y[2], w, ALPHA, BETA, RHO)
    return np.array([[c.item() if np.ndim(c) else c for c in row] for row in o3._full(comps)])


@pytest.mark.parametrize("y", [(12.0, -7.0, 20.0), (40.0, 3.0, -5.0), (0.0, 0.0, 15.0)])
def test_closed_form_equals_the_potential_representation(y):
    w = 2 * np.pi * 10.0
    ks, kp = w / BETA, w / ALPHA
    F = lambda p: (np.exp(-1j * ks * np.linalg.norm(p)) - np.exp(-1j * kp * np.linalg.norm(p))) / (4 * math.pi * np.linalg.norm(p))
    d = 1e-3
    y = np.array(y)
    E = np.eye(3)
    H = np.empty((3, 3), dtype=complex)
    for i in range(3):
        for j in range(3):
            H[i, j] = (F(y + d * E[i] + d * E[j]) - F(y + d * E[i] - d * E[j]) - F(y - d * E[i] + d * E[j])
                       + F(y - d * E[i] - d * E[j])) / (4 * d * d)
    r = np.linalg.norm(y)
    gs = np.exp(-1j * ks * r) / (4 * math.pi * r)
    want = (ks * ks * gs * np.eye(3) + H) / (RHO * w * w)
    got = G_full(y, w)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()


def test_wave_equation_by_finite_differences():
    """mu Lap G + (lambda + mu) grad div G + rho w^2 G = 0 away from the source, O(d^2)."""
    w = 2 * np.pi * 12.0
    mu, lam = RHO * BETA ** 2, RHO * (ALPHA ** 2 - 2 * BETA ** 2)
    y0 = np.array([30.0, -20.0, 25.0])
    E = np.eye(3)

    def residual(d):
        G = lambda p: G_full(p, w)
        g0 = G(y0)
        lap = sum(G(y0 + d * E[k]) - 2 * g0 + G(y0 - d * E[k]) for k in range(3)) / d ** 2
        # (grad div G)_i m = sum_j d_i d_j G_jm
        gd = np.zeros((3, 3), dtype=complex)
        for i in range(3):
            for j in range(3):
                dij = (G(y0 + d * E[i] + d * E[j]) - G(y0 + d * E[i] - d * E[j]) - G(y0 - d * E[i] + d * E[j])
                       + G(y0 - d * E[i] - d * E[j])) / (4 * d * d)
                gd[i] += dij[j]
        r = mu * lap + (lam + mu) * gd + RHO * w * w * g0
        return np.abs(r).max() / (RHO * w * w * np.abs(g0).max())

    r1, r2 = residual(1.0), residual(0.5)
    assert r1 < 2e-3 and 3.5 < r1 / r2 < 4.5


def test_self_cell_against_a_ball_quadrature():
    """The ball mean by quadrature of the closed form: the 6-point octahedral rule is exact on the
    sphere for the quadratic angular dependence (the 1/r^3 near-field part averages to zero at
    every radius), Gauss-Legendre in r."""
    h, w = 10.0, 2 * np.pi * 15.0
    a = h * (3 / (4 * math.pi)) ** (1 / 3)
    x, wt = np.polynomial.legendre.leggauss(40)
    r = 0.5 * a * (x + 1)
    wr = 0.5 * a * wt
    dirs = np.vstack([np.eye(3), -np.eye(3)])
    acc = np.zeros((3, 3), dtype=complex)
    for rk, wk in zip(r, wr):
        ang = sum(G_full(rk * d, w) for d in dirs) / 6.0
        acc += wk * rk * rk * ang
    mean = 3.0 / a ** 3 * acc
    s = o3.green_3d_self_cell(h, w, ALPHA, BETA, RHO)
    assert abs(mean[0, 0] - s) <= 1e-10 * abs(s)
    assert np.abs(mean - s * np.eye(3)).max() <= 1e-10 * abs(s)


def test_direct_sum_equals_fft():
    nz, ny, nx, h = 3, 2, 4, 10.0
    w = 2 * np.pi * 9.0
    G = o3.green_lattice_3d(nz, ny, nx, h, w, ALPHA, BETA, RHO)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((3, nz, ny, nx)) + 1j * rng.standard_normal((3, nz, ny, nx))
    direct = o3.convolve_direct_3d(s, G, h)
    for L in ((2 * nz, 2 * ny, 2 * nx), (8, 4, 16)):
        fft = o3.convolve_fft_3d(s, o3.green_spectrum_3d(G, *L), h)
        assert np.linalg.norm(fft - direct) <= 1e-12 * np.linalg.norm(direct)


def case(nz=4, ny=3, nx=5, amp=0.1, seed=2):
    rng = np.random.default_rng(seed)
    ref = o3.reference_params_3d(RHO, ALPHA, BETA)
    model = ref[:, None, None, None] * (1 + amp * (2 * rng.random((6, nz, ny, nx)) - 1))
    orc = o3.LSOracle3D(nz, ny, nx, 10.0, 2 * nz, 2 * ny, 2 * nx, RHO, ALPHA, BETA, [2 * np.pi * 10.0])
    return orc, model, ref


def test_zero_contrast_is_the_identity():
    orc, _, ref = case()
    model = np.broadcast_to(ref[:, None, None, None], (6, 4, 3, 5))
    u = orc.incident(0, (1, 1, 2), (0.0, 0.3, 1.0))
    assert np.array_equal(orc.apply(u, model, 0), u)


def test_born_series_equals_the_solve():
    orc, model, ref = case(amp=0.01)
    u0 = orc.incident(0, (0, 1, 2), (0.2, 0.0, 1.0))
    u, info = orc.solve(u0, model, 0, tol=1e-13)
    dm = model - ref[:, None, None, None]
    K = lambda v: orc.convolve(o3.contrast_source_3d(v, dm, orc.omegas[0], orc.h), 0)
    term, series = u0, u0.copy()
    for _ in range(40):
        term = K(term)
        series = series + term
    assert np.linalg.norm(series - u) <= 1e-10 * np.linalg.norm(u)


def test_reciprocity():
    """The discrete response at cell r, component i, to a unit force at s along j equals the
    response at s, component j, to a force at r along i (the contrast operator is real symmetric
    and G_h complex symmetric)."""
    orc, model, _ = case(amp=0.2)
    s, r = (0, 1, 1), (3, 2, 4)
    for i, j in ((0, 2), (1, 1), (2, 0)):
        fj, fi = np.eye(3)[j], np.eye(3)[i]
        u_s, _ = orc.solve(orc.incident(0, s, fj), model, 0, tol=1e-13)
        u_r, _ = orc.solve(orc.incident(0, r, fi), model, 0, tol=1e-13)
        a, b = u_s[i][r], u_r[j][s]
        assert abs(a - b) <= 1e-10 * abs(a), (i, j)


def products_case():
    orc, model, ref = case(nz=4, ny=3, nx=5, amp=0.1, seed=8)
    rng = np.random.default_rng(9)
    srcs = [(0, 1, 2), (0, 0, 4)]
    forces = [(0.0, 0.0, 1.0), (0.3, 0.0, 1.0)]
    fidx = [0, 0]
    U_b = np.stack([orc.solve(orc.incident(0, s, fv), model, 0, tol=1e-13)[0] for s, fv in zip(srcs, forces)])
    rec = [(0, y, x) for y in range(3) for x in range(0, 5, 2)]
    return orc, model, ref, rng, fidx, U_b, rec, srcs, forces


def test_frechet_adjoint_dot_product():
    """<J dm, r>_Re = <dm, Re J^H r> for real dm: the imaging of every parameter is the exact adjoint
    of its virtual source (a wrong B matrix, sign or conjugation breaks it)."""
    orc, model, ref, rng, fidx, U_b, rec, _, _ = products_case()
    dm = ref[:, None, None, None] * 0.01 * rng.standard_normal((6, 4, 3, 5))
    r = rng.standard_normal((2, len(rec), 3)) + 1j * rng.standard_normal((2, len(rec), 3))
    Jdm = o3.frechet_3d(orc, model, U_b, fidx, dm, rec, tol=1e-13)
    g = o3.adjoint_3d(orc, model, U_b, fidx, r, rec, tol=1e-13)
    lhs = float(np.real(np.vdot(r, Jdm)))
    rhs = float(np.sum(dm * g))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_frechet_equals_the_derivative_of_the_forward_map():
    """J dm against the central difference of d(m) = P A(m)^-1 u0 (step 1e-4 of the perturbation):
    the operator is affine in the model, so the difference is exact up to O(step^2)."""
    orc, model, ref, rng, fidx, U_b, rec, srcs, forces = products_case()
    dm = ref[:, None, None, None] * 0.05 * rng.standard_normal((6, 4, 3, 5))
    Jdm = o3.frechet_3d(orc, model, U_b, fidx, dm, rec, tol=1e-13)
    eps = 1e-4

    def data(m):
        return np.stack([o3.sample_3d(orc.solve(orc.incident(0, s, fv), m, 0, tol=1e-14)[0], rec)
                         for s, fv in zip(srcs, forces)])

    fd = (data(model + eps * dm) - data(model - eps * dm)) / (2 * eps)
    assert np.linalg.norm(fd - Jdm) <= 1e-6 * np.linalg.norm(Jdm)


def test_normal_cg_against_a_dense_solve():
    """Enough CG steps on the 3D normal equation reach the dense solution of
    (Re J~^T J~ + lambda I) x = Re J~^T dd built column by column from the Frechet product."""
    orc, model, ref, rng, fidx, U_b, rec, _, _ = products_case()
    dd = rng.standard_normal((2, len(rec), 3)) + 1j * rng.standard_normal((2, len(rec), 3))
    sc = o3.param_scale_3d(orc.rho0, orc.alpha0, orc.beta0)[:, None, None, None]
    n = 6 * 4 * 3 * 5
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(o3.frechet_3d(orc, model, U_b, fidx, sc * e.reshape(6, 4, 3, 5), rec, tol=1e-13).reshape(-1))
    J = np.stack(cols, axis=1)
    lam = 1e-3 * np.linalg.norm(J, 2) ** 2
    b = np.real(J.conj().T @ dd.reshape(-1))
    x_dense = np.linalg.solve(np.real(J.conj().T @ J) + lam * np.eye(n), b)
    dm, lam_out, hist = o3.normal_cg_3d(orc, model, U_b, fidx, dd, rec, iters=150, lam=lam, tol=1e-13)
    assert lam_out == lam and hist[-1] < 1e-8 * hist[0]
    assert np.linalg.norm(dm / sc - x_dense.reshape(6, 4, 3, 5)) <= 1e-6 * np.linalg.norm(x_dense)


def _vti_stiffness(C11, C13, C33, C55, C66):
    """C_ijkl of a VTI medium with symmetry axis x3 (0-based indices), from the tensor's minor and
    major symmetries and the five independent moduli: C_1111 = C_2222 = C11, C_3333 = C33,
    C_1122 = C11 - 2 C66 (isotropy in the x1-x2 plane), C_1133 = C_2233 = C13,
    C_2323 = C_1313 = C55 (= C44), C_1212 = C66; every other entry is zero."""
    C = {}

    def put(i, j, k, l, v):
        for a, b in ((i, j), (j, i)):
            for c, d in ((k, l), (l, k)):
                C[(a, b, c, d)] = v
                C[(c, d, a, b)] = v

    put(0, 0, 0, 0, C11)
    put(1, 1, 1, 1, C11)
    put(2, 2, 2, 2, C33)
    put(0, 0, 1, 1, C11 - 2 * C66)
    put(0, 0, 2, 2, C13)
    put(1, 1, 2, 2, C13)
    put(1, 2, 1, 2, C55)
    put(0, 2, 0, 2, C55)
    put(0, 1, 0, 1, C66)
    return lambda i, j, k, l: C.get((i, j, k, l), 0)


def test_contrast_source_equals_the_tensor_form():
    """For quadratic u and linear contrasts the central differences are exact, so on cells two or
    more from the edge the oracle's Voigt-form source equals w^2 drho u_i + d_j (C_ijkl eps_kl)
    computed symbolically from the full stiffness tensor and eps_kl = (d_k u_l + d_l u_k) / 2.
    Catches a wrong Voigt index, shear factor, C12, axis mapping or divergence index."""
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x1 x2 x3")
    rng = np.random.default_rng(41)
    c = lambda: complex(rng.normal(), rng.normal())  # noqa: E731
    monomials = [1, *X, *(X[a] * X[b] for a in range(3) for b in range(a, 3))]
    u = [sum(c() * m for m in monomials) for _ in range(3)]
    lin = lambda s: s * (1 + sum(0.01 * rng.normal() * x for x in X))  # noqa: E731
    drho = lin(170.0)
    mod = [lin(3e8), lin(-1e8), lin(2e8), lin(7e7), lin(9e7)]  # C11, C13, C33, C55, C66
    Cijkl = _vti_stiffness(*mod)
    eps = [[(sp.diff(u[l], X[k]) + sp.diff(u[k], X[l])) / 2 for l in range(3)] for k in range(3)]
    sig = [[sum(Cijkl(i, j, k, l) * eps[k][l] for k in range(3) for l in range(3)) for j in range(3)]
           for i in range(3)]
    omega = 2 * math.pi * 6.0
    src = [omega ** 2 * drho * u[i] + sum(sp.diff(sig[i][j], X[j]) for j in range(3)) for i in range(3)]
    nz, ny, nx, h = 7, 8, 9, 3.0
    Z, Y, Xg = np.meshgrid(np.arange(nz) * h, np.arange(ny) * h, np.arange(nx) * h, indexing="ij")

    def ev(e):
        return np.broadcast_to(sp.lambdify(X, e, "numpy")(Xg, Y, Z), (nz, ny, nx)).astype(complex)

    field = np.stack([ev(ui) for ui in u])
    dmod = np.stack([ev(drho).real] + [ev(m).real for m in mod])
    got = o3.contrast_source_3d(field, dmod, omega, h)
    want = np.stack([ev(s) for s in src])
    sl = (slice(None), slice(2, nz - 2), slice(2, ny - 2), slice(2, nx - 2))
    assert np.max(np.abs(got[sl] - want[sl])) < 1e-9 * np.max(np.abs(want[sl]))


@pytest.mark.parametrize("j", [0, 2])
def test_green_point_force_traction(j):
    """The traction of column j of G on a small sphere around the source integrates to -e_j: G is
    the response to a unit point force (fixes its scale and sign, which the homogeneous wave
    equation cannot). Radius 1e-3 of the S wavelength over 2 pi (dynamic correction ~ (k r)^2);
    4th-order differences of the closed form; Gauss-Legendre in cos(theta) x trapezoid in phi,
    exact for the traction's low-degree angular dependence."""
    omega = 2 * math.pi * 10.0
    mu, lam = RHO * BETA ** 2, RHO * (ALPHA ** 2 - 2 * BETA ** 2)
    eps = 1e-3 * BETA / omega
    d = 1e-2 * eps
    E = np.eye(3)

    def col(p):
        return G_full(p, omega)[:, j]

    def grad(p):  # du[i][k] = d u_i / d x_k
        g = np.empty((3, 3), dtype=np.complex128)
        for k in range(3):
            e = d * E[k]
            g[:, k] = (-col(p + 2 * e) + 8 * col(p + e) - 8 * col(p - e) + col(p - 2 * e)) / (12 * d)
        return g

    mus, wmu = np.polynomial.legendre.leggauss(12)
    nphi = 24
    total = np.zeros(3, dtype=np.complex128)
    for m, wm in zip(mus, wmu):
        s = math.sqrt(1 - m * m)
        for phi in np.arange(nphi) * 2 * math.pi / nphi:
            n = np.array([s * math.cos(phi), s * math.sin(phi), m])
            du = grad(eps * n)
            sig = lam * np.trace(du) * E + mu * (du + du.T)
            total += (sig @ n) * wm * (2 * math.pi / nphi) * eps * eps
    assert np.max(np.abs(total + E[j])) < 1e-4


def test_green_far_field_outgoing():
    """Far from the source on the x3 axis G33 is the P wave exp(-i k_p r) / (4 pi rho alpha^2 r)
    and G11 the S wave exp(-i k_s r) / (4 pi rho beta^2 r) (the point-force radiation pattern):
    the phase falls at the wavenumber's rate (outgoing for exp(+i w t), the 2D tensor's
    convention) and the amplitudes decay like 1/r with the stated constants (at 200 km the near
    field and the other wave type are ~3e-4 of the far field on this axis)."""
    omega = 2 * math.pi * 15.0
    r0, dr = 200000.0, 0.5
    for comp, c in ((2, ALPHA), (0, BETA)):
        k = omega / c
        g = [G_full((0.0, 0.0, r), omega)[comp, comp] for r in (r0, r0 + dr)]
        rate = np.angle(g[1] / g[0]) / dr
        assert abs(rate + k) < 2e-3 * k, comp
        far = 1.0 / (4 * math.pi * RHO * c * c * r0)
        assert abs(abs(g[0]) / far - 1) < 2e-3, comp


def test_incident_field_is_the_point_force_response():
    """u0 of a point force f at cell x_s (Eq. 7) is the convolution of G_h with the force density
    f delta(x - x_s) / h^3 (the discrete delta), and away from the source it is the closed form
    G(x - x_s) f (pins the window offsets and the scale of the incident field)."""
    orc, _, _ = case(nz=4, ny=3, nx=5)
    src, force = (1, 2, 3), np.array([0.3, -0.2, 1.0])
    u0 = orc.incident(0, src, force)
    s = np.zeros((3, 4, 3, 5), dtype=np.complex128)
    s[:, src[0], src[1], src[2]] = force / orc.h ** 3
    conv = orc.convolve(s, 0)
    assert np.linalg.norm(u0 - conv) <= 1e-12 * np.linalg.norm(conv)
    w = orc.omegas[0]
    for cell in ((0, 0, 0), (3, 1, 4), (1, 2, 0)):
        y = [(cell[2] - src[2]) * orc.h, (cell[1] - src[1]) * orc.h, (cell[0] - src[0]) * orc.h]  # x1, x2, x3
        want = G_full(y, w) @ force
        got = u0[:, cell[0], cell[1], cell[2]]
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), cell

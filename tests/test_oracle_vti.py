"""Pins of the oracle's Green's tensor for a homogeneous VTI reference (its spectral representation
over slowness directions), CPU only: the isotropic limit against the closed form of Appendix A
(the Hankel functions), the self-cell mean against the isotropic disk average, the elastic wave
equation of a VTI medium by finite differences away from the source (residual falling as h^2),
the mirror symmetries, the LS operator with a VTI reference against the isotropic one when
the VTI stiffness is isotropic, and the unit point force of the anisotropic medium (traction
balance on a small circle)."""
import math

import numpy as np
import pytest

import oracle as O

RHO, ALPHA, BETA = 2000.0, 2000.0, 1155.0


def vti_params(rho=2200.0, alpha_v=2500.0, eps=0.2, delta=0.1):
    """(rho, C11, C13, C33, C55) of a VTI medium from vertical velocities and Thomsen's epsilon,
    delta: C33 = rho a^2, C55 = rho b^2 (b = a / sqrt 3), C11 = (1 + 2 eps) C33,
    (C13 + C55)^2 = (C33 - C55)(C33 (1 + 2 delta) - C55)."""
    c33 = rho * alpha_v ** 2
    c55 = rho * (alpha_v / math.sqrt(3.0)) ** 2
    c11 = (1.0 + 2.0 * eps) * c33
    c13 = math.sqrt((c33 - c55) * (c33 * (1.0 + 2.0 * delta) - c55)) - c55
    return rho, c11, c13, c33, c55


@pytest.mark.parametrize("y", [(10.0, 0.0), (0.0, -20.0), (30.0, -20.0), (-7.0, 55.0), (400.0, 130.0)])
def test_isotropic_limit_equals_the_closed_form(y):
    w = 2 * np.pi * 9.0
    g = O.green_vti_2d(y[0], y[1], w, *O.reference_params(RHO, ALPHA, BETA))
    h = [c.item() for c in O.green_2d(np.array([y[0]]), np.array([y[1]]), w, ALPHA, BETA, RHO)]
    scale = max(abs(c) for c in h)
    for a, b in zip(g, h):
        assert abs(a - b) <= 1e-9 * scale


def test_isotropic_self_cell_equals_the_disk_average():
    w, h = 2 * np.pi * 13.0, 10.0
    g = O.green_vti_self_cell(h, w, *O.reference_params(RHO, ALPHA, BETA))
    want = O.green_self_cell(h, w, ALPHA, BETA, RHO)
    assert abs(g[0] - want[0]) <= 1e-12 * abs(want[0])
    assert abs(g[2] - want[2]) <= 1e-12 * abs(want[2])
    assert abs(g[1]) <= 1e-14 * abs(want[0])


def test_vti_tensor_solves_the_wave_equation():
    """(C : grad grad + rho w^2) G = 0 away from the source, with the 2D VTI stiffness written
    out component by component; central differences of spacing d leave a residual O(d^2)."""
    rho, c11, c13, c33, c55 = vti_params()
    w = 2 * np.pi * 12.0
    y0 = (40.0, 25.0)

    def G(y1, y3, params):
        g11, g13, g33 = O.green_vti_2d(y1, y3, w, *params, epsabs=1e-13, epsrel=1e-10)
        return np.array([[g11, g13], [g13, g33]])

    def residual(d, params=(rho, c11, c13, c33, c55)):
        c = {(i, j): G(y0[0] + i * d, y0[1] + j * d, params) for i in (-1, 0, 1) for j in (-1, 0, 1)}
        g = c[(0, 0)]
        d11 = (c[(1, 0)] - 2 * g + c[(-1, 0)]) / d ** 2
        d33 = (c[(0, 1)] - 2 * g + c[(0, -1)]) / d ** 2
        d13 = (c[(1, 1)] - c[(1, -1)] - c[(-1, 1)] + c[(-1, -1)]) / (4 * d * d)
        r = np.empty((2, 2), dtype=complex)
        for m in range(2):  # column m of G: the response to a force along x_m
            r[0, m] = c11 * d11[0, m] + c55 * d33[0, m] + (c13 + c55) * d13[1, m] + rho * w * w * g[0, m]
            r[1, m] = c55 * d11[1, m] + c33 * d33[1, m] + (c13 + c55) * d13[0, m] + rho * w * w * g[1, m]
        return np.abs(r).max() / (rho * w * w * np.abs(g).max())

    r1, r2 = residual(2.0), residual(1.0)
    assert r1 < 4e-3 and r2 < 1e-3
    assert 3.5 < r1 / r2 < 4.5  # second-order: halving d divides the residual by 4
    # planted mistakes in the tensor's medium (C11 and C33 exchanged, C13 10 % off) are caught
    assert residual(1.0, (rho, c33, c13, c11, c55)) > 1e-2
    assert residual(1.0, (rho, c11, 1.1 * c13, c33, c55)) > 1e-2


def test_mirror_symmetries():
    rho, c11, c13, c33, c55 = vti_params()
    w = 2 * np.pi * 7.0
    a = O.green_vti_2d(23.0, 14.0, w, rho, c11, c13, c33, c55)
    for s1, s3 in ((-1, 1), (1, -1), (-1, -1)):
        b = O.green_vti_2d(s1 * 23.0, s3 * 14.0, w, rho, c11, c13, c33, c55)
        assert abs(b[0] - a[0]) <= 1e-10 * abs(a[0])
        assert abs(b[2] - a[2]) <= 1e-10 * abs(a[2])
        assert abs(b[1] - s1 * s3 * a[1]) <= 1e-10 * abs(a[1])
    # and the anisotropy is real: the response differs between the two axes
    x, z = O.green_vti_2d(30.0, 0.0, w, rho, c11, c13, c33, c55), O.green_vti_2d(0.0, 30.0, w, rho, c11, c13, c33, c55)
    assert abs(x[0] - z[2]) > 1e-2 * abs(x[0])


def test_ls_operator_with_an_isotropic_vti_reference():
    nz, nx, h = 6, 5, 10.0
    w = [2 * np.pi * 9.0]
    iso = O.LSOracle(nz, nx, h, 2 * nz, 2 * nx, RHO, ALPHA, BETA, w)
    vti = O.LSOracle(nz, nx, h, 2 * nz, 2 * nx, RHO, ALPHA, BETA, w, ref_vti=O.reference_params(RHO, ALPHA, BETA),
                     vti_epsrel=1e-11)
    assert np.abs(vti.G_lat[0] - iso.G_lat[0]).max() <= 1e-9 * np.abs(iso.G_lat[0]).max()
    rng = np.random.default_rng(4)
    model = O.reference_params(RHO, ALPHA, BETA)[:, None, None] * (1 + 0.1 * rng.standard_normal((5, nz, nx)))
    u = rng.standard_normal((2, nz, nx)) + 1j * rng.standard_normal((2, nz, nx))
    a, b = vti.apply(u, model, 0), iso.apply(u, model, 0)
    assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b - u)


def test_zero_contrast_against_a_vti_reference():
    """A model equal to the VTI reference has no contrast: A = I, and the scattered field of a
    point source vanishes."""
    ref = vti_params()
    nz, nx = 5, 4
    orc = O.LSOracle(nz, nx, 5.0, 2 * nz, 2 * nx, ref[0], 2500.0, 1443.0, [2 * np.pi * 8.0], ref_vti=ref,
                     vti_epsrel=1e-9)
    model = np.broadcast_to(np.asarray(ref)[:, None, None], (5, nz, nx))
    u0 = orc.incident(0, (0, 2), (0.0, 1.0))
    assert np.array_equal(orc.apply(u0, model, 0), u0)
    assert np.abs(orc.G_lat[0][0]).max() > 0


def test_far_offset_quadrature_against_multiprecision():
    """The adaptive quadrature at an offset of 90 radians of phase, against the same integral in
    20-digit arithmetic by mpmath's tanh-sinh rule on 100 pieces (the closed-form and wave-equation
    pins above fix the representation; this one fixes the quadrature's accuracy far out)."""
    mp = pytest.importorskip("mpmath")
    rho, c11, c13, c33, c55 = vti_params(eps=0.1, delta=0.1)
    w, y1, y3 = 2 * np.pi * 19.0, 630.0, 630.0
    g = O.green_vti_2d(y1, y3, w, rho, c11, c13, c33, c55)
    mp.mp.dps = 20
    R = [mp.mpf(v) for v in (rho, c11, c13, c33, c55)]
    r, phi, om = mp.sqrt(mp.mpf(y1) ** 2 + mp.mpf(y3) ** 2), mp.atan2(y3, y1), 2 * mp.pi * 19

    def entry(c, part):
        def f(psi):
            n1, n3 = mp.cos(phi + psi), mp.sin(phi + psi)
            g11, g33 = R[1] * n1 ** 2 + R[4] * n3 ** 2, R[4] * n1 ** 2 + R[3] * n3 ** 2
            g13 = (R[2] + R[4]) * n1 * n3
            mean, rad = (g11 + g33) / 2, mp.sqrt(((g11 - g33) / 2) ** 2 + g13 ** 2)
            tot = mp.mpf(0)
            for lam, other in ((mean + rad, mean - rad), (mean - rad, mean + rad)):
                P = ((g11 - other) / (lam - other), g13 / (lam - other), (g33 - other) / (lam - other))[c]
                x = om * mp.sqrt(R[0] / lam) * r * mp.cos(psi)
                j = -mp.cos(x) * mp.ci(x) - mp.sin(x) * mp.si(x) if part == 0 else -mp.pi / 2 * mp.cos(x)
                tot += P / lam * j
            return tot
        return float(mp.quad(f, [-mp.pi / 2 + mp.pi * i / 100 for i in range(101)]) / (2 * mp.pi ** 2))

    scale = max(abs(v) for v in g)
    for c in range(3):
        want = entry(c, 0) + 1j * entry(c, 1)
        assert abs(g[c] - want) <= 1e-12 * scale, c


def test_vti_point_force_traction():
    """The traction of the VTI tensor's column for a vertical force, on a small circle around the
    source, integrates to -e_3: G is the response to a unit point force in the anisotropic medium
    too. The isotropic-limit pin cannot see a normalisation error that depends on the anisotropy
    (a constant factor leaves the homogeneous wave equation satisfied); this pin can. Stress from
    the VTI stiffness in the x1-x3 plane: s11 = C11 e11 + C13 e33, s33 = C13 e11 + C33 e33,
    s13 = 2 C55 e13; radius 1e-4 of the S wavelength over 2 pi; central differences of step
    1e-3 of the radius; 24-point trapezoid over the circle."""
    rho, c11, c13, c33, c55 = vti_params()
    omega = 2 * math.pi * 10.0
    eps = 1e-4 * math.sqrt(c55 / rho) / omega
    d = 1e-3 * eps

    def u(y1, y3):  # column 3 of G: (G13, G33)
        g11, g13, g33 = O.green_vti_2d(y1, y3, omega, rho, c11, c13, c33, c55, epsrel=1e-13)
        return np.array([g13, g33])

    n = 24
    total = np.zeros(2, dtype=np.complex128)
    for t in (np.arange(n) + 0.5) * 2 * math.pi / n:
        n1, n3 = math.cos(t), math.sin(t)
        y1, y3 = eps * n1, eps * n3
        d1 = (u(y1 + d, y3) - u(y1 - d, y3)) / (2 * d)  # d/dx1 of (u1, u3)
        d3 = (u(y1, y3 + d) - u(y1, y3 - d)) / (2 * d)  # d/dx3
        e11, e33, e13 = d1[0], d3[1], 0.5 * (d3[0] + d1[1])
        s11, s33, s13 = c11 * e11 + c13 * e33, c13 * e11 + c33 * e33, 2 * c55 * e13
        total += np.array([s11 * n1 + s13 * n3, s13 * n1 + s33 * n3]) * (2 * math.pi * eps / n)
    assert np.max(np.abs(total - np.array([0.0, -1.0]))) < 1e-4, total

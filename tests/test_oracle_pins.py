"""Pins of the CPU oracle against facts that do not come from the oracle itself: the elastic wave
equation, the point-force condition, the radiation condition, independent quadrature, symbolic
calculus (sympy), brute-force dense linear algebra, series expansions, finite differences and the
B matrices printed in Appendix C of the paper. None of these tests needs a GPU."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2402_02116_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

RHO, ALPHA, BETA = 2000.0, 2000.0, 1155.0
LAM = RHO * (ALPHA ** 2 - 2 * BETA ** 2)
MU = RHO * BETA ** 2


def _col(y1, y3, omega, j):
    """Displacement (u1, u3) of a unit force along j (0: x1, 1: x3) at offset (y1, y3)."""
    G11, G13, G33 = O.green_2d(y1, y3, omega, ALPHA, BETA, RHO)
    return (G11, G13) if j == 0 else (G13, G33)


def _d(fun, y1, y3, axis, d):
    """Fourth-order central first derivative of fun(y1, y3) along axis 0 (x1) or 1 (x3)."""
    e1, e3 = (d, 0.0) if axis == 0 else (0.0, d)
    return (-fun(y1 + 2 * e1, y3 + 2 * e3) + 8 * fun(y1 + e1, y3 + e3)
            - 8 * fun(y1 - e1, y3 - e3) + fun(y1 - 2 * e1, y3 - 2 * e3)) / (12 * d)


def _navier_residual(y1, y3, omega, j, d):
    """w^2 rho u + (lambda + mu) grad div u + mu lap u for u = column j of G (Eq. 3 with C0)."""
    u = lambda a, b, i: _col(a, b, omega, j)[i]  # noqa: E731
    res = []
    for i in range(2):
        lap = 0.0
        for ax in range(2):
            lap += _d(lambda a, b: _d(lambda p, q: u(p, q, i), a, b, ax, d), y1, y3, ax, d)
        graddiv = 0.0
        for k in range(2):
            graddiv += _d(lambda a, b: _d(lambda p, q: u(p, q, k), a, b, k, d), y1, y3, i, d)
        res.append(omega ** 2 * RHO * u(y1, y3, i) + (LAM + MU) * graddiv + MU * lap)
    return np.array(res), omega ** 2 * RHO * np.abs(np.array([u(y1, y3, 0), u(y1, y3, 1)]))


@pytest.mark.parametrize("j", [0, 1])
def test_green_satisfies_navier_equation(j):
    """Away from the source every column of G solves the homogeneous elastic equation (Eq. 3),
    and the finite-difference residual falls like step^4 (4th-order stencils)."""
    omega = 2 * math.pi * 12.0
    pts = [(37.0, 23.0), (-55.0, 81.0), (140.0, -9.0), (3.0, 60.0)]
    for (y1, y3) in pts:
        r1, scale = _navier_residual(y1, y3, omega, j, 0.8)
        r2, _ = _navier_residual(y1, y3, omega, j, 0.4)
        assert np.max(np.abs(r2)) < 1e-6 * np.max(scale)
        assert np.max(np.abs(r2)) < np.max(np.abs(r1)) / 8.0


@pytest.mark.parametrize("j", [0, 1])
def test_green_point_force_traction(j):
    """The traction of column j of G on a small circle around the source integrates to -e_j:
    the unit point force of Eq. 3 (fixes the scale 1/(8 i rho) together with H^(2))."""
    omega = 2 * math.pi * 10.0
    eps = 1e-4 * BETA / omega
    d = 1e-2 * eps
    n = 96
    total = np.zeros(2, dtype=np.complex128)
    for t in (np.arange(n) + 0.5) * 2 * math.pi / n:
        n1, n3 = math.cos(t), math.sin(t)
        y1, y3 = eps * n1, eps * n3
        du = np.zeros((2, 2), dtype=np.complex128)  # du[i][k] = d u_i / d x_k
        for i in range(2):
            for k in range(2):
                du[i, k] = _d(lambda a, b: _col(a, b, omega, j)[i], y1, y3, k, d)
        div = du[0, 0] + du[1, 1]
        sig = LAM * div * np.eye(2) + MU * (du + du.T)
        total += (sig @ np.array([n1, n3])) * (2 * math.pi * eps / n)
    expect = -np.eye(2)[j]
    assert np.max(np.abs(total - expect)) < 1e-5


def test_green_outgoing_and_amplitude():
    """Far from the source along x3, G33 is the P wave (1/(4 i rho alpha^2)) H0^(2)(k r): its phase
    decreases at rate k_alpha (outgoing for exp(+i w t)) and |G| decays like r^{-1/2}."""
    omega = 2 * math.pi * 15.0
    k = omega / ALPHA
    r = np.array([20000.0, 20000.5])
    _, _, G33 = O.green_2d(np.zeros(2), r, omega, ALPHA, BETA, RHO)
    dphase = np.angle(G33[1] / G33[0]) / 0.5
    assert abs(dphase + k) < 1e-2 * k  # S near field perturbs the rate at ~1e-3
    far = np.sqrt(2 / (math.pi * k * r[0])) / (4 * RHO * ALPHA ** 2)
    assert abs(abs(G33[0]) / far - 1) < 1e-2


def test_self_cell_is_disk_average():
    """The self-cell value equals the mean of the closed-form G over the disk of area h^2, computed
    by independent quadrature in polar coordinates (periodic trapezoid in angle, adaptive in r)."""
    from scipy.integrate import quad
    h = 10.0
    omega = 2 * math.pi * 10.0
    a = h / math.sqrt(math.pi)
    t = (np.arange(64) + 0.5) * 2 * math.pi / 64
    got = O.green_self_cell(h, omega, ALPHA, BETA, RHO)
    tiny = 1e-14 * abs(got[0])

    def ring(r, comp, part):
        g = O.green_2d(r * np.cos(t), r * np.sin(t), omega, ALPHA, BETA, RHO)[comp]
        return getattr(np.mean(g), part) * 2 * math.pi * r

    import warnings
    from scipy.integrate import IntegrationWarning
    for comp in range(3):
        with warnings.catch_warnings():
            # G13 has zero angular mean: its ring values are rounding noise near r = 0
            warnings.simplefilter("ignore", IntegrationWarning)
            re = quad(lambda r: ring(r, comp, "real"), 0, a, limit=200, epsabs=tiny, epsrel=1e-12)[0]
            im = quad(lambda r: ring(r, comp, "imag"), 0, a, limit=200, epsabs=tiny, epsrel=1e-12)[0]
        mean = (re + 1j * im) / (math.pi * a * a)
        assert abs(mean - got[comp]) < 1e-9 * abs(got[0]), (comp, mean, got[comp])


def test_green_lattice_symmetries():
    """G(-y) = G(y); G11, G33 are even in each coordinate and G13 is odd in each (Eq. A-3)."""
    G = O.green_lattice(7, 9, 10.0, 2 * math.pi * 9.0, ALPHA, BETA, RHO)
    assert np.allclose(G, G[:, ::-1, ::-1], rtol=1e-14, atol=0)
    assert np.allclose(G[0], G[0][:, ::-1], rtol=1e-14, atol=0)
    assert np.allclose(G[2], G[2][::-1, :], rtol=1e-14, atol=0)
    assert np.allclose(G[1], -G[1][:, ::-1], rtol=1e-14, atol=1e-30)
    assert np.allclose(G[1], -G[1][::-1, :], rtol=1e-14, atol=1e-30)


def test_contrast_source_exact_on_polynomials():
    """Central differences are exact for quadratics: with dC linear in space and u quadratic, the
    discrete source w^2 drho u + div(dC : grad u) equals the symbolic one (sympy) on cells two or
    more cells from the edge. Catches a wrong index, sign, transposed stiffness or derivative axis."""
    sp = pytest.importorskip("sympy")
    x1, x3 = sp.symbols("x1 x3")
    rng = np.random.default_rng(5)
    c = lambda: complex(rng.normal(), rng.normal())  # noqa: E731
    u1 = c() * x1 ** 2 + c() * x1 * x3 + c() * x3 ** 2 + c() * x1 + c()
    u3 = c() * x1 ** 2 + c() * x1 * x3 + c() * x3 ** 2 + c() * x3 + c()
    lin = lambda s: s * (1 + 0.01 * rng.normal() * x1 + 0.02 * rng.normal() * x3)  # noqa: E731
    drho = lin(150.0)
    C11, C13, C33, C55 = lin(3e8), lin(-1e8), lin(2e8), lin(7e7)
    e1, e3, e5 = sp.diff(u1, x1), sp.diff(u3, x3), sp.diff(u1, x3) + sp.diff(u3, x1)
    s1_1, s1_3, s1_5 = C11 * e1 + C13 * e3, C13 * e1 + C33 * e3, C55 * e5
    omega = 2 * math.pi * 7.0
    s1 = omega ** 2 * drho * u1 + sp.diff(s1_1, x1) + sp.diff(s1_5, x3)
    s3 = omega ** 2 * drho * u3 + sp.diff(s1_5, x1) + sp.diff(s1_3, x3)
    nz, nx, h = 9, 11, 3.0
    X3, X1 = np.meshgrid(np.arange(nz) * h, np.arange(nx) * h, indexing="ij")
    ev = lambda e: np.broadcast_to(sp.lambdify((x1, x3), e, "numpy")(X1, X3), (nz, nx)).astype(complex)  # noqa: E731
    u = np.stack([ev(u1), ev(u3)])
    dmod = np.stack([ev(drho).real, ev(C11).real, ev(C13).real, ev(C33).real, ev(C55).real])
    got = O.contrast_source(u, dmod, omega, h)
    want = np.stack([ev(s1), ev(s3)])
    sl = (slice(None), slice(2, nz - 2), slice(2, nx - 2))
    assert np.max(np.abs(got[sl] - want[sl])) < 1e-9 * np.max(np.abs(want[sl]))


def test_contrast_operator_is_symmetric():
    """With fields zero outside the grid, summation by parts makes the contrast operator
    s(u) = w^2 drho u - D^T dC D u real symmetric: sum v . s(u) = sum u . s(v) (no conjugation)."""
    rng = np.random.default_rng(2)
    nz, nx, h = 7, 6, 5.0
    u = inputs.seeded_complex((2, nz, nx), 1)
    v = inputs.seeded_complex((2, nz, nx), 2)
    dmod = rng.normal(size=(5, nz, nx)) * np.array([100, 1e8, 1e8, 1e8, 1e8])[:, None, None]
    a = np.sum(v * O.contrast_source(u, dmod, 30.0, h))
    b = np.sum(u * O.contrast_source(v, dmod, 30.0, h))
    assert abs(a - b) < 1e-13 * abs(a)


def test_b_matrices_match_appendix_c():
    """The 2D imaging condition uses the {1,3,5} rows/columns of the Appendix C matrices: the
    oracle's gradient for each stiffness equals -Re(eps_a^T B eps_b) with the printed B, and
    C(m + e_p) - C(m) reproduces the printed B restricted to 2D."""
    blocks = {}
    with open(os.path.join(GOLDEN, "appendix_c_b_matrices.txt")) as fh:
        lines = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for k in range(0, len(lines), 7):
        blocks[lines[k][0]] = np.array(lines[k + 1:k + 7], dtype=float)
    idx = [0, 2, 4]  # Voigt 1, 3, 5
    B2 = {name: blocks[name][np.ix_(idx, idx)] for name in blocks}
    assert np.all(B2["B66"] == 0)  # C66 does not enter 2D P-SV
    base = dict(c11=3.0, c13=1.0, c33=2.5, c55=0.7)
    for name, key in (("B11", "c11"), ("B13", "c13"), ("B33", "c33"), ("B55", "c55")):
        pert = dict(base)
        pert[key] += 1.0
        assert np.array_equal(O.voigt_2d(**pert) - O.voigt_2d(**base), B2[name])
    nz, nx, h = 6, 5, 2.0
    ua = inputs.seeded_complex((2, nz, nx), 3)
    ub = inputs.seeded_complex((2, nz, nx), 4)
    g = O.LSOracle.imaging(ua, ub, 3.0, h)
    ea, eb = O.strain(ua, h), O.strain(ub, h)
    for p, name in ((1, "B11"), (2, "B13"), (3, "B33"), (4, "B55")):
        want = -np.real(np.einsum("izx,ij,jzx->zx", ea, B2[name], eb))
        assert np.allclose(g[p], want, rtol=1e-13, atol=0)
    assert np.allclose(g[0], np.real(9.0 * (ua[0] * ub[0] + ua[1] * ub[1])))


@pytest.mark.parametrize("shape,L", [((5, 7), (10, 14)), ((6, 4), (11, 9)), ((8, 8), (16, 16))])
def test_fft_convolution_equals_direct_sum(shape, L):
    """Eq. 12 on the zero-padded grid equals the direct sum over the domain (brute force)."""
    nz, nx = shape
    G = O.green_lattice(nz, nx, 7.0, 2 * math.pi * 11.0, ALPHA, BETA, RHO)
    s = inputs.seeded_complex((2, nz, nx), 9)
    a = O.convolve_direct(s, G, 7.0)
    b = O.convolve_fft(s, O.green_spectrum(G, *L), 7.0)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_incident_field_is_convolution_of_point_force():
    """u0 = G_h(x - x_s) f (Eq. 7) equals h^2 G convolved with the cell-delta f / h^2."""
    w = inputs.small_case(nz=9, nx=7)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    src = np.zeros((2, w.nz, w.nx), dtype=complex)
    src[:, 0, 3] = np.array([0.3, 1.0]) / w.h ** 2
    a = orc.incident(0, (0, 3), (0.3, 1.0))
    b = orc.convolve(src, 0)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


def test_zero_contrast_is_identity():
    """At zero contrast A = I (Eq. 10), so the LS solution is the incident field."""
    w = inputs.small_case(nz=8, nx=6)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    ref = inputs.isotropic_model(w.nz, w.nx, w.rho0, w.alpha0, w.beta0)
    u = inputs.seeded_complex((2, w.nz, w.nx), 5)
    assert np.max(np.abs(orc.apply(u, ref, 0) - u)) < 1e-12 * np.max(np.abs(u))
    u0 = orc.incident(1, (0, 2), (0.0, 1.0))
    assert np.max(np.abs(orc.solve(u0, ref, 1) - u0)) == 0.0


def _neumann(orc, model, f, u0, terms):
    dmod = O.contrast(model, orc.rho0, orc.alpha0, orc.beta0)
    out = u0.copy()
    term = u0.copy()
    for _ in range(terms):
        term = orc.convolve(O.contrast_source(term, dmod, orc.omegas[f], orc.h), f)
        out = out + term
    return out


def test_weak_contrast_matches_born_series():
    """For a weak contrast the BiCGSTAB solution of Eq. 11 equals the Neumann (Born) series."""
    w = inputs.small_case(nz=10, nx=8, amp=0.01)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    u0 = orc.incident(0, (0, 4), (0.3, 1.0))
    u = orc.solve(u0, w.model, 0, tol=1e-14)
    s = _neumann(orc, w.model, 0, u0, 40)
    assert O.normalized_error(u, s) < 1e-11


def test_solution_matches_dense_solve():
    """BiCGSTAB on a 10 % random contrast equals numpy.linalg.solve of the assembled matrix,
    with both the direct-sum and the FFT convolution."""
    w = inputs.small_case(nz=6, nx=5, amp=0.10, vti=True)
    for method in ("direct", "fft"):
        orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas,
                         method=method)
        n = 2 * w.nz * w.nx
        A = np.zeros((n, n), dtype=complex)
        for k in range(n):
            e = np.zeros(n, dtype=complex)
            e[k] = 1.0
            A[:, k] = orc.apply(e.reshape(2, w.nz, w.nx), w.model, 1).reshape(-1)
        u0 = orc.incident(1, (0, 2), (0.3, 1.0))
        want = np.linalg.solve(A, u0.reshape(-1)).reshape(u0.shape)
        got, info = orc.solve_info(u0, w.model, 1, tol=1e-13)
        assert info["converged"]
        assert O.normalized_error(got, want) < 1e-10


def test_reciprocity_of_heterogeneous_response():
    """Discrete reciprocity: the j-component response at x_r to a unit force e_i at x_s equals the
    i-component response at x_s to e_j at x_r (A^{-1} G is complex symmetric)."""
    w = inputs.small_case(nz=9, nx=8, amp=0.15, vti=True)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    xs, xr = (0, 2), (6, 5)
    for i in range(2):
        for j in range(2):
            ui = orc.solve(orc.incident(0, xs, np.eye(2)[i]), w.model, 0)
            uj = orc.solve(orc.incident(0, xr, np.eye(2)[j]), w.model, 0)
            a, b = ui[j][xr], uj[i][xs]
            assert abs(a - b) < 1e-10 * abs(a)


def _small_setup(seed=21, nz=8, nx=7):
    w = inputs.small_case(nz=nz, nx=nx, amp=0.12, vti=True, seed=seed)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx = w.problem_fidx()
    srcs = w.src_cells[w.problem_src()]
    forces = w.src_force[w.problem_src()]
    return w, orc, fidx, srcs, forces


def _data(orc, model, fidx, srcs, forces, rec):
    U = orc.forward(model, fidx, srcs, forces)
    return np.stack([orc.sample(U[b], rec) for b in range(len(fidx))])


def test_frechet_matches_finite_difference_of_forward_map():
    """J dm equals the central finite difference of the discrete forward data map (O(eps^2))."""
    w, orc, fidx, srcs, forces = _small_setup()
    sc = orc.param_scale()[:, None, None]
    dm = sc * inputs.seeded_real((5, w.nz, w.nx), 7)
    U = orc.forward(w.model, fidx, srcs, forces)
    J = orc.frechet(w.model, U, fidx, dm, w.rec_cells)
    errs = []
    for eps in (1e-3, 5e-4):
        dp = _data(orc, w.model + eps * dm, fidx, srcs, forces, w.rec_cells)
        dn = _data(orc, w.model - eps * dm, fidx, srcs, forces, w.rec_cells)
        errs.append(O.normalized_error((dp - dn) / (2 * eps), J))
    assert errs[1] < 1e-6
    assert errs[1] < errs[0] / 3.0  # second order


def test_adjoint_dot_product():
    """<J dm, r> (real part of the complex data inner product) = <dm, Re J^H r> (Eq. B-1, B-2)."""
    w, orc, fidx, srcs, forces = _small_setup(seed=22)
    U = orc.forward(w.model, fidx, srcs, forces)
    dm = inputs.seeded_real((5, w.nz, w.nx), 8) * orc.param_scale()[:, None, None]
    R = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 9)
    lhs = np.real(np.vdot(R, orc.frechet(w.model, U, fidx, dm, w.rec_cells)))
    rhs = np.sum(dm * orc.adjoint(w.model, U, fidx, R, w.rec_cells))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_misfit_gradient_matches_finite_difference():
    """The adjoint-state gradient of Phi = 1/2 ||P u - d_obs||^2 equals the central difference of
    Phi for single-cell perturbations of each parameter."""
    w, orc, fidx, srcs, forces = _small_setup(seed=23, nz=7, nx=6)
    d_obs = _data(orc, w.model * 1.03, fidx, srcs, forces, w.rec_cells)
    phi, g, _ = orc.misfit(w.model, fidx, srcs, forces, d_obs, w.rec_cells)
    sc = orc.param_scale()
    rng = np.random.default_rng(4)
    for _ in range(6):
        p, iz, ix = rng.integers(5), rng.integers(w.nz), rng.integers(w.nx)
        eps = 1e-4 * sc[p]
        mp = w.model.copy()
        mp[p, iz, ix] += eps
        mn = w.model.copy()
        mn[p, iz, ix] -= eps
        fp = orc.misfit(mp, fidx, srcs, forces, d_obs, w.rec_cells)[0]
        fn = orc.misfit(mn, fidx, srcs, forces, d_obs, w.rec_cells)[0]
        fd = (fp - fn) / (2 * eps)
        assert abs(fd - g[p, iz, ix]) < 1e-6 * np.max(np.abs(g[p])) + 1e-8 * abs(fd), (p, fd, g[p, iz, ix])


def test_normal_cg_matches_dense_tikhonov_solve():
    """CG on (Re J~^H J~ + lambda I) x = Re J~^H dd reaches the dense solution built column by
    column from the Frechet and adjoint products; the normal residual shrinks."""
    w, orc, fidx, srcs, forces = _small_setup(seed=24, nz=5, nx=4)
    U = orc.forward(w.model, fidx, srcs, forces)
    dd = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 10) * 1e-12
    sc = orc.param_scale()[:, None, None]
    n = 5 * w.nz * w.nx
    H = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        x = e.reshape(5, w.nz, w.nx)
        H[:, k] = (sc * orc.adjoint(w.model, U, fidx, orc.frechet(w.model, U, fidx, sc * x,
                                                                   w.rec_cells), w.rec_cells)).reshape(-1)
    assert np.allclose(H, H.T, rtol=1e-9, atol=1e-12 * np.max(np.abs(H)))
    lam = 1e-3 * np.max(np.linalg.eigvalsh(0.5 * (H + H.T)))
    rhs = (sc * orc.adjoint(w.model, U, fidx, dd, w.rec_cells)).reshape(-1)
    want = np.linalg.solve(H + lam * np.eye(n), rhs).reshape(5, w.nz, w.nx) * sc
    got, lam_used, hist = orc.normal_cg(w.model, U, fidx, dd, w.rec_cells, iters=150, lam=lam)
    assert O.normalized_error(got, want) < 1e-6
    assert hist[-1] < 1e-6 * hist[0]
    # the power-iteration estimate of lambda_max is a lower bound within a few per cent
    _, lam_est, _ = orc.normal_cg(w.model, U, fidx, dd, w.rec_cells, iters=0,
                                  power_start=inputs.seeded_real((5, w.nz, w.nx), 3), power_iters=10)
    assert 0.5 * lam <= lam_est <= 1.0000001 * lam


# ---------------------------------------------------------------------------------------------
# Orientation of the offset lattice, and the assembled LS solution against the elastic equation
# ---------------------------------------------------------------------------------------------
def _axis_phase_rates(G, nz, nx, h):
    """Mean phase rate (rad/m, positive for outgoing waves under exp(+i w t)) of G11 and G33 along
    the depth offsets (dz, 0), dz = 4..8, and along the lateral offsets (0, dx), dx = 6..14, of a
    lattice laid out as [c][dz + nz - 1][dx + nx - 1]; one-cell steps, so no phase wraps."""
    def rate(line, d0, d1):
        return float(-np.angle(line[d0 + 1:d1 + 1] / line[d0:d1]).mean() / h)
    z = {c: G[c][nz - 1:, nx - 1] for c in (0, 2)}
    x = {c: G[c][nz - 1, nx - 1:] for c in (0, 2)}
    return {"z": {"G11": rate(z[0], 4, 8), "G33": rate(z[2], 4, 8)},
            "x": {"G11": rate(x[0], 6, 14), "G33": rate(x[2], 6, 14)}}


def _orientation_ok(G, nz, nx, h, omega):
    """A unit force along x3 radiates P along x3 and S along x1 (Eq. A-3: with g = e3 the B term
    turns G33 into H0(k_alpha r)/alpha^2 and G11 into H0(k_beta r)/beta^2 in the far field); a force
    along x1 does the opposite. So G33 must travel at k_alpha along depth and at k_beta along x1, and
    G11 the other way round; each rate within 12 % of its wavenumber (near-field terms bend it a
    little at a few wavelengths)."""
    ka, kb = omega / ALPHA, omega / BETA
    r = _axis_phase_rates(G, nz, nx, h)
    want = {"z": {"G33": ka, "G11": kb}, "x": {"G11": ka, "G33": kb}}
    return all(abs(r[a][c] / want[a][c] - 1.0) < 0.12 for a in want for c in want[a]), r


def test_green_lattice_orientation_on_a_non_square_lattice():
    """Entry [c][dz + nz - 1][dx + nx - 1] of the lattice is component c at y = (x1, x3) = (dx h,
    dz h): on a 9 x 15 lattice the depth axis carries the P phase rate in G33 and the S rate in
    G11, the lateral axis the reverse. The same check on a lattice with y1 and y3 exchanged (a
    planted mistake) fails, so the pin sees the orientation that evenness and oddness cannot."""
    nz, nx, h, omega = 9, 15, 10.0, 2 * math.pi * 25.0
    G = O.green_lattice(nz, nx, h, omega, ALPHA, BETA, RHO)
    ok, rates = _orientation_ok(G, nz, nx, h, omega)
    assert ok, rates
    swapped = O.green_lattice(nx, nz, h, omega, ALPHA, BETA, RHO).transpose(0, 2, 1)
    assert swapped.shape == G.shape
    assert not _orientation_ok(swapped, nz, nx, h, omega)[0]


def _div_c_grad(u, model, h):
    """div(C : grad u) of the 2D VTI stiffness (C11, C13, C33, C55 = model[1:5]) by numpy's central
    differences (np.gradient; written apart from the oracle's stencils, exact in the interior)."""
    du1_dz, du1_dx = np.gradient(u[0], h)
    du3_dz, du3_dx = np.gradient(u[1], h)
    c11, c13, c33, c55 = model[1], model[2], model[3], model[4]
    s1 = c11 * du1_dx + c13 * du3_dz
    s3 = c13 * du1_dx + c33 * du3_dz
    s5 = c55 * (du1_dz + du3_dx)
    return np.stack([np.gradient(s1, h, axis=1) + np.gradient(s5, h, axis=0),
                     np.gradient(s5, h, axis=1) + np.gradient(s3, h, axis=0)])


def _elastic_residual_under_refinement(levels=3):
    """Relative residual of the heterogeneous elastic equation w^2 rho u + div(C : grad u) = 0
    (Eq. 3, away from the source) for the assembled LS solution u = A^-1 u0 (Eq. 11) on grids of
    spacing 20, 10, 5 m over one physical domain (240 m x 360 m, the coarse samples kept in every
    finer grid): a smooth anisotropic Gaussian contrast (sigma 45 m, +10 % rho, +12 % C11, -8 % C13,
    +10 % C33, +15 % C55) that vanishes at the edges of D, a 6 Hz point force away from it, and the
    residual by central differences at the coarse samples three cells from the edges and four from
    the source, relative to max w^2 rho |u| there. Returns one value per level."""
    out = []
    nz0, nx0, h0 = 13, 19, 20.0
    omega = 2 * math.pi * 6.0
    ref = O.reference_params(RHO, ALPHA, BETA)
    pert = np.array([0.10, 0.12, -0.08, 0.10, 0.15])
    for lev in range(levels):
        s = 2 ** lev
        nz, nx, h = (nz0 - 1) * s + 1, (nx0 - 1) * s + 1, h0 / s
        z = np.arange(nz)[:, None] * h
        x = np.arange(nx)[None, :] * h
        bump = np.exp(-((z - 160.0) ** 2 + (x - 220.0) ** 2) / (2 * 45.0 ** 2))
        model = ref[:, None, None] * (1 + pert[:, None, None] * bump[None])
        orc = O.LSOracle(nz, nx, h, 2 * nz, 2 * nx, RHO, ALPHA, BETA, [omega])
        u, info = orc.solve_info(orc.incident(0, (2 * s, 3 * s), (0.3, 1.0)), model, 0, tol=1e-13)
        assert info["converged"]
        R = omega ** 2 * model[0] * u + _div_c_grad(u, model, h)
        Z, X = np.meshgrid(np.arange(3, nz0 - 3) * s, np.arange(3, nx0 - 3) * s, indexing="ij")
        keep = np.hypot(Z / s - 2, X / s - 3) >= 4
        res = np.abs(R[:, Z, X])[:, keep].max()
        scale = np.abs(omega ** 2 * model[0][Z, X][keep] * u[:, Z, X][:, keep]).max()
        out.append(float(res / scale))
    return out


def _converges(r):
    # second order: the residual falls about 4x per halving of h (3.9x observed)
    return r[-1] < 0.02 and all(a > 3.0 * b for a, b in zip(r, r[1:]))


def test_ls_solution_solves_the_elastic_equation():
    """The discrete LS solution converges to a solution of the heterogeneous elastic wave equation:
    its finite-difference residual falls as O(h^2) under refinement (0.17, 0.044, 0.011). This ties
    the whole assembled operator (lattice, self cell, stencils, contrast, convolution, solve) to
    the physics rather than to itself."""
    r = _elastic_residual_under_refinement()
    assert _converges(r), r


@pytest.mark.parametrize("plant", ["swap_lattice_axes", "divergence_sign", "drop_density_term"])
def test_elastic_equation_pin_catches_planted_errors(plant, monkeypatch):
    """Planted mistakes in the oracle (y1 and y3 exchanged in the lattice, the stress divergence
    with the wrong sign, the w^2 drho u term left out) each stop the residual from converging."""
    import oracle.dbi_oracle as D
    if plant == "swap_lattice_axes":
        lat = D.green_lattice
        monkeypatch.setattr(D, "green_lattice",
                            lambda nz, nx, h, w, a, b, r: lat(nx, nz, h, w, a, b, r).transpose(0, 2, 1))
    elif plant == "divergence_sign":
        monkeypatch.setattr(D, "contrast_source", lambda u, dm, w, h: w * w * dm[0] * u
                            - D.divergence(D.stress(D.strain(u, h), dm), h))
    else:
        monkeypatch.setattr(D, "contrast_source", lambda u, dm, w, h: D.divergence(D.stress(D.strain(u, h), dm), h))
    assert not _converges(_elastic_residual_under_refinement())

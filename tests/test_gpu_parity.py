"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 unless stated): complex128 path 1e-10 for single operator passes, 1e-8
for solves; complex64 path 1e-5 for wavefields and data (the wavefield tolerance of the
benchmark configurations) and 1e-4 for gradients. The complex64 bound comes from FP32 rounding
(u = 6e-8) amplified by the O(log L) depth of the FFTs and the stencil's cancellation.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.problem import DeviceProblem

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {dbi.C64: 1e-5, dbi.C128: 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def npy(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_for(w, method="fft"):
    return O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas, method=method)


SHAPES = [
    dict(nz=12, nx=10),                  # ragged, single tile
    dict(nz=5, nx=9, lz=16, lx=32),      # non-square FFT grid
    dict(nz=1, nx=8),                    # one row
    dict(nz=40, nx=24, vti=True),        # several row tiles, VTI background
    dict(nz=64, nx=64, lz=128, lx=128),  # several column tiles
    dict(nz=21, nx=30, lz=64, lx=512, vti=True),  # 512-long rows (one thread per column), ragged
    dict(nz=9, nx=256, lz=32, lx=512),   # 512-long rows at full width (nx = 256)
]


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("nz", "nx")))
def test_greens_tables(precision, shape):
    w = inputs.small_case(freqs=(3.0, 17.0), **shape)
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    # FP64: CUDA's and scipy's Bessel routines differ by a few ulp, amplified near the zeros of
    # J_n, Y_n and by the cancellation of the 1/r^2 parts of H2 between the P and S terms
    tol = 1e-10 if precision == dbi.C128 else 1e-6
    for f in range(w.nf):
        Gs = O.embed_circulant(orc.G_lat[f], w.lz, w.lx)
        assert rel(npy(P.Gspace[f]), Gs) < tol
        Gh = orc.G_hat[f] * w.h * w.h / (w.lz * w.lx)
        assert rel(npy(P.Ghat[f]), np.swapaxes(Gh, -1, -2)) < 10 * tol  # stored [c][kx][kz]


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_incident_field(precision):
    w = inputs.small_case(nz=14, nx=11, n_src=3, freqs=(6.0, 11.0))
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    u0 = npy(P.incident())
    srcs = w.problem_src()
    for b, f in enumerate(w.problem_fidx()):
        want = orc.incident(f, w.src_cells[srcs[b]], w.src_force[srcs[b]])
        assert rel(u0[b], want) < (1e-10 if precision == dbi.C128 else 1e-6)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("nz", "nx")))
def test_green_convolve(precision, shape):
    w = inputs.small_case(freqs=(5.0, 12.0), **shape)
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    src = inputs.seeded_complex((w.n_problems, 2, w.nz, w.nx), 3)
    out = npy(P.convolve(P.to_field(src)))
    for b, f in enumerate(w.problem_fidx()):
        assert rel(out[b], orc.convolve(src[b], f)) < TOL[precision]


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("nz", "nx")))
def test_ls_apply(precision, shape):
    w = inputs.small_case(freqs=(7.0, 15.0), amp=0.15, **shape)
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    u = inputs.seeded_complex((w.n_problems, 2, w.nz, w.nx), 4)
    out = npy(P.apply(P.to_field(u)))
    for b, f in enumerate(w.problem_fidx()):
        want = orc.apply(u[b], w.model, f)
        assert rel(out[b], want) < TOL[precision]
        # the scattered part alone (A u - u) also matches to the same relative accuracy
        assert rel(out[b] - u[b], want - u[b]) < 20 * TOL[precision]


def test_ls_apply_direct_sum_tiny():
    """The operator equals the oracle's direct O(N^4) sum (no FFT on the oracle side)."""
    w = inputs.small_case(nz=7, nx=6, amp=0.2, vti=True)
    P = DeviceProblem(w, dbi.C128)
    orc = oracle_for(w, method="direct")
    u = inputs.seeded_complex((w.n_problems, 2, w.nz, w.nx), 5)
    out = npy(P.apply(P.to_field(u)))
    for b, f in enumerate(w.problem_fidx()):
        assert rel(out[b], orc.apply(u[b], w.model, f)) < 1e-10


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_ls_solve(precision):
    w = inputs.small_case(nz=20, nx=18, amp=0.12, vti=True, n_src=2, freqs=(6.0, 13.0))
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    u, iters, relres, code = P.forward(tol=tol)
    u = npy(u)
    assert np.all(npy(code) == dbi.CONVERGED)
    assert np.all(npy(relres) <= tol)
    srcs = w.problem_src()
    for b, f in enumerate(w.problem_fidx()):
        want = orc.solve(orc.incident(f, w.src_cells[srcs[b]], w.src_force[srcs[b]]), w.model, f, tol=1e-13)
        assert rel(u[b], want) < (1e-8 if precision == dbi.C128 else 1e-5)


def test_config1_tiny_complex128():
    """The 32 x 32 isotropic inclusion case, complex128 BiCGSTAB to 1e-8, against the oracle."""
    w = inputs.config1_tiny()
    P = DeviceProblem(w, dbi.C128)
    orc = oracle_for(w)
    u, iters, relres, code = P.forward(tol=1e-8)
    assert npy(code)[0] == dbi.CONVERGED and npy(relres)[0] <= 1e-8
    want = orc.solve(orc.incident(0, w.src_cells[0], w.src_force[0]), w.model, 0, tol=1e-13)
    assert rel(npy(u)[0], want) < 1e-7
    d = npy(P.sample(u))[0]
    assert rel(d, orc.sample(want, w.rec_cells)) < 1e-7


def test_solver_status_and_edge_cases():
    w = inputs.small_case(nz=10, nx=10, amp=0.1)
    P = DeviceProblem(w, dbi.C64)
    u0 = P.incident()
    # an iteration cap of one leaves the problems unconverged after exactly one iteration
    _, iters, relres, code = P.solve(u0, tol=1e-12, max_iter=1, check_every=1)
    assert np.all(npy(iters) == 1) and np.all(npy(code) == dbi.NOT_CONVERGED)
    # a zero right-hand side converges at once to zero, whatever the initial guess
    z = torch.zeros_like(u0)
    x, iters, relres, code = P.solve(z, u0=u0, tol=1e-6)
    assert np.all(npy(code) == dbi.CONVERGED) and np.all(npy(iters) == 0)
    assert float(torch.abs(x).max()) == 0.0
    # the solver is scale-invariant: a right-hand side of 2^-90 (squares far below FP32's range)
    # gives the same solution scaled by 2^-90
    x, _, _, code = P.solve(u0, tol=1e-6)
    xt, _, _, code_t = P.solve(u0 * 2.0 ** -90, tol=1e-6)
    assert np.all(npy(code_t) == dbi.CONVERGED)
    assert rel(npy(xt).astype(np.complex128) * 2.0 ** 90, npy(x)) < 1e-6
    # a converged initial guess takes no iterations
    _, iters, _, code = P.solve(u0, u0=x, tol=1e-3)
    assert np.all(npy(iters) == 0)
    # an empty batch is a no-op
    w0 = inputs.small_case(nz=8, nx=8, n_src=0 + 1, freqs=(5.0,))
    P0 = DeviceProblem(w0, dbi.C64)
    empty = torch.zeros((0, 2, 8, 8), dtype=torch.complex64, device="cuda")
    out = dbi.ls_apply(P0.grid, P0.ref, P0.m, P0.omega, P0.fidx[:0], P0.Ghat, empty)
    assert out.shape == (0, 2, 8, 8)


def test_largest_fft_grid():
    """512 x 512 cells on the 1024 x 1024 FFT grid (the largest supported), one problem."""
    w = inputs.small_case(nz=512, nx=512, n_src=1, freqs=(9.0,), amp=0.1, h=5.0)
    P = DeviceProblem(w, dbi.C64)
    orc = oracle_for(w)
    u = inputs.seeded_complex((1, 2, 512, 512), 6)
    out = npy(P.apply(P.to_field(u)))
    assert rel(out[0], orc.apply(u[0], w.model, 0)) < TOL[dbi.C64]
    # the solver's fused kernels on the same grid; the FP64 oracle confirms the residual
    u0 = P.incident()
    x, _, relres, code = P.solve(u0, tol=1e-5)
    assert int(npy(code)[0]) == dbi.CONVERGED
    x0, b0 = npy(x)[0].astype(np.complex128), npy(u0)[0].astype(np.complex128)
    assert rel(orc.apply(x0, w.model, 0), b0) < 3e-5


def _dbi_setup(precision, seed=31):
    w = inputs.small_case(nz=12, nx=11, amp=0.12, vti=True, n_src=2, freqs=(7.0, 12.0), seed=seed)
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    fidx = w.problem_fidx()
    srcs = w.src_cells[w.problem_src()]
    forces = w.src_force[w.problem_src()]
    U = orc.forward(w.model, fidx, srcs, forces)
    return w, P, orc, fidx, U


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_frechet_apply(precision):
    w, P, orc, fidx, U = _dbi_setup(precision)
    dm = inputs.seeded_real((5, w.nz, w.nx), 12) * orc.param_scale()[:, None, None] * 0.01
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    d = npy(P.frechet(P.to_field(U), P.to_model(dm), tol=tol))
    want = orc.frechet(w.model, U, fidx, dm, w.rec_cells)
    assert rel(d, want) < (1e-8 if precision == dbi.C128 else 1e-5)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_adjoint_apply(precision):
    w, P, orc, fidx, U = _dbi_setup(precision)
    R = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 13)
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    g = npy(P.adjoint(P.to_field(U), P.to_field(R), tol=tol))
    want = orc.adjoint(w.model, U, fidx, R, w.rec_cells)
    for p in range(5):
        assert rel(g[p], want[p]) < (1e-8 if precision == dbi.C128 else 1e-4), p


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_gpu_dot_product_test(precision):
    """<J dm, r> = <dm, Re J^H r> with both products from the CUDA path."""
    w, P, orc, fidx, U = _dbi_setup(precision, seed=33)
    tol = 1e-12 if precision == dbi.C128 else 1e-7
    Ub = P.to_field(U)
    dm = inputs.seeded_real((5, w.nz, w.nx), 14) * orc.param_scale()[:, None, None] * 0.01
    R = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 15)
    Jd = npy(P.frechet(Ub, P.to_model(dm), tol=tol)).astype(np.complex128)
    g = npy(P.adjoint(Ub, P.to_field(R), tol=tol)).astype(np.float64)
    lhs = np.real(np.vdot(R, Jd))
    rhs = np.sum(npy(P.to_model(dm)).astype(np.float64) * g)
    assert abs(lhs - rhs) / abs(lhs) < (1e-10 if precision == dbi.C128 else 1e-5)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_data_residual(precision):
    w, P, orc, fidx, U = _dbi_setup(precision)
    dobs = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 16) * 1e-10
    r, phi = P.residual(P.to_field(U), P.to_field(dobs))
    want = np.stack([orc.sample(U[b], w.rec_cells) for b in range(len(fidx))]) - dobs
    assert rel(npy(r), want) < (1e-12 if precision == dbi.C128 else 1e-6)
    assert abs(float(phi.detach()) - 0.5 * np.sum(np.abs(want) ** 2)) < 1e-5 * 0.5 * np.sum(np.abs(want) ** 2)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_normal_cg(precision):
    """complex128: lambda, the residual history and dm match the oracle's CG step for step.
    complex64: an unconverged CG iterate is sensitive to the operator's rounding (relative noise of
    1e-5 in each Hessian application moves the 12th oracle iterate by about 6 %), so the check is
    on what the iterate achieves: the FP64 oracle evaluates the normal-equation residual of the
    GPU's dm, which must be as small as that of the oracle's own iterate."""
    w = inputs.small_case(nz=8, nx=7, amp=0.1, vti=True, n_src=2, freqs=(8.0, 13.0), seed=41)
    P = DeviceProblem(w, precision)
    orc = oracle_for(w)
    fidx = w.problem_fidx()
    U = orc.forward(w.model, fidx, w.src_cells[w.problem_src()], w.src_force[w.problem_src()])
    dd = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 17) * 1e-12
    start = inputs.seeded_real((5, w.nz, w.nx), 18)
    tol = 1e-12 if precision == dbi.C128 else 1e-7
    dm, lam, hist = P.normal_cg(P.to_field(U), P.to_field(dd), iters=12, power_start=start, tol=tol)
    want, lam_o, hist_o = orc.normal_cg(w.model, U, fidx, dd, w.rec_cells, iters=12, power_start=start)
    lam_err = abs(lam - lam_o) / lam_o
    if precision == dbi.C128:
        assert lam_err < 1e-8
        assert rel(np.asarray(hist), np.asarray(hist_o)) < 1e-7
        assert rel(npy(dm), want) < 1e-7
        return
    assert lam_err < 5e-4
    sc = orc.param_scale()[:, None, None]

    def normal_residual(dmv):
        x = dmv / sc
        Hx = sc * orc.adjoint(w.model, U, fidx, orc.frechet(w.model, U, fidx, sc * x, w.rec_cells), w.rec_cells)
        rhs = sc * orc.adjoint(w.model, U, fidx, dd, w.rec_cells)
        return np.linalg.norm(rhs - Hx - lam_o * x), np.linalg.norm(rhs)

    r_gpu, r0 = normal_residual(npy(dm).astype(np.float64))
    r_orc, _ = normal_residual(want)
    assert r_gpu < 1.3 * r_orc and r_gpu < 0.2 * r0, (r_gpu / r0, r_orc / r0)
    assert hist[-1] < 0.2 * hist[0]


@pytest.mark.parametrize("lz,lx", [(1024, 16), (768, 32)])
def test_normal_cg_on_the_split_stages(lz, lx):
    """The Tikhonov normal-equation CG (Frechet and adjoint solves in every step) on the complex64
    stages of FFT lengths 1024 and 768: the normal-equation residual of the GPU's 12th iterate,
    evaluated by the FP64 oracle, is as small as that of the oracle's own iterate."""
    w = inputs.small_case(nz=8, nx=7, lz=lz, lx=lx, amp=0.1, vti=True, n_src=2, freqs=(8.0, 13.0), seed=41)
    P = DeviceProblem(w, dbi.C64)
    orc = oracle_for(w)
    fidx = w.problem_fidx()
    U = orc.forward(w.model, fidx, w.src_cells[w.problem_src()], w.src_force[w.problem_src()])
    dd = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 17) * 1e-12
    start = inputs.seeded_real((5, w.nz, w.nx), 18)
    dm, lam, hist = P.normal_cg(P.to_field(U), P.to_field(dd), iters=12, power_start=start, tol=1e-7)
    want, lam_o, _ = orc.normal_cg(w.model, U, fidx, dd, w.rec_cells, iters=12, power_start=start)
    assert abs(lam - lam_o) / lam_o < 5e-4
    sc = orc.param_scale()[:, None, None]

    def normal_residual(dmv):
        x = dmv / sc
        Hx = sc * orc.adjoint(w.model, U, fidx, orc.frechet(w.model, U, fidx, sc * x, w.rec_cells), w.rec_cells)
        rhs = sc * orc.adjoint(w.model, U, fidx, dd, w.rec_cells)
        return np.linalg.norm(rhs - Hx - lam_o * x), np.linalg.norm(rhs)

    r_gpu, r0 = normal_residual(npy(dm).astype(np.float64))
    r_orc, _ = normal_residual(want)
    assert r_gpu < 1.3 * r_orc and r_gpu < 0.2 * r0, (r_gpu / r0, r_orc / r0)


# --- the batched-forward workload at full size, in the benchmark's launch configuration --------
@pytest.fixture(scope="module")
def config2():
    w = inputs.config2_batched_forward()
    return w, DeviceProblem(w, dbi.C64)


def test_config2_apply_sampled(config2):
    """All 256 problems of the 256 x 256 VTI workload in one batched apply; two problems (two
    frequencies) checked against the oracle."""
    w, P = config2
    orc = oracle_for(w)
    u = P.incident()
    out = npy(P.apply(u))
    un = npy(u)
    for b in (3, w.n_problems - 5):
        f = int(w.problem_fidx()[b])
        assert rel(out[b], orc.apply(un[b].astype(np.complex128), w.model, f)) < TOL[dbi.C64]


def test_config2_solve_residual_sampled(config2):
    """The batched complex64 solve converges for all 256 problems; for sampled problems the FP64
    oracle confirms the residual of the returned wavefield (a property that holds at any size)."""
    w, P = config2
    orc = oracle_for(w)
    u0 = P.incident()
    u, iters, relres, code = P.solve(u0, tol=1e-5, max_iter=3000)
    assert np.all(npy(code) == dbi.CONVERGED), np.unique(npy(code), return_counts=True)
    un, u0n = npy(u).astype(np.complex128), npy(u0).astype(np.complex128)
    for b in (0, w.n_problems - 1):
        f = int(w.problem_fidx()[b])
        res = rel(orc.apply(un[b], w.model, f), u0n[b])
        assert res < 3e-5, (b, res, float(npy(relres)[b]))


# --- the linear DBI step at full size: 128 x 128, 16 sources x 4 frequencies, 30 CG iterations --
def test_config3_linear_dbi_step():
    """Frechet and adjoint products of the 64-problem DBI step pass the dot-product test to 1e-5
    (complex64), and 30 normal-equation CG iterations with lambda = 1e-3 of the power-iteration
    estimate of ||J||^2 reduce both the normal residual and the linearised data misfit."""
    w = inputs.config3_linear_dbi()
    P = DeviceProblem(w, dbi.C64)
    u_b, _, _, code = P.forward(tol=1e-6)
    assert bool((code == dbi.CONVERGED).all())
    # data residual of the true model against the background
    Pt = DeviceProblem(w, dbi.C64, model=w.model_true)
    u_t, _, _, code = Pt.forward(tol=1e-6)
    assert bool((code == dbi.CONVERGED).all())
    dd = Pt.sample(u_t) - P.sample(u_b)
    del u_t, Pt
    a2 = w.rho0 * w.alpha0 ** 2
    sc = np.array([w.rho0, a2, a2, a2, w.rho0 * w.beta0 ** 2])[:, None, None]
    dm = P.to_model(inputs.seeded_real((5, w.nz, w.nx), 31) * sc * 1e-3)
    R = P.to_field(inputs.seeded_complex((P.B, len(w.rec_cells), 2), 32) * 1e-12)
    Jd = npy(P.frechet(u_b, dm, tol=1e-7)).astype(np.complex128)
    g = npy(P.adjoint(u_b, R, tol=1e-7)).astype(np.float64)
    lhs = np.real(np.vdot(npy(R).astype(np.complex128), Jd))
    rhs = float(np.sum(npy(dm).astype(np.float64) * g))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    start = inputs.seeded_real((5, w.nz, w.nx), 33)
    dm_cg, lam, hist = P.normal_cg(u_b, dd, iters=30, lambda_rel=1e-3, power_iters=10, power_start=start,
                                   tol=1e-6)
    assert lam > 0 and np.all(np.isfinite(hist))
    assert hist[-1] < 0.05 * hist[0]
    pred = P.frechet(u_b, dm_cg, tol=1e-6)
    r0 = float(torch.linalg.norm(dd.to(torch.complex128)))
    r1 = float(torch.linalg.norm((dd - pred).to(torch.complex128)))
    assert r1 < 0.5 * r0, (r1 / r0)


@pytest.mark.parametrize("L", [16, 32, 128, 256, 1024])
@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_second_radix_plan_matches_oracle(L, precision):
    """The radix order with the smaller radix first (plan 1) gives the same operator."""
    n = min(L // 2, 24)
    w = inputs.small_case(nz=n, nx=max(1, n - 3), lz=L, lx=L, vti=True, n_src=2, freqs=(9.0,), seed=L)
    P = DeviceProblem(w, precision)
    u = torch.as_tensor(inputs.seeded_complex((P.B, 2, w.nz, w.nx), L + 1)).to(P.device, P.cdt)
    orc = oracle_for(w)
    try:
        dbi.set_radix_plan(precision, L, 1)
        out = npy(P.apply(u))
    finally:
        dbi.set_radix_plan(precision, L, 0)
    for b in range(P.B):
        want = orc.apply(npy(u[b]).astype(np.complex128), w.model, 0)
        assert rel(out[b], want) < TOL[precision], b


def test_binding_rejects_host_or_mistyped_outputs_with_device_inputs():
    """With device inputs, a host output, an output of the other precision and a Green's table of
    the other precision or size are errors before the library is called (each would have the
    kernels write through a host address or past the tensor's end)."""
    w = inputs.small_case(nz=6, nx=5, n_src=1, freqs=(8.0,))
    P = DeviceProblem(w, dbi.C64)
    u = P.incident()
    n0 = dbi.kernel_launches()
    with pytest.raises(dbi.DBIError, match="CUDA tensor"):
        dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=torch.empty_like(u, device="cpu"))
    with pytest.raises(dbi.DBIError, match="needs"):
        dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, out=u.to(torch.complex128))
    with pytest.raises(dbi.DBIError, match="needs"):
        dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat.to(torch.complex128), u)
    with pytest.raises(dbi.DBIError, match="FFT-grid points"):
        dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat[:, :2].contiguous(), u)
    with pytest.raises(dbi.DBIError, match="CUDA tensor"):
        dbi.ls_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat.cpu(), u)
    assert dbi.kernel_launches() == n0


# FFT length 1024 (complex64) runs each half-pruned transform as two 512-point transforms and the
# contrast source by its own kernel in chunks of 32 rows: ragged row and column counts, one row,
# one column, and 1024 along one axis only.
SPLIT_SHAPES = [
    dict(nz=37, nx=300, lz=1024, lx=1024),   # two source chunks, ragged columns
    dict(nz=1, nx=511, lz=16, lx=1024),      # one row, split rows only
    dict(nz=500, nx=1, lz=1024, lx=16),      # one column, split columns only
    dict(nz=70, nx=45, lz=1024, lx=128),     # split columns, a partial source chunk
    dict(nz=64, nx=512, lz=128, lx=1024, vti=True),  # full-width rows, split rows
]


@pytest.mark.parametrize("shape", SPLIT_SHAPES, ids=lambda s: f"{s['nz']}x{s['nx']}_L{s['lz']}x{s['lx']}")
def test_length_1024_split_stages(shape):
    w = inputs.small_case(freqs=(4.0, 15.0), n_src=2, amp=0.12, h=5.0, **shape)
    P = DeviceProblem(w, dbi.C64)
    orc = oracle_for(w)
    u = inputs.seeded_complex((P.B, 2, w.nz, w.nx), 77)
    out = npy(P.apply(P.to_field(u)))
    conv = npy(P.convolve(P.to_field(u)))
    for b, f in enumerate(w.problem_fidx()):
        want = orc.apply(u[b], w.model, f)
        assert rel(out[b] - u[b], want - u[b]) < TOL[dbi.C64], b
        assert rel(conv[b], orc.convolve(u[b].astype(np.complex128), f)) < TOL[dbi.C64], b
    # the fused inner products of the solver on the same stages
    u0 = P.incident()
    x, _, _, code = P.solve(u0, tol=1e-6)
    assert np.all(npy(code) == dbi.CONVERGED)
    xs, bs = npy(x).astype(np.complex128), npy(u0).astype(np.complex128)
    for b, f in enumerate(w.problem_fidx()):
        ref = orc.solve(bs[b], w.model, f, tol=1e-12)
        assert rel(xs[b], ref) < 1e-5, b


# FFT length 768 = 3 x 256 (complex64): each half-pruned transform as three 256-point transforms of
# the folded, twiddled line, the contrast source by the 32-row source kernel, the Green's tables by
# the FP64 768-point table FFT (stored residue-major along kz). Ragged rows and columns, more than
# 256 points (the fold's second third), one row, one column, 768 along one axis only and beside
# 1024 along the other.
S3_SHAPES = [
    dict(nz=37, nx=300, lz=768, lx=768),     # ragged, nx > 256
    dict(nz=1, nx=384, lz=16, lx=768),       # one row at full width, triple rows only
    dict(nz=384, nx=1, lz=768, lx=16),       # one column at full height, triple columns only
    dict(nz=130, nx=45, lz=768, lx=128, vti=True),  # triple columns, a partial source chunk
    dict(nz=200, nx=380, lz=768, lx=1024),   # triple columns beside pair rows
    dict(nz=300, nx=257, lz=1024, lx=768),   # pair columns beside triple rows
]


def residue_major_to_natural(Ghat_kz_last, lz):
    """Entries [..., kz] in natural order from the stored order (residue-major at lz = 768)."""
    if lz != 768:
        return Ghat_kz_last
    slots = np.array([(k % 3) * 256 + k // 3 for k in range(768)])
    return Ghat_kz_last[..., slots]


@pytest.mark.parametrize("shape", S3_SHAPES, ids=lambda s: f"{s['nz']}x{s['nx']}_L{s['lz']}x{s['lx']}")
def test_length_768_triple_stages(shape):
    w = inputs.small_case(freqs=(4.0, 15.0), n_src=2, amp=0.12, h=5.0, **shape)
    P = DeviceProblem(w, dbi.C64)
    orc = oracle_for(w)
    for f in range(w.nf):
        Gh = np.swapaxes(orc.G_hat[f] * w.h * w.h / (w.lz * w.lx), -1, -2)  # [c][kx][kz]
        assert rel(residue_major_to_natural(npy(P.Ghat[f]), w.lz), Gh) < 1e-5, f
        assert rel(npy(P.Gspace[f]), O.embed_circulant(orc.G_lat[f], w.lz, w.lx)) < 1e-6, f
    u = inputs.seeded_complex((P.B, 2, w.nz, w.nx), 78)
    out = npy(P.apply(P.to_field(u)))
    conv = npy(P.convolve(P.to_field(u)))
    for b, f in enumerate(w.problem_fidx()):
        want = orc.apply(u[b], w.model, f)
        assert rel(out[b] - u[b], want - u[b]) < TOL[dbi.C64], b
        assert rel(conv[b], orc.convolve(u[b].astype(np.complex128), f)) < TOL[dbi.C64], b
    # the incident field and the solver's fused inner products on the same stages
    u0 = P.incident()
    srcs = w.problem_src()
    x, _, _, code = P.solve(u0, tol=1e-6)
    assert np.all(npy(code) == dbi.CONVERGED)
    xs, bs = npy(x).astype(np.complex128), npy(u0).astype(np.complex128)
    for b, f in enumerate(w.problem_fidx()):
        assert rel(bs[b], orc.incident(f, w.src_cells[srcs[b]], w.src_force[srcs[b]])) < 1e-6, b
        assert rel(xs[b], orc.solve(bs[b], w.model, f, tol=1e-12)) < 1e-5, b


def test_length_768_products():
    """The distorted-Born products on the length-768 stages: the Frechet derivative against the
    oracle, and the dot test between it and the adjoint imaging."""
    w = inputs.small_case(nz=40, nx=300, lz=128, lx=768, amp=0.12, vti=True, n_src=2, freqs=(7.0, 12.0),
                          seed=35, h=5.0)
    P = DeviceProblem(w, dbi.C64)
    orc = oracle_for(w)
    fidx = w.problem_fidx()
    U = orc.forward(w.model, fidx, w.src_cells[w.problem_src()], w.src_force[w.problem_src()])
    Ub = P.to_field(U)
    dm = inputs.seeded_real((5, w.nz, w.nx), 16) * orc.param_scale()[:, None, None] * 0.01
    Jd = npy(P.frechet(Ub, P.to_model(dm), tol=1e-7)).astype(np.complex128)
    assert rel(Jd, orc.frechet(w.model, U, fidx, dm, w.rec_cells)) < 1e-5
    R = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 17)
    g = npy(P.adjoint(Ub, P.to_field(R), tol=1e-7)).astype(np.float64)
    lhs = np.real(np.vdot(R, Jd))
    rhs = np.sum(npy(P.to_model(dm)).astype(np.float64) * g)
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_length_768_largest_grid():
    """384 x 384 VTI cells on the 768 x 768 FFT grid (the largest grid length 768 serves), two
    frequencies: the operator against the oracle, and the solver's fused kernels on the same grid,
    whose solution the FP64 oracle's operator confirms by its residual."""
    w = inputs.small_case(nz=384, nx=384, lz=768, lx=768, n_src=1, freqs=(6.0, 14.0), amp=0.1, h=5.0,
                          vti=True, seed=12)
    P = DeviceProblem(w, dbi.C64)
    orc = oracle_for(w)
    u = inputs.seeded_complex((P.B, 2, 384, 384), 79)
    out = npy(P.apply(P.to_field(u)))
    for b, f in enumerate(w.problem_fidx()):
        want = orc.apply(u[b], w.model, f)
        assert rel(out[b] - u[b], want - u[b]) < TOL[dbi.C64], b
    u0 = P.incident()
    x, _, _, code = P.solve(u0, tol=1e-5)
    assert np.all(npy(code) == dbi.CONVERGED)
    xs, bs = npy(x).astype(np.complex128), npy(u0).astype(np.complex128)
    for b, f in enumerate(w.problem_fidx()):
        assert rel(orc.apply(xs[b], w.model, f), bs[b]) < 3e-5, b

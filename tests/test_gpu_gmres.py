"""Restarted GMRES on the GPU (ls_solve_gmres) against the FP64 oracle's GMRES and BiCGSTAB: the
iterate after k Arnoldi steps of one cycle equals the oracle's (the minimal-residual iterate of
the same Krylov space), converged solutions match with and without restarts in both precisions,
initial guesses, zero right-hand sides and the iteration limit behave as stated, and the full
256^2 batch converges with the true residual of sampled problems checked by the oracle's
operator."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.problem import DeviceProblem

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def npy(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_for(w):
    return O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)


def oracle_gmres(orc, w, q, rhs, restart, tol, maxiter, x0=None):
    shape = rhs.shape
    f = int(w.problem_fidx()[q])
    x, info = O.gmres(lambda v: orc.apply(v.reshape(shape), w.model, f).reshape(-1), rhs.reshape(-1),
                      restart=restart, tol=tol, maxiter=maxiter,
                      x0=None if x0 is None else x0.reshape(-1))
    return x.reshape(shape), info


@pytest.mark.parametrize("k", [1, 4, 9])
def test_one_cycle_equals_the_oracle_iterate(k):
    """k steps of one cycle, no convergence test (tol 0): the minimal-residual iterate of the
    Krylov space, so the GPU and the oracle agree to rounding, whatever Gram-Schmidt variant."""
    w = inputs.small_case(nz=12, nx=10, n_src=2, freqs=(8.0, 14.0))
    P = DeviceProblem(w, dbi.C128)
    u0 = P.incident()
    u, iters, relres, code = P.solve_gmres(u0, restart=k, tol=0.0, max_iter=k, check_every=0)
    assert bool((iters == k).all()) and bool((code == dbi.NOT_CONVERGED).all())
    orc = oracle_for(w)
    for q in range(P.B):
        x, info = oracle_gmres(orc, w, q, npy(u0[q]), restart=k, tol=0.0, maxiter=k)
        assert rel(npy(u[q]), x) < 1e-10, q
        assert float(relres[q]) == pytest.approx(info["resvec"][-1], rel=1e-8)


SHAPES = [
    dict(nz=12, nx=10),
    dict(nz=5, nx=9, lz=16, lx=32),
    dict(nz=1, nx=8),
    dict(nz=40, nx=24, vti=True),
    dict(nz=21, nx=30, lz=64, lx=512, vti=True),
]


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("restart", [30, 5])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(str(s[k]) for k in ("nz", "nx")))
def test_solution_matches_oracle(precision, restart, shape):
    w = inputs.small_case(freqs=(6.0, 13.0), n_src=2, **shape)
    P = DeviceProblem(w, precision)
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    u, iters, relres, code = P.solve_gmres(P.incident(), restart=restart, tol=tol, max_iter=800, check_every=4)
    assert bool((code == dbi.CONVERGED).all()) and float(relres.max()) <= tol
    orc = oracle_for(w)
    fidx, srcs = w.problem_fidx(), w.problem_src()
    for q in range(P.B):
        u0 = orc.incident(fidx[q], w.src_cells[srcs[q]], w.src_force[srcs[q]])
        want = orc.solve(u0, w.model, fidx[q], tol=1e-13)
        assert rel(npy(u[q]), want) < (1e-8 if precision == dbi.C128 else 1e-5), q


# GMRES over the complex64 stages of FFT lengths 1024 (pairs of 512-point transforms) and 768
# (triples of 256-point transforms), whose kernels complex128 does not use.
SPLIT_SHAPES = [
    dict(nz=37, nx=300, lz=1024, lx=1024),
    dict(nz=37, nx=300, lz=768, lx=768),
    dict(nz=130, nx=45, lz=768, lx=128, vti=True),
]


@pytest.mark.parametrize("shape", SPLIT_SHAPES, ids=lambda s: f"{s['nz']}x{s['nx']}_L{s['lz']}x{s['lx']}")
def test_solution_on_the_split_stages_matches_oracle(shape):
    w = inputs.small_case(freqs=(6.0, 13.0), n_src=1, **shape)
    P = DeviceProblem(w, dbi.C64)
    u, iters, relres, code = P.solve_gmres(P.incident(), restart=30, tol=1e-6, max_iter=800, check_every=4)
    assert bool((code == dbi.CONVERGED).all()) and float(relres.max()) <= 1e-6
    orc = oracle_for(w)
    fidx, srcs = w.problem_fidx(), w.problem_src()
    for q in range(P.B):
        u0 = orc.incident(fidx[q], w.src_cells[srcs[q]], w.src_force[srcs[q]])
        assert rel(npy(u[q]), orc.solve(u0, w.model, fidx[q], tol=1e-13)) < 1e-5, q


def test_restart_matches_the_oracle_restart_count():
    """GMRES(4) in complex128: the same number of Arnoldi steps to the tolerance as the oracle's
    GMRES(4) (the iterates agree to rounding cycle by cycle), and the same solution."""
    w = inputs.small_case(nz=14, nx=11, n_src=1, freqs=(9.0,))
    P = DeviceProblem(w, dbi.C128)
    u0 = P.incident()
    u, iters, relres, code = P.solve_gmres(u0, restart=4, tol=1e-9, max_iter=400, check_every=1)
    orc = oracle_for(w)
    x, info = oracle_gmres(orc, w, 0, npy(u0[0]), restart=4, tol=1e-9, maxiter=400)
    assert int(code[0]) == dbi.CONVERGED and info["converged"]
    assert abs(int(iters[0]) - info["iters"]) <= 1
    assert rel(npy(u[0]), x) < 1e-8


def test_initial_guess_zero_rhs_and_iteration_limit():
    w = inputs.small_case(nz=12, nx=10, n_src=3, freqs=(8.0,))
    P = DeviceProblem(w, dbi.C128)
    rhs = P.incident()
    rhs[1] = 0  # problem 1: zero right-hand side
    ref, _, _, _ = P.solve_gmres(rhs, tol=1e-12, max_iter=500)
    assert not bool(ref[1].abs().max() > 0)
    # starting from the solution: converged before the first step
    u, iters, relres, code = P.solve_gmres(rhs, u0=ref, tol=1e-8, max_iter=500)
    assert bool((code == dbi.CONVERGED).all()) and int(iters.max()) == 0
    # starting from a perturbed solution: converges to the same solution
    noise = torch.as_tensor(inputs.seeded_complex(tuple(rhs.shape), 5)).to(rhs) * 1e-3 * float(ref.abs().max())
    u, iters, relres, code = P.solve_gmres(rhs, u0=ref + noise, tol=1e-12, max_iter=500)
    assert bool((code == dbi.CONVERGED).all())
    assert float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref)) < 1e-9
    # iteration limit inside a cycle
    u, iters, relres, code = P.solve_gmres(rhs, restart=30, tol=1e-14, max_iter=7)
    assert int(code[0]) == dbi.NOT_CONVERGED and int(iters[0]) == 7 and int(iters[1]) == 0
    assert int(code[1]) == dbi.CONVERGED


def test_argument_errors():
    w = inputs.small_case(nz=8, nx=8, freqs=(5.0,))
    P = DeviceProblem(w, dbi.C64)
    rhs = P.incident()
    for bad in (0, 65):
        assert dbi.gmres_workspace_bytes(P.grid, P.B, dbi.C64, bad) == 0
    lib = dbi.load()
    model = dbi._model(P.grid, P.ref, P.m, dbi.C64)
    batch = dbi._batch(P.omega, P.fidx)
    n = dbi.gmres_workspace_bytes(P.grid, P.B, dbi.C64, 10)
    work = torch.empty(n, dtype=torch.uint8, device=P.device)
    u = torch.empty_like(rhs)
    (it, rr, cd), st = dbi._status(P.B, P.device)
    opts = dbi._kopts(1e-6, 100, 4, zero_guess=True)
    rc = lib.ls_solve_gmres(ctypes.byref(model), ctypes.byref(batch), dbi._ptr(P.Ghat), dbi._ptr(rhs), dbi._ptr(u),
                            ctypes.byref(opts), 65, ctypes.byref(st), dbi.C64, dbi._ptr(work), n, dbi._stream(P.device))
    assert rc != 0 and b"restart" in lib.dbi_last_error()
    rc = lib.ls_solve_gmres(ctypes.byref(model), ctypes.byref(batch), dbi._ptr(P.Ghat), dbi._ptr(rhs), dbi._ptr(u),
                            ctypes.byref(opts), 10, ctypes.byref(st), dbi.C64, dbi._ptr(work), n - 1,
                            dbi._stream(P.device))
    assert rc != 0 and b"work buffer" in lib.dbi_last_error()
    torch.cuda.synchronize()


def test_vti_256_batch():
    """The 256^2 VTI workload (32 sources x 8 frequencies, complex64) to 1e-5 with GMRES(30):
    every problem converges; sampled problems' true residuals under the oracle's operator stay
    near the tolerance and their solutions agree with BiCGSTAB's."""
    w = inputs.config2_batched_forward()
    P = DeviceProblem(w, dbi.C64)
    u0 = P.incident()
    torch.cuda.synchronize()
    u, iters, relres, code = P.solve_gmres(u0, restart=30, tol=1e-5, max_iter=3000)
    assert bool((code == dbi.CONVERGED).all()), np.unique(npy(code), return_counts=True)
    ub, itb, _, codeb = P.solve(u0, tol=1e-5, max_iter=3000)
    assert bool((codeb == dbi.CONVERGED).all())
    print(f"\nGMRES(30) Arnoldi steps mean {float(iters.float().mean()):.1f} max {int(iters.max())}; "
          f"BiCGSTAB iterations mean {float(itb.float().mean()):.1f} (2 operator passes each)")
    orc = oracle_for(w)
    for q in (0, 100, P.B - 1):
        f = int(w.problem_fidx()[q])
        x = npy(u[q]).astype(np.complex128)
        r = np.linalg.norm(orc.apply(x, w.model, f) - npy(u0[q])) / np.linalg.norm(npy(u0[q]))
        assert r < 3e-5, (q, r)
        assert rel(npy(u[q]), npy(ub[q])) < 1e-3, q

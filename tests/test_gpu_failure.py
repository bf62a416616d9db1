"""Failure detection on the GPU without a GPU fault: NaN injected on the host into one problem's
right-hand side, into the model, or into the data residual of the adjoint stops the affected
problems with DBI_NONFINITE within one iteration (the others converge as before), for BiCGSTAB and
GMRES in both precisions and on the complex64 stages of FFT lengths 1024 and 768; nothing hangs
and the context stays usable (a clean solve follows)."""
import numpy as np
import pytest
import torch

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


# (precision, FFT grid): the default grid, and in complex64 the stages of FFT lengths 1024 (pairs of
# 512-point transforms) and 768 (triples of 256-point transforms) with their contrast-source kernel
@pytest.fixture(params=[(dbi.C64, None), (dbi.C128, None), (dbi.C64, 1024), (dbi.C64, 768)],
                ids=["c64", "c128", "c64_L1024", "c64_L768"])
def problem(request):
    precision, L = request.param
    grid = {} if L is None else dict(lz=L, lx=L)
    w = inputs.small_case(nz=20, nx=16, n_src=2, freqs=(7.0, 11.0), vti=True, amp=0.12, seed=8, **grid)
    return DeviceProblem(w, precision)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_nan_in_one_right_hand_side(problem, solver):
    P = problem
    u0 = P.incident()
    bad = u0.clone()
    bad[1, 0, 3, 4] = float("nan")
    solve = P.solve if solver == "bicgstab" else P.solve_gmres
    u, iters, relres, code = solve(bad, tol=1e-6, max_iter=300)
    code, iters = npy(code), npy(iters)
    assert code[1] == dbi.NONFINITE and iters[1] == 0, (code, iters)
    others = [b for b in range(P.B) if b != 1]
    assert np.all(code[others] == dbi.CONVERGED), code
    # the context is still usable: the clean system converges for every problem
    _, _, _, code2 = solve(u0, tol=1e-6, max_iter=300)
    assert np.all(npy(code2) == dbi.CONVERGED)


@pytest.mark.parametrize("solver", ["bicgstab", "gmres"])
def test_nan_in_the_model(problem, solver):
    P = problem
    m = P.m.clone()
    m[2, 7, 5] = float("nan")
    solve = P.solve if solver == "bicgstab" else P.solve_gmres
    _, iters, _, code = solve(P.incident(), m=m, tol=1e-6, max_iter=300)
    assert np.all(npy(code) == dbi.NONFINITE), npy(code)
    assert np.all(npy(iters) <= 1), npy(iters)


def test_nan_in_the_adjoint_residual(problem):
    P = problem
    u, _, _, code = P.forward(tol=1e-8 if P.precision == dbi.C128 else 1e-6)
    assert np.all(npy(code) == dbi.CONVERGED)
    r = P.to_field(inputs.seeded_complex((P.B, P.rec_cells.shape[0], 2), 3) * 1e-10)
    r[2, 1, 0] = float("inf")
    _, (iters, _, code) = dbi.adjoint_apply(P.grid, P.ref, P.m, P.omega, P.fidx, P.Ghat, u, P.rec_cells, r,
                                            tol=1e-6, max_iter=300, with_status=True)
    code = npy(code)
    assert code[2] == dbi.NONFINITE and npy(iters)[2] == 0, code
    assert np.all(code[[0, 1, 3]] == dbi.CONVERGED), code

"""Pins of the oracle's restarted GMRES (CPU only), by properties that do not retype its steps:
the minimal-residual property against a brute-force least-squares problem over an explicitly
built Krylov matrix, exact convergence in n steps on an n x n system, monotone residuals,
one-step convergence on an invariant subspace, and agreement with the oracle's BiCGSTAB on the
LS operator, with and without restarts."""
import numpy as np
import pytest

import oracle as O


def system(n=12, seed=3, shift=4.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + shift * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_exact_in_n_steps():
    A, b = system()
    x, info = O.gmres(lambda v: A @ v, b, restart=12, tol=1e-13, maxiter=12)
    assert info["iters"] <= 12 and info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(x)


@pytest.mark.parametrize("k", [1, 3, 6])
@pytest.mark.parametrize("with_x0", [False, True])
def test_one_cycle_minimises_the_residual_over_the_krylov_space(k, with_x0):
    """After k steps of one cycle, x = x0 + z with z minimising ||r0 - A z|| over
    span(r0, A r0, ..., A^(k-1) r0): solved here by least squares on that explicit basis."""
    A, b = system(n=10, seed=7)
    rng = np.random.default_rng(11)
    x0 = rng.standard_normal(10) + 1j * rng.standard_normal(10) if with_x0 else np.zeros(10, complex)
    x, info = O.gmres(lambda v: A @ v, b, restart=k, tol=0.0, maxiter=k, x0=x0)
    r0 = b - A @ x0
    K = np.stack([np.linalg.matrix_power(A, i) @ r0 for i in range(k)], axis=1)
    c, *_ = np.linalg.lstsq(A @ K, r0, rcond=None)
    x_bf = x0 + K @ c
    assert np.linalg.norm(x - x_bf) <= 1e-9 * np.linalg.norm(x_bf)
    # the last step's minimal residual is the true residual of the returned iterate
    assert info["resvec"][-1] == pytest.approx(np.linalg.norm(b - A @ x) / np.linalg.norm(b), rel=1e-9)


def test_residuals_do_not_increase_and_restarts_converge():
    A, b = system(n=40, seed=5, shift=15.0)
    x, info = O.gmres(lambda v: A @ v, b, restart=5, tol=1e-12, maxiter=400)
    rv = np.asarray(info["resvec"])
    assert info["converged"] and len(rv) > 10  # several cycles
    assert np.all(rv[1:] <= rv[:-1] * (1 + 1e-10))
    assert info["relres"] <= 1e-11


def test_invariant_subspace_stops_after_one_step():
    """b an eigenvector of A: A v_1 lies in span(v_1), the new basis vector vanishes and the
    solution b / lambda comes out of the first step."""
    d = np.array([2.0, 3.0 + 1j, 5.0, -1.5j])
    b = np.array([0, 1.0 - 2j, 0, 0])
    x, info = O.gmres(lambda v: d * v, b, restart=4, tol=1e-14, maxiter=4)
    assert info["iters"] == 1
    assert np.allclose(x, b / d[1], rtol=1e-14, atol=0)


def test_zero_right_hand_side():
    x, info = O.gmres(lambda v: 2 * v, np.zeros(5, complex))
    assert info["converged"] and info["iters"] == 0 and not np.any(x)


def test_planted_conjugation_error_is_caught():
    """A Givens rotation that forgets the conjugate still reduces a real problem but not a
    complex one: the minimal-residual pin above must fail for it."""
    A, b = system(n=10, seed=7)
    good = O.givens

    def bad(a, bb):
        c, s, r = good(a, bb)
        return c, np.conj(s), r

    O_g = O.dbi_oracle
    O_g.givens = bad
    try:
        x, _ = O.gmres(lambda v: A @ v, b, restart=4, tol=0.0, maxiter=4)
    finally:
        O_g.givens = good
    K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(4)], axis=1)
    c, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
    assert np.linalg.norm(x - K @ c) > 1e-6 * np.linalg.norm(K @ c)


@pytest.mark.parametrize("restart", [30, 4])
def test_ls_operator_gmres_equals_bicgstab(restart):
    nz, nx = 9, 8
    rng = np.random.default_rng(2)
    orc = O.LSOracle(nz, nx, 10.0, 2 * nz, 2 * nx, 2000.0, 2000.0, 1155.0, [2 * np.pi * 11.0])
    ref = O.reference_params(2000.0, 2000.0, 1155.0)
    model = ref[:, None, None] * (1.0 + 0.15 * (2.0 * rng.random((5, nz, nx)) - 1.0))
    u0 = orc.incident(0, (0, 3), (0.3, 1.0))
    ub = orc.solve(u0, model, 0, tol=1e-13)
    ug, info = orc.solve_gmres(u0, model, 0, restart=restart, tol=1e-13)
    assert info["converged"] and info["relres"] <= 1e-12
    assert np.linalg.norm(ug - ub) <= 1e-10 * np.linalg.norm(ub)

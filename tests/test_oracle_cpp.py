"""The C++17 FP64 oracle (oracle/cpp/dbi_oracle.cpp: own radix-2 FFT, C++17 Bessel functions,
OpenMP over problems) against the numpy oracle, whose pins tie it to the paper and to physics
(tests/test_oracle_pins.py): the Green's lattice, the operator by the FFT and by the direct sum,
and the misfit gradient of a batch agree to rounding. CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import cpp_oracle as C
from paper_2402_02116_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("nz,nx,f", [(5, 7, 9.0), (9, 15, 25.0), (16, 3, 3.0)])
def test_green_lattice_matches_numpy_oracle(nz, nx, f):
    w = 2 * math.pi * f
    a = C.green_lattice(nz, nx, 10.0, w, 2000.0, 1155.0, 2000.0)
    b = O.green_lattice(nz, nx, 10.0, w, 2000.0, 1155.0, 2000.0)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


CASES = [dict(nz=12, nx=10), dict(nz=5, nx=9, lz=16, lx=32), dict(nz=1, nx=8), dict(nz=20, nx=14, vti=True)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['nz']}x{c['nx']}")
def test_operator_matches_numpy_oracle_and_direct_sum(case):
    w = inputs.small_case(freqs=(6.0, 13.0), **case)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx = w.problem_fidx()
    u = inputs.seeded_complex((len(fidx), 2, w.nz, w.nx), 3)
    co = C.for_workload(w)
    got = co.apply(fidx, u)
    direct = co.apply(fidx, u, direct=True)
    for b, f in enumerate(fidx):
        want = orc.apply(u[b], w.model, f)
        assert rel(got[b] - u[b], want - u[b]) < 1e-12, b
        assert rel(direct[b] - u[b], got[b] - u[b]) < 1e-12, b


def test_gradient_matches_numpy_oracle():
    """Forward solves, residuals at the receivers, adjoint solves and imaging of a 4-problem batch
    (two sources, two frequencies) to 1e-13: gradient, residuals and wavefields agree to 1e-9."""
    w = inputs.small_case(nz=14, nx=12, amp=0.1, vti=True, n_src=2, freqs=(7.0, 12.0), seed=51)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx = w.problem_fidx()
    srcs, forces = w.src_cells[w.problem_src()], w.src_force[w.problem_src()]
    d_obs = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 6) * 1e-10
    phi, g_o, U = orc.misfit(w.model, fidx, srcs, forces, d_obs, w.rec_cells, tol=1e-13)
    g, r, passes, relres, u = C.for_workload(w).gradient(fidx, srcs, forces, w.rec_cells, d_obs, tol=1e-13,
                                                         keep_fields=True)
    assert np.all(relres < 1e-12) and np.all(passes > 2)
    assert rel(u, U) < 1e-9
    R = np.stack([orc.sample(U[b], w.rec_cells) for b in range(len(fidx))]) - d_obs
    assert rel(r, R) < 1e-9
    for p in range(5):
        assert rel(g[p], g_o[p]) < 1e-9, p


def test_threads_do_not_change_the_result():
    """OpenMP over problems: one thread and every thread give the same bits."""
    w = inputs.small_case(nz=10, nx=9, n_src=3, freqs=(6.0, 11.0), vti=True, seed=4)
    fidx = w.problem_fidx()
    srcs, forces = w.src_cells[w.problem_src()], w.src_force[w.problem_src()]
    d_obs = inputs.seeded_complex((len(fidx), len(w.rec_cells), 2), 2) * 1e-10
    co = C.for_workload(w)
    g1 = co.gradient(fidx, srcs, forces, w.rec_cells, d_obs, tol=1e-10, threads=1)[0]
    gn = co.gradient(fidx, srcs, forces, w.rec_cells, d_obs, tol=1e-10, threads=0)[0]
    assert np.array_equal(g1, gn)

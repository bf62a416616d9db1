"""Accuracy of the complex64 path at the benchmark sizes, against the FP64 oracle.

On the 512 x 512 VTI gradient workload (1024 x 1024 FFT grid, frequencies 3-18 Hz) sampled
wavefields, receiver data and residuals of the batched complex64 solve (BiCGSTAB to 1e-6, the
benchmark's tolerance) are within 1e-5 of the oracle's solution to 1e-12, and the gradient of a
sub-batch (adjoint solve and imaging) within 1e-4 per parameter; on the 256 x 256 workload the same
for sampled wavefields. The oracle's problems run in spawned processes, one core each."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.problem import DeviceProblem

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GPU_TOL = 1e-6      # BiCGSTAB relative residual of the benchmark's solves
ORACLE_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _workload(name, n_src):
    if name == "vti512":
        return inputs.config4_misfit(n_src=n_src)
    return inputs.config2_batched_forward()


def _observed(w):
    return (inputs.seeded_complex((w.n_problems, len(w.rec_cells), 2), 17) * 1e-10).astype(np.complex64)


def _oracle_problem(task):
    """FP64 oracle: problem b's wavefield and data to ORACLE_TOL and, if asked, its gradient
    contribution against the observed data (inputs rounded as the GPU reads them)."""
    name, n_src, b, with_gradient = task
    w = _workload(name, n_src)
    f, s = int(w.problem_fidx()[b]), int(w.problem_src()[b])
    model = np.asarray(w.model, dtype=np.float32).astype(np.float64)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas[f:f + 1])
    u, info = orc.solve_info(orc.incident(0, w.src_cells[s], w.src_force[s]), model, 0, tol=ORACLE_TOL)
    assert info["converged"]
    d = orc.sample(u, w.rec_cells)
    out = {"u": u, "d": d}
    if with_gradient:
        r = d - _observed(w)[b].astype(np.complex128)
        ua, info = orc.solve_info(orc.convolve(orc.inject(np.conj(r), w.rec_cells), 0), model, 0, tol=ORACLE_TOL)
        assert info["converged"]
        out["r"] = r
        out["g"] = orc.imaging(ua, u, orc.omegas[0], orc.h)
    return out


def _oracle_parallel(tasks):
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    with cf.ProcessPoolExecutor(max_workers=len(tasks), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_problem, tasks))


def test_config4_sampled_wavefields_data_and_gradient():
    """512 x 512 VTI workload with 4 sources x 6 frequencies (24 problems, the full grid and
    frequencies): the problems at 3 Hz (first source) and 18 Hz (third source) of the batched
    solve against the oracle at 1e-5 (wavefield, receiver data, data residual), and the gradient
    of that two-problem sub-batch (adjoint_apply at the benchmark's tolerance) at 1e-4 for every
    parameter."""
    w = _workload("vti512", 4)
    P = DeviceProblem(w, dbi.C64)
    sampled = [0, (w.nf - 1) * w.n_src + 2]
    futs = _oracle_parallel([("vti512", 4, b, True) for b in sampled])
    u0 = P.incident()
    u, iters, relres, code = P.solve(u0, tol=GPU_TOL, max_iter=3000)
    assert bool((code == dbi.CONVERGED).all())
    d_obs = P.to_field(_observed(w))
    r, _ = dbi.data_residual(P.grid, P.omega, P.fidx, P.rec_cells, u, d_obs)
    idx = torch.tensor(sampled, device=P.device)
    us, rs = u.index_select(0, idx).contiguous(), r.index_select(0, idx).contiguous()
    g = dbi.adjoint_apply(P.grid, P.ref, P.m, P.omega, P.fidx.index_select(0, idx).contiguous(), P.Ghat, us,
                          P.rec_cells, rs, tol=GPU_TOL, max_iter=3000)
    us, rs = us.cpu().numpy().astype(np.complex128), rs.cpu().numpy().astype(np.complex128)
    g = g.cpu().numpy().astype(np.float64)
    obs = _observed(w).astype(np.complex128)
    g_or = np.zeros_like(g)
    for k, (b, want) in enumerate(zip(sampled, futs)):
        assert rel(us[k], want["u"]) < 1e-5, (b, rel(us[k], want["u"]))
        assert rel(rs[k] + obs[b], want["d"]) < 1e-5, (b, rel(rs[k] + obs[b], want["d"]))
        assert rel(rs[k], want["r"]) < 1e-5, (b, rel(rs[k], want["r"]))
        g_or += want["g"]
    for p in range(5):
        assert rel(g[p], g_or[p]) < 1e-4, (inputs.PARAMS[p], rel(g[p], g_or[p]))


def test_config2_sampled_wavefields():
    """256 x 256 VTI workload, all 256 problems in one batched complex64 solve to 1e-6: the
    wavefields and receiver data of the first and last problems (5 and 20 Hz) are within 1e-5 of
    the oracle's solution to 1e-12."""
    w = _workload("vti256", 32)
    P = DeviceProblem(w, dbi.C64)
    sampled = [0, w.n_problems - 1]
    futs = _oracle_parallel([("vti256", 32, b, False) for b in sampled])
    u, iters, relres, code = P.solve(P.incident(), tol=GPU_TOL, max_iter=3000)
    assert bool((code == dbi.CONVERGED).all())
    d = P.sample(u).cpu().numpy().astype(np.complex128)
    un = u.cpu().numpy()
    for b, want in zip(sampled, futs):
        assert rel(un[b].astype(np.complex128), want["u"]) < 1e-5, (b, rel(un[b], want["u"]))
        assert rel(d[b], want["d"]) < 1e-5, b

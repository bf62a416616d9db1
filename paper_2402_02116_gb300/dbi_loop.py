"""The distorted-Born iterative (DBI) inversion loop with sequential frequencies.

For each frequency, from the lowest to the highest (the paper's sequential-frequency scheme), the
loop repeats: background wavefields u_b = A_b^-1 u0 in the current model (Eq. 11); synthetic data
and the normalised data error eps_d = ||d_cal - d_obs|| / ||d_obs||; the Tikhonov normal equation
(Re J^H J + lambda I) dm = Re J^H (d_obs - d_cal) (Eq. 23, 24) solved by matrix-free CG; the
update m_b <- m_b + dm (the DBI step of the section on the distorted Born iterative method). A
frequency stops when eps_d < eps_d_stop or after max_iter updates (the experiments' criteria:
1e-3 and 10). The regularisation weight starts at lambda_rel times the power-iteration estimate of
lambda_max and is multiplied by `cooling` after every update (the paper reduces it progressively
without giving constants). With a true model, the normalised model error eps_m = ||m - m_true|| /
||m_true|| is recorded too.

Every operator, solve, Fréchet and adjoint product runs in the CUDA library through
`DeviceProblem`; this module only orchestrates the calls and reads back scalars.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass, field

import numpy as np
import torch

from . import dbi
from .problem import DeviceProblem


@dataclass
class DBIRecord:
    freq_hz: float
    iteration: int              # updates done at this frequency before the record
    eps_d: float
    eps_m: float | None
    lam: float | None = None    # lambda of the update that follows (None when the frequency stops)
    solve_iters_max: int = 0


@dataclass
class DBIResult:
    m: torch.Tensor
    history: list = field(default_factory=list)


def single_frequency(w, f_index: int):
    """A copy of workload w with only its frequency f_index (all sources)."""
    s = copy.copy(w)
    s.freqs_hz = np.asarray([w.freqs_hz[f_index]], dtype=np.float64)
    return s


def normalized(a: torch.Tensor, b: torch.Tensor) -> float:
    """||a - b|| / ||b|| in FP64."""
    a64, b64 = a.to(torch.complex128 if a.is_complex() else torch.float64), b.to(
        torch.complex128 if b.is_complex() else torch.float64)
    return float(torch.linalg.norm((a64 - b64).reshape(-1)) / torch.linalg.norm(b64.reshape(-1)))


def observed_data(w, m_true, precision=dbi.C64, tol=None):
    """Synthetic observed data per frequency: [nf] list of [n_src][n_rec][2] complex tensors."""
    out = []
    for fi in range(len(w.freqs_hz)):
        P = DeviceProblem(single_frequency(w, fi), precision, model=m_true, with_space=True)
        u, _, _, code = P.forward(tol=tol)
        if not bool((code == dbi.CONVERGED).all()):
            raise RuntimeError("forward solve for the observed data did not converge")
        out.append(P.sample(u))
    return out


def dbi_inversion(w, d_obs, m0, precision=dbi.C64, max_iter=10, eps_d_stop=1e-3, cg_iters=30,
                  lambda_rel=1e-3, cooling=0.5, m_true=None, tol=None, power_iters=10, power_seed=17,
                  problem=DeviceProblem, device="cuda"):
    """Run the DBI loop from model m0 ([5][nz][nx], absolute values) against d_obs (from
    observed_data); returns the final model and one DBIRecord per data-error evaluation.
    `problem` builds the per-frequency problem (the library's DeviceProblem; the CPU tests of the
    loop's control logic pass a stand-in with the same methods) on `device`."""
    rdt = dbi.real_dtype(precision)
    m = torch.as_tensor(np.asarray(m0, dtype=np.float64)).to(device, rdt).contiguous()
    mt = None if m_true is None else torch.as_tensor(np.asarray(m_true, dtype=np.float64)).to(device, torch.float64)
    rng = np.random.default_rng(power_seed)
    power_start = rng.standard_normal((5, w.nz, w.nx))
    res = DBIResult(m=m)
    order = np.argsort(np.asarray(w.freqs_hz))
    for fi in order:
        P = problem(single_frequency(w, int(fi)), precision, model=m.double().cpu().numpy())
        d = d_obs[int(fi)].to(P.device, P.cdt)
        lam = None
        for k in range(max_iter + 1):
            u_b, iters, _, code = P.solve(P.incident(), m=m, tol=tol)
            if not bool((code == dbi.CONVERGED).all()):
                raise RuntimeError(f"background solve did not converge at {w.freqs_hz[fi]} Hz")
            d_cal = P.sample(u_b)
            eps_d = normalized(d_cal, d)
            eps_m = None if mt is None else normalized(m.double(), mt)
            rec = DBIRecord(float(w.freqs_hz[fi]), k, eps_d, eps_m, solve_iters_max=int(iters.max()))
            res.history.append(rec)
            if eps_d < eps_d_stop or k == max_iter:
                break
            dm, lam_used, _ = P.normal_cg(u_b, (d - d_cal).contiguous(), iters=cg_iters, lam=lam,
                                          lambda_rel=lambda_rel, power_iters=power_iters,
                                          power_start=power_start, m_b=m, tol=tol)
            rec.lam = lam_used
            lam = lam_used * cooling
            m = (m + dm).contiguous()
        res.m = m
    return res


# ---------------------------------------------------------------------------------------------
# 3D (the paper's 3D VTI example): the same loop over the 3D entry points
# ---------------------------------------------------------------------------------------------
def observed_data_3d(w, m_true, precision=dbi.C64, tol=None):
    """Synthetic observed data per frequency of a 3D workload: [nf] list of [n_src][n_rec][3]."""
    from .problem import DeviceProblem3D
    out = []
    for fi in range(len(w.freqs_hz)):
        P = DeviceProblem3D(single_frequency(w, fi), precision, model=m_true)
        u, _, _, code = P.solve(P.incident(), tol=tol)
        if not bool((code == dbi.CONVERGED).all()):
            raise RuntimeError("3D forward solve for the observed data did not converge")
        out.append(P.sample(u))
    return out


def dbi_inversion_3d(w, d_obs, m0, precision=dbi.C64, max_iter=10, eps_d_stop=1e-3, cg_iters=30,
                     lambda_rel=1e-3, cooling=0.5, m_true=None, tol=None, power_iters=10, power_seed=17,
                     problem=None, device="cuda"):
    """The DBI loop of dbi_inversion for a 3D workload (models [6][nz][ny][nx]): background GMRES
    solves, sampled data, the 3D normal equation, model updates, per frequency from the lowest.
    `problem` defaults to the library's DeviceProblem3D."""
    if problem is None:
        from .problem import DeviceProblem3D as problem
    rdt = dbi.real_dtype(precision)
    m = torch.as_tensor(np.asarray(m0, dtype=np.float64)).to(device, rdt).contiguous()
    mt = None if m_true is None else torch.as_tensor(np.asarray(m_true, dtype=np.float64)).to(device, torch.float64)
    rng = np.random.default_rng(power_seed)
    power_start = rng.standard_normal((6, w.nz, w.ny, w.nx))
    res = DBIResult(m=m)
    for fi in np.argsort(np.asarray(w.freqs_hz)):
        P = problem(single_frequency(w, int(fi)), precision, model=m.double().cpu().numpy())
        d = d_obs[int(fi)].to(P.device, P.cdt)
        ps = P.to_model(power_start)
        lam = None
        for k in range(max_iter + 1):
            u_b, iters, relres, code = P.solve(P.incident(), m=m, tol=tol)
            if not bool((code == dbi.CONVERGED).all()):
                raise RuntimeError(f"3D background solve did not converge at {w.freqs_hz[fi]} Hz, update {k}: "
                                   f"codes {code.tolist()}, steps {iters.tolist()}, residuals {relres.tolist()}")
            d_cal = P.sample(u_b)
            eps_d = normalized(d_cal, d)
            eps_m = None if mt is None else normalized(m.double(), mt)
            rec = DBIRecord(float(w.freqs_hz[fi]), k, eps_d, eps_m, solve_iters_max=int(iters.max()))
            res.history.append(rec)
            if eps_d < eps_d_stop or k == max_iter:
                break
            dm, lam_used, _ = P.normal_cg(u_b, (d - d_cal).contiguous(), iters=cg_iters, lam=lam,
                                          lambda_rel=lambda_rel, power_iters=power_iters, power_start=ps, m_b=m,
                                          tol=tol)
            rec.lam = lam_used
            lam = lam_used * cooling
            m = (m + dm).contiguous()
        res.m = m
    return res

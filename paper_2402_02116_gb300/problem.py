"""A workload held on one CUDA device, with the library's entry points bound to it.

`DeviceProblem` copies a workload description (grid, reference medium, model, frequencies,
sources, receivers) to the device once and forwards calls to the C ABI binding in `dbi.py`.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dbi


def next_pow2(n: int) -> int:
    p = 16
    while p < n:
        p *= 2
    return p


class DeviceProblem:
    def __init__(self, w, precision: int = dbi.C64, device="cuda", model=None, with_space=True):
        self.w = w
        self.precision = precision
        self.device = torch.device(device)
        self.rdt = dbi.real_dtype(precision)
        self.cdt = dbi.complex_dtype(precision)
        self.grid = dbi.make_grid(w.nz, w.nx, w.lz, w.lx, w.h)
        self.ref = (dbi.make_medium_vti(*w.ref_vti) if getattr(w, "ref_vti", None) is not None
                    else dbi.make_medium(w.rho0, w.alpha0, w.beta0))
        dev = self.device
        self.omega = torch.tensor(np.asarray(w.omegas, dtype=np.float64), device=dev)
        self.fidx = torch.tensor(w.problem_fidx(), dtype=torch.int32, device=dev)
        srcs = w.problem_src()
        self.src_cells = torch.tensor(np.asarray(w.src_cells)[srcs], dtype=torch.int32, device=dev).contiguous()
        self.forces = torch.tensor(np.asarray(w.src_force, dtype=np.float64)[srcs], device=dev).contiguous()
        self.rec_cells = torch.tensor(np.asarray(w.rec_cells), dtype=torch.int32, device=dev).contiguous()
        self.m = self.to_model(w.model if model is None else model)
        self.Ghat, self.Gspace = dbi.greens_tabulate(self.grid, self.ref, self.omega, precision, with_space)

    @property
    def B(self) -> int:
        return int(self.fidx.numel())

    def to_model(self, arr) -> torch.Tensor:
        return torch.as_tensor(np.asarray(arr, dtype=np.float64)).to(self.device, self.rdt).contiguous()

    def to_field(self, arr) -> torch.Tensor:
        return torch.as_tensor(np.asarray(arr)).to(self.device, self.cdt).contiguous()

    # --- entry points --------------------------------------------------------------------------
    def incident(self):
        return dbi.incident_field(self.grid, self.omega, self.fidx, self.Gspace, self.src_cells, self.forces)

    def convolve(self, src):
        return dbi.green_convolve(self.grid, self.omega, self.fidx, self.Ghat, src)

    def apply(self, u, m=None):
        return dbi.ls_apply(self.grid, self.ref, self.m if m is None else m, self.omega, self.fidx, self.Ghat, u)

    def solve(self, rhs, m=None, tol=None, max_iter=2000, check_every=8, u0=None):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.ls_solve(self.grid, self.ref, self.m if m is None else m, self.omega, self.fidx, self.Ghat,
                            rhs, u0=u0, tol=tol, max_iter=max_iter, check_every=check_every)

    def forward(self, m=None, tol=None, max_iter=2000):
        u, iters, relres, code = self.solve(self.incident(), m=m, tol=tol, max_iter=max_iter)
        return u, iters, relres, code

    def solve_gmres(self, rhs, m=None, restart=30, tol=None, max_iter=2000, check_every=8, u0=None):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.ls_solve_gmres(self.grid, self.ref, self.m if m is None else m, self.omega, self.fidx, self.Ghat,
                                  rhs, u0=u0, restart=restart, tol=tol, max_iter=max_iter, check_every=check_every)

    # paper-literal form of Eq. 9 (derivative tables tabulated on first use)
    @property
    def Dhat(self):
        if getattr(self, "_Dhat", None) is None:
            self._Dhat = dbi.greens_tabulate_k(self.grid, self.ref, self.omega, self.precision)
        return self._Dhat

    def apply_k(self, u, m=None):
        return dbi.ls_apply_k(self.grid, self.ref, self.m if m is None else m, self.omega, self.fidx, self.Ghat,
                              self.Dhat, u)

    def solve_k(self, rhs, m=None, tol=None, max_iter=2000, check_every=8, u0=None):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.ls_solve_k(self.grid, self.ref, self.m if m is None else m, self.omega, self.fidx, self.Ghat,
                              self.Dhat, rhs, u0=u0, tol=tol, max_iter=max_iter, check_every=check_every)

    def sample(self, u):
        d, _ = dbi.data_residual(self.grid, self.omega, self.fidx, self.rec_cells, u,
                                 torch.zeros((self.B, self.rec_cells.shape[0], 2), dtype=self.cdt, device=self.device))
        return d

    def frechet(self, u_b, dm, m_b=None, tol=None, max_iter=2000):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.frechet_apply(self.grid, self.ref, self.m if m_b is None else m_b, self.omega, self.fidx,
                                 self.Ghat, u_b, self.rec_cells, dm, tol=tol, max_iter=max_iter)

    def adjoint(self, u_b, r, m_b=None, tol=None, max_iter=2000):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.adjoint_apply(self.grid, self.ref, self.m if m_b is None else m_b, self.omega, self.fidx,
                                 self.Ghat, u_b, self.rec_cells, r, tol=tol, max_iter=max_iter)

    def residual(self, u, d_obs):
        return dbi.data_residual(self.grid, self.omega, self.fidx, self.rec_cells, u, d_obs)

    def normal_cg(self, u_b, dd, iters=30, lam=None, lambda_rel=1e-3, power_iters=10, power_start=None,
                  m_b=None, tol=None, max_iter=2000):
        tol = self.w.krylov_tol if tol is None else tol
        ps = None if power_start is None else self.to_model(power_start)
        return dbi.normal_cg(self.grid, self.ref, self.m if m_b is None else m_b, self.omega, self.fidx,
                             self.Ghat, u_b, self.rec_cells, dd, iters=iters, lam=lam, lambda_rel=lambda_rel,
                             power_iters=power_iters, power_start=ps, tol=tol, max_iter=max_iter)


class DeviceProblem3D:
    """A 3D workload (inputs.Workload3D) copied to the device once; forwards to the 3D entry points."""

    def __init__(self, w, precision: int = dbi.C64, device="cuda", model=None, with_space=True):
        self.w = w
        self.precision = precision
        self.device = torch.device(device)
        self.rdt = dbi.real_dtype(precision)
        self.cdt = dbi.complex_dtype(precision)
        self.grid = dbi.make_grid3(w.nz, w.ny, w.nx, w.lz, w.ly, w.lx, w.h)
        self.ref = dbi.make_medium(w.rho0, w.alpha0, w.beta0)
        dev = self.device
        self.omega = torch.tensor(np.asarray(w.omegas, dtype=np.float64), device=dev)
        self.fidx = torch.tensor(w.problem_fidx(), dtype=torch.int32, device=dev)
        srcs = w.problem_src()
        self.src_cells = torch.tensor(np.asarray(w.src_cells)[srcs], dtype=torch.int32, device=dev).contiguous()
        self.forces = torch.tensor(np.asarray(w.src_force, dtype=np.float64)[srcs], device=dev).contiguous()
        self.m = torch.as_tensor(np.asarray(w.model if model is None else model, dtype=np.float64)).to(
            dev, self.rdt).contiguous()
        self.rec_cells = torch.tensor(np.asarray(w.rec_cells), dtype=torch.int32, device=dev).contiguous()
        self.Ghat, self.Gspace = dbi.greens_tabulate_3d(self.grid, self.ref, self.omega, precision, with_space)

    @property
    def B(self) -> int:
        return int(self.fidx.numel())

    def to_field(self, arr) -> torch.Tensor:
        return torch.as_tensor(np.asarray(arr)).to(self.device, self.cdt).contiguous()

    def incident(self):
        return dbi.incident_field_3d(self.grid, self.omega, self.fidx, self.Gspace, self.src_cells, self.forces)

    def apply(self, u):
        return dbi.ls_apply_3d(self.grid, self.ref, self.m, self.omega, self.fidx, self.Ghat, u)

    def to_model(self, arr) -> torch.Tensor:
        return torch.as_tensor(np.asarray(arr, dtype=np.float64)).to(self.device, self.rdt).contiguous()

    def sample(self, u):
        return dbi.sample_3d(self.grid, self.rec_cells, u)

    def frechet(self, u_b, dm, m_b=None, tol=None, max_iter=2000, restart=30):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.frechet_apply_3d(self.grid, self.ref, self.m if m_b is None else m_b, self.omega, self.fidx,
                                    self.Ghat, u_b, self.rec_cells, dm, tol=tol, max_iter=max_iter, restart=restart)

    def adjoint(self, u_b, r, m_b=None, tol=None, max_iter=2000, restart=30):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.adjoint_apply_3d(self.grid, self.ref, self.m if m_b is None else m_b, self.omega, self.fidx,
                                    self.Ghat, u_b, self.rec_cells, r, tol=tol, max_iter=max_iter, restart=restart)

    def normal_cg(self, u_b, dd, iters=30, lam=None, lambda_rel=1e-3, power_iters=10, power_start=None, m_b=None,
                  tol=None, max_iter=2000, restart=30):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.normal_cg_3d(self.grid, self.ref, self.m if m_b is None else m_b, self.omega, self.fidx,
                                self.Ghat, u_b, self.rec_cells, dd, iters=iters, lam=lam, lambda_rel=lambda_rel,
                                power_iters=power_iters, power_start=power_start, tol=tol, max_iter=max_iter,
                                restart=restart)

    def solve(self, rhs, m=None, restart=30, tol=None, max_iter=2000, check_every=8, u0=None):
        tol = self.w.krylov_tol if tol is None else tol
        return dbi.ls_solve_3d(self.grid, self.ref, self.m if m is None else m, self.omega, self.fidx, self.Ghat,
                               rhs, u0=u0,
                               restart=restart, tol=tol, max_iter=max_iter, check_every=check_every)

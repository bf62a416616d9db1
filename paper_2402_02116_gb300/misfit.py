"""Differentiable L2 data misfit of the elastic LS forward problem (a torch.autograd.Function).

    phi(m) = 1/2 sum_{s,f} || P u_{s,f}(m) - d_obs[s,f] ||^2,   A(m) u_{s,f} = u0_{s,f}   (Eq. 11, 23)

forward: incident fields, batched BiCGSTAB solves and the data residual, all in the CUDA library.
backward: the adjoint-state gradient Re J^H r (Eq. 25, 32-35) by `adjoint_apply`, i.e. one more
batched solve with conj(r) injected at the receivers and the imaging condition; the result is
d phi / d m for m = (rho, C11, C13, C33, C55) per cell.

Memory: the forward wavefields are kept for the backward pass when the whole batch fits in
`memory_budget` bytes; otherwise the batch is processed in chunks of problems that fit, only the
receiver residuals are kept, and each chunk's wavefields are recomputed in the backward pass.
"""
from __future__ import annotations

import math

import torch

from . import dbi


class MisfitProblem:
    """Device-resident description of the misfit: grid, reference medium, frequencies, sources,
    receivers, observed data and solver settings. `P` is a DeviceProblem."""

    def __init__(self, P, d_obs: torch.Tensor, tol: float = 1e-6, max_iter: int = 3000,
                 memory_budget: int | None = None):
        self.P = P
        self.d_obs = d_obs.to(P.device, P.cdt).contiguous()
        self.tol = float(tol)
        self.max_iter = int(max_iter)
        per_problem = 2 * P.grid.nz * P.grid.nx * torch.empty((), dtype=P.cdt).element_size()
        # each chunk holds its wavefields plus the solver's work (about 8 fields per problem)
        if memory_budget is None:
            self.chunk = P.B
        else:
            self.chunk = max(1, min(P.B, int(memory_budget // (9 * per_problem))))
        self.keep_fields = self.chunk >= P.B
        self.last_stats = {}

    def chunks(self):
        for b0 in range(0, self.P.B, self.chunk):
            yield b0, min(self.P.B, b0 + self.chunk)

    def forward_chunk(self, m, b0, b1):
        P = self.P
        fidx = P.fidx[b0:b1].contiguous()
        u0 = dbi.incident_field(P.grid, P.omega, fidx, P.Gspace, P.src_cells[b0:b1].contiguous(),
                                P.forces[b0:b1].contiguous())
        u, iters, relres, code = dbi.ls_solve(P.grid, P.ref, m, P.omega, fidx, P.Ghat, u0, tol=self.tol,
                                              max_iter=self.max_iter)
        return u, fidx, iters, code


class ElasticMisfit(torch.autograd.Function):
    """phi = ElasticMisfit.apply(m, problem): m is [5][nz][nx] (float32 for the complex64 path,
    float64 for complex128) on the problem's device; phi is a float64 scalar tensor."""

    @staticmethod
    def forward(ctx, m, problem: MisfitProblem):
        m = m.contiguous()
        P = problem.P
        phis, residuals, fields = [], [], []
        iters = []
        for b0, b1 in problem.chunks():
            u, fidx, it, code = problem.forward_chunk(m, b0, b1)
            r, phi = dbi.data_residual(P.grid, P.omega, fidx, P.rec_cells, u, problem.d_obs[b0:b1].contiguous())
            phis.append(phi)
            residuals.append(r)
            iters.append(it)
            if problem.keep_fields:
                fields.append(u)
        ctx.problem = problem
        ctx.residuals = residuals
        ctx.fields = fields if problem.keep_fields else None
        ctx.save_for_backward(m)
        problem.last_stats["forward_iters"] = torch.cat(iters)
        return torch.stack(phis).sum()

    @staticmethod
    def backward(ctx, grad_phi):
        (m,) = ctx.saved_tensors
        problem = ctx.problem
        P = problem.P
        g = None
        iters = []
        for k, (b0, b1) in enumerate(problem.chunks()):
            fidx = P.fidx[b0:b1].contiguous()
            if ctx.fields is not None:
                u = ctx.fields[k]
            else:  # recompute the chunk's wavefields instead of having stored them
                u, fidx, _, _ = problem.forward_chunk(m, b0, b1)
            gk, (it, _, _) = dbi.adjoint_apply(P.grid, P.ref, m, P.omega, fidx, P.Ghat, u, P.rec_cells,
                                               ctx.residuals[k], tol=problem.tol, max_iter=problem.max_iter,
                                               with_status=True)
            iters.append(it)
            g = gk.to(torch.float64) if g is None else g + gk.to(torch.float64)
        problem.last_stats["adjoint_iters"] = torch.cat(iters)
        return (grad_phi * g).to(m.dtype), None


def misfit(m: torch.Tensor, problem: MisfitProblem) -> torch.Tensor:
    """phi(m), differentiable with respect to m."""
    return ElasticMisfit.apply(m, problem)


def chunk_count(problem: MisfitProblem) -> int:
    return math.ceil(problem.P.B / problem.chunk)

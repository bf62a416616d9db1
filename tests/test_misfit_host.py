"""Host logic of the differentiable misfit (misfit.py) on the CPU: the library calls it makes are
replaced by a linear stand-in (the wavefield of problem b is the model itself, its data residual
r_b = J_f m - d_b with one complex matrix per frequency f, and the adjoint product Re J_f^H r_b
summed over the problems of the call), so that the chunk plan under a memory budget, the kept and
the recomputed wavefields, the per-chunk residuals and the FP64 gradient accumulation can be
checked against the gradient of phi = 1/2 sum_b ||J_f m - d_b||^2 written out densely."""
import types

import numpy as np
import pytest
import torch

from paper_2402_02116_gb300 import misfit as M

NZ, NX, NF, NSRC, NDATA = 3, 4, 2, 3, 10
B = NF * NSRC


def J(f):
    rng = np.random.default_rng(100 + int(f))
    return torch.as_tensor(rng.standard_normal((NDATA, 5 * NZ * NX)) + 1j * rng.standard_normal((NDATA, 5 * NZ * NX)))


class FakeDbi:
    """The four library calls misfit.py makes, as the linear stand-in."""

    def __init__(self):
        self.solves = 0

    def incident_field(self, grid, omega, fidx, Gspace, src_cells, forces):
        return torch.zeros((fidx.numel(), 1), dtype=torch.complex128)

    def ls_solve(self, grid, ref, m, omega, fidx, Ghat, u0, tol=None, max_iter=None):
        self.solves += 1
        n = fidx.numel()
        u = m.reshape(1, -1).to(torch.complex128).repeat(n, 1)
        return u, torch.ones(n, dtype=torch.int32), torch.zeros(n), torch.zeros(n, dtype=torch.int32)

    def data_residual(self, grid, omega, fidx, rec_cells, u, d_obs):
        r = torch.stack([J(int(f)) @ u[k] - d_obs[k] for k, f in enumerate(fidx.tolist())])
        return r, 0.5 * torch.sum(torch.abs(r) ** 2).to(torch.float64)

    def adjoint_apply(self, grid, ref, m, omega, fidx, Ghat, u, rec_cells, r, tol=None, max_iter=None,
                      with_status=False):
        g = sum(torch.real(J(int(f)).conj().T @ r[k]) for k, f in enumerate(fidx.tolist()))
        n = fidx.numel()
        return g.reshape(m.shape).to(m.dtype), (torch.ones(n, dtype=torch.int32), None, None)


def fake_problem():
    fidx = torch.repeat_interleave(torch.arange(NF, dtype=torch.int32), NSRC)
    return types.SimpleNamespace(
        B=B, grid=types.SimpleNamespace(nz=NZ, nx=NX), device=torch.device("cpu"), cdt=torch.complex128,
        fidx=fidx, omega=None, Gspace=None, Ghat=None, ref=None, rec_cells=None,
        src_cells=torch.zeros((B, 2), dtype=torch.int32), forces=torch.zeros((B, 2), dtype=torch.float64))


def observed():
    rng = np.random.default_rng(7)
    return torch.as_tensor(rng.standard_normal((B, NDATA)) + 1j * rng.standard_normal((B, NDATA)))


def dense(m, d):
    """phi and its gradient written out over all problems."""
    phi, g = 0.0, torch.zeros(5 * NZ * NX, dtype=torch.float64)
    fidx = fake_problem().fidx.tolist()
    for b in range(B):
        r = J(fidx[b]) @ m.reshape(-1).to(torch.complex128) - d[b]
        phi += 0.5 * float(torch.sum(torch.abs(r) ** 2))
        g += torch.real(J(fidx[b]).conj().T @ r)
    return phi, g.reshape(m.shape)


@pytest.fixture
def fake(monkeypatch):
    f = FakeDbi()
    monkeypatch.setattr(M, "dbi", f)
    return f


@pytest.mark.parametrize("budget, chunk", [(None, B), (10 ** 9, B), (9 * 2 * NZ * NX * 16 * 4, 4),
                                           (9 * 2 * NZ * NX * 16, 1), (1, 1)])
def test_chunk_plan(fake, budget, chunk):
    prob = M.MisfitProblem(fake_problem(), observed(), memory_budget=budget)
    assert prob.chunk == chunk and prob.keep_fields == (chunk >= B)
    spans = list(prob.chunks())
    assert spans[0][0] == 0 and spans[-1][1] == B and all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
    assert M.chunk_count(prob) == len(spans)


@pytest.mark.parametrize("budget", [None, 9 * 2 * NZ * NX * 16 * 4, 1])
def test_misfit_and_gradient_equal_the_dense_form(fake, budget):
    d = observed()
    prob = M.MisfitProblem(fake_problem(), d, memory_budget=budget)
    rng = np.random.default_rng(3)
    m = torch.as_tensor(rng.standard_normal((5, NZ, NX))).requires_grad_(True)
    phi = M.misfit(m, prob)
    (3.0 * phi).backward()
    phi_d, g_d = dense(m.detach(), d)
    assert float(phi.detach()) == pytest.approx(phi_d, rel=1e-12)
    assert torch.allclose(m.grad, 3.0 * g_d, rtol=1e-12, atol=0)
    chunks = M.chunk_count(prob)
    # forward solves per chunk, and the backward pass recomputes them only when fields are not kept
    assert fake.solves == (chunks if prob.keep_fields else 2 * chunks)

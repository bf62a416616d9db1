"""The differentiable misfit (torch.autograd.Function over the CUDA library) against the FP64 oracle
and against central finite differences, on small grids and on the 512 x 512 VTI misfit workload."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.misfit import MisfitProblem, chunk_count, misfit
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


def _small(seed=51):
    w = inputs.small_case(nz=14, nx=12, amp=0.1, vti=True, n_src=2, freqs=(7.0, 12.0), seed=seed)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx = w.problem_fidx()
    srcs, forces = w.src_cells[w.problem_src()], w.src_force[w.problem_src()]
    U = orc.forward(w.model * 1.02, fidx, srcs, forces)
    d_obs = np.stack([orc.sample(U[b], w.rec_cells) for b in range(len(fidx))])
    return w, orc, fidx, srcs, forces, d_obs


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_misfit_and_gradient_match_oracle(precision):
    w, orc, fidx, srcs, forces, d_obs = _small()
    P = DeviceProblem(w, precision)
    prob = MisfitProblem(P, P.to_field(d_obs), tol=1e-12 if precision == dbi.C128 else 1e-7)
    m = P.m.clone().requires_grad_(True)
    phi = misfit(m, prob)
    phi.backward()
    phi_o, g_o, _ = orc.misfit(w.model, fidx, srcs, forces, d_obs, w.rec_cells)
    assert abs(float(phi.detach()) - phi_o) < (1e-9 if precision == dbi.C128 else 1e-5) * phi_o
    g = npy(m.grad).astype(np.float64)
    for p in range(5):
        assert rel(g[p], g_o[p]) < (1e-7 if precision == dbi.C128 else 1e-4), p


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_recomputed_fields_give_the_same_gradient(precision):
    """With a memory budget below the batch's wavefields the forward pass keeps only residuals and
    the backward pass recomputes each chunk's fields; phi and the gradient do not change."""
    w, orc, fidx, srcs, forces, d_obs = _small(seed=52)
    P = DeviceProblem(w, precision)
    keep = MisfitProblem(P, P.to_field(d_obs), tol=1e-10)
    per = 2 * w.nz * w.nx * (8 if precision == dbi.C64 else 16)
    chunked = MisfitProblem(P, P.to_field(d_obs), tol=1e-10, memory_budget=9 * per)
    assert keep.keep_fields and not chunked.keep_fields and chunk_count(chunked) == P.B
    grads, phis = [], []
    for prob in (keep, chunked):
        m = P.m.clone().requires_grad_(True)
        phi = misfit(m, prob)
        phi.backward()
        grads.append(npy(m.grad).astype(np.float64))
        phis.append(float(phi.detach()))
    tol = 1e-12 if precision == dbi.C128 else 1e-6
    assert abs(phis[0] - phis[1]) <= tol * phis[0]
    assert rel(grads[1], grads[0]) < tol


def test_gradient_matches_finite_differences_on_cells():
    """Central differences of phi (complex128 path) for single-cell perturbations of each
    parameter agree with the complex128 and complex64 adjoint gradients."""
    w, orc, fidx, srcs, forces, d_obs = _small(seed=53)
    P128, P64 = DeviceProblem(w, dbi.C128), DeviceProblem(w, dbi.C64)
    pr128 = MisfitProblem(P128, P128.to_field(d_obs), tol=1e-13)
    pr64 = MisfitProblem(P64, P64.to_field(d_obs), tol=1e-7)
    m = P128.m.clone().requires_grad_(True)
    misfit(m, pr128).backward()
    g128 = npy(m.grad)
    m64 = P64.m.clone().requires_grad_(True)
    misfit(m64, pr64).backward()
    g64 = npy(m64.grad).astype(np.float64)
    sc = orc.param_scale()
    rng = np.random.default_rng(7)
    for _ in range(20):
        p, iz, ix = rng.integers(5), rng.integers(w.nz), rng.integers(w.nx)
        eps = 1e-5 * sc[p]
        mp, mn = P128.m.clone(), P128.m.clone()
        mp[p, iz, ix] += eps
        mn[p, iz, ix] -= eps
        fd = (float(misfit(mp, pr128)) - float(misfit(mn, pr128))) / (2 * eps)
        scale = np.max(np.abs(g128[p]))
        assert abs(fd - g128[p, iz, ix]) < 1e-6 * scale, (p, fd, g128[p, iz, ix])
        assert abs(fd - g64[p, iz, ix]) < 1e-4 * scale, (p, fd, g64[p, iz, ix])


def test_misfit_512_vti_workload_with_recomputation():
    """The 512 x 512 VTI workload (64 sources x 6 frequencies, 256 receivers; smooth random
    contrast): complex64 misfit and gradient with the forward fields recomputed chunk by chunk
    under a 4 GB budget equal those of the keep-everything pass, and the gradient predicts the
    change of phi along a smooth direction (central difference)."""
    w = inputs.config4_misfit()
    P = DeviceProblem(w, dbi.C64)
    # observed data from the true model
    Pt = DeviceProblem(w, dbi.C64, model=w.model_true)
    u_true, _, _, code = Pt.forward(tol=1e-6)
    assert bool((code == dbi.CONVERGED).all())
    d_obs = Pt.sample(u_true)
    del u_true, Pt
    keep = MisfitProblem(P, d_obs, tol=1e-6)
    chunked = MisfitProblem(P, d_obs, tol=1e-6, memory_budget=4 << 30)
    assert chunk_count(chunked) > 1
    out = []
    for prob in (keep, chunked):
        m = P.m.clone().requires_grad_(True)
        phi = misfit(m, prob)
        phi.backward()
        out.append((float(phi.detach()), m.grad.detach().clone()))
    (phi_k, g_k), (phi_c, g_c) = out
    assert np.isfinite(phi_k) and phi_k > 0
    assert abs(phi_k - phi_c) <= 1e-6 * phi_k
    gk64, gc64 = g_k.double(), g_c.double()  # per-cell gradients are ~1e-25: norms in FP64
    assert torch.isfinite(gk64).all() and float(gk64.abs().max()) > 0
    assert float(torch.linalg.norm(gc64 - gk64) / torch.linalg.norm(gk64)) < 1e-5
    # directional derivative: a smooth perturbation of every parameter
    a2 = w.rho0 * w.alpha0 ** 2
    sc = torch.tensor([w.rho0, a2, a2, a2, w.rho0 * w.beta0 ** 2], dtype=torch.float64)
    d = torch.as_tensor(inputs.seeded_real((5, w.nz, w.nx), 9))
    d = torch.nn.functional.avg_pool2d(d[None], 31, stride=1, padding=15)[0]
    d = d / d.abs().amax(dim=(1, 2), keepdim=True)  # smooth, max |d_p| = 1 per parameter
    d = (d * sc[:, None, None] * 1e-3).to(P.device, P.rdt)
    eps = 1.0
    fp = float(misfit(P.m + eps * d, keep))
    fn = float(misfit(P.m - eps * d, keep))
    fd = (fp - fn) / (2 * eps)
    pred = float((g_k.double() * d.double()).sum())
    assert abs(fd - pred) < 2e-3 * abs(pred), (fd, pred)


def test_config4_gradient_matches_finite_differences_on_20_cells():
    """The 512 x 512 VTI workload at full grid size with one source x all 6 frequencies (3-18 Hz),
    complex128: the adjoint gradient (wavefields recomputed chunk by chunk) equals the central
    difference of phi for single-cell perturbations on 20 seeded cells (random parameter, cells in
    the upper 48 rows where the receivers' sensitivity is not negligible), to 1e-4 of the cell's
    value plus 1e-7 of the parameter's largest gradient."""
    w = inputs.config4_misfit(n_src=1)
    P = DeviceProblem(w, dbi.C128)
    d_obs = (inputs.seeded_complex((P.B, len(w.rec_cells), 2), 19) * 1e-10)
    prob = MisfitProblem(P, P.to_field(d_obs), tol=1e-13, memory_budget=3 * 9 * 2 * w.nz * w.nx * 16)
    assert chunk_count(prob) == 2
    m = P.m.clone().requires_grad_(True)
    misfit(m, prob).backward()
    g = npy(m.grad)
    a2 = w.rho0 * w.alpha0 ** 2
    sc = np.array([w.rho0, a2, a2, a2, w.rho0 * w.beta0 ** 2])
    rng = np.random.default_rng(44)
    for _ in range(20):
        p, iz, ix = int(rng.integers(5)), int(rng.integers(1, 48)), int(rng.integers(w.nx))
        eps = 1e-4 * sc[p]
        mp_, mn_ = P.m.clone(), P.m.clone()
        mp_[p, iz, ix] += eps
        mn_[p, iz, ix] -= eps
        fd = (float(misfit(mp_, prob)) - float(misfit(mn_, prob))) / (2 * eps)
        tol = 1e-4 * abs(g[p, iz, ix]) + 1e-7 * np.max(np.abs(g[p]))
        assert abs(fd - g[p, iz, ix]) < tol, (p, iz, ix, fd, g[p, iz, ix])

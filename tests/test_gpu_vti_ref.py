"""A homogeneous VTI reference medium on the GPU (greens_tabulate with VTI stiffness): its Green's
tables from the spectral representation against the oracle's (adaptive quadrature of the same
representation, pinned by the isotropic closed form and the VTI wave equation), the isotropic
special case against the closed-form tables, the LS operator and its solve with a VTI reference
against the oracle, and the effect of the reference on the 256^2 VTI workload (Krylov
iterations, the solution)."""
import dataclasses
import time

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


def background_params(w):
    """(rho, C11, C13, C33, C55) of the homogeneous VTI background the workload's model perturbs."""
    m = inputs.vti_background(1, 1)
    return tuple(float(m[p, 0, 0]) for p in range(5))


def with_vti_reference(w, ref=None):
    return dataclasses.replace(w, ref_vti=background_params(w) if ref is None else tuple(ref))


def test_isotropic_stiffness_reproduces_the_closed_form_tables():
    w = inputs.small_case(nz=20, nx=16, lz=64, lx=32, freqs=(4.0, 17.0))
    iso = DeviceProblem(w, dbi.C128)
    vti = DeviceProblem(with_vti_reference(w, O.reference_params(w.rho0, w.alpha0, w.beta0)), dbi.C128)
    assert rel(npy(vti.Gspace), npy(iso.Gspace)) < 1e-10
    assert rel(npy(vti.Ghat), npy(iso.Ghat)) < 1e-10


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_vti_tables_match_the_oracle(precision):
    w = with_vti_reference(inputs.small_case(nz=6, nx=5, vti=True, freqs=(11.0,)))
    P = DeviceProblem(w, precision)
    lat = O.green_lattice_vti(w.nz, w.nx, w.h, w.omegas[0], *w.ref_vti, epsrel=1e-12)
    tol = 1e-9 if precision == dbi.C128 else 1e-6
    assert rel(npy(P.Gspace[0]), O.embed_circulant(lat, w.lz, w.lx)) < tol
    Gh = O.green_spectrum(lat, w.lz, w.lx) * w.h * w.h / (w.lz * w.lx)
    assert rel(npy(P.Ghat[0]), np.swapaxes(Gh, -1, -2)) < 10 * tol


def test_far_offsets_match_the_oracle():
    """Offsets up to 90 wavelengths of phase (the oscillatory panels of the quadrature)."""
    w = with_vti_reference(inputs.small_case(nz=64, nx=64, lz=128, lx=128, h=10.0, vti=True, freqs=(19.0,)))
    P = DeviceProblem(w, dbi.C128)
    Gs = npy(P.Gspace[0])
    for dz, dx in ((63, 63), (-50, 7), (0, 61), (33, -2), (1, 0)):
        want = O.green_vti_2d(dx * w.h, dz * w.h, w.omegas[0], *w.ref_vti)
        got = [Gs[c, dz % w.lz, dx % w.lx] for c in range(3)]
        scale = max(abs(v) for v in want)
        for c in range(3):
            assert abs(got[c] - want[c]) <= 1e-9 * scale, (dz, dx, c)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_apply_and_solve_with_a_vti_reference(precision):
    w = with_vti_reference(inputs.small_case(nz=7, nx=6, vti=True, freqs=(9.0,), n_src=2))
    P = DeviceProblem(w, precision)
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas, ref_vti=w.ref_vti,
                     vti_epsrel=1e-12)
    ud = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 12))
    u = npy(ud).astype(np.complex128)
    got = npy(P.apply(ud))
    tol = 1e-9 if precision == dbi.C128 else 1e-5
    for q in range(P.B):
        want = orc.apply(u[q], w.model, 0)
        assert np.linalg.norm(got[q] - want) <= tol * np.linalg.norm(want - u[q]), q
    stol = 1e-11 if precision == dbi.C128 else 1e-6
    x, iters, relres, code = P.solve(P.incident(), tol=stol, max_iter=500, check_every=4)
    assert bool((code == dbi.CONVERGED).all())
    srcs = w.problem_src()
    for q in range(P.B):
        u0 = orc.incident(0, w.src_cells[srcs[q]], w.src_force[srcs[q]])
        assert rel(npy(x[q]), orc.solve(u0, w.model, 0, tol=1e-13)) < (1e-8 if precision == dbi.C128 else 1e-5), q


def test_vti_reference_on_the_256_workload():
    """The 256^2 VTI model (8 frequencies 5-20 Hz, 4 sources) with its homogeneous VTI background
    as the reference instead of the isotropic one: the anisotropy leaves the contrast, BiCGSTAB
    needs fewer iterations, and sampled table entries match the oracle."""
    w_iso = inputs.config2_batched_forward(n_src=4)
    w_vti = with_vti_reference(w_iso)
    torch.cuda.synchronize()
    t0 = time.time()
    P = DeviceProblem(w_vti, dbi.C64)
    torch.cuda.synchronize()
    t_tab = time.time() - t0
    Q = DeviceProblem(w_iso, dbi.C64)
    u_v, it_v, _, c_v = P.solve(P.incident(), tol=1e-5, max_iter=3000)
    u_i, it_i, _, c_i = Q.solve(Q.incident(), tol=1e-5, max_iter=3000)
    assert bool((c_v == dbi.CONVERGED).all()) and bool((c_i == dbi.CONVERGED).all())
    d = rel(npy(u_v), npy(u_i))
    print(f"\nVTI reference: tables for 8 frequencies in {t_tab:.2f} s; BiCGSTAB iterations mean "
          f"{float(it_v.float().mean()):.1f} (isotropic reference {float(it_i.float().mean()):.1f}); "
          f"wavefields differ by {d:.3e} (the two discretisations)")
    assert float(it_v.float().mean()) < float(it_i.float().mean())
    f = w_vti.nf - 1
    Gs = npy(P.Gspace[f])
    for dz, dx in ((255, 255), (17, -200), (0, 1)):
        want = O.green_vti_2d(dx * w_vti.h, dz * w_vti.h, w_vti.omegas[f], *w_vti.ref_vti)
        scale = max(abs(v) for v in want)
        for c in range(3):
            assert abs(Gs[c, dz % w_vti.lz, dx % w_vti.lx] - want[c]) <= 1e-6 * scale, (dz, dx, c)

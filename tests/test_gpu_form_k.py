"""The paper-literal form of the LS operator (Eq. 9: central differences on the Green's tensor, five
convolved sources) on the GPU, against the FP64 oracle's form K: the derivative tables, single
operator passes on ragged and multi-tile grids in both precisions, the Krylov solve, and the
identity with the divergence form (Eq. 6 with the stencil on the stress) when the stiffness
contrast vanishes on the outer ring of cells of D. The size of the difference between the two
forms on a contrast that reaches the boundary is measured on the 256^2 VTI workload."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.problem import DeviceProblem

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = {dbi.C64: 1e-5, dbi.C128: 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def npy(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_for(w):
    return O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)


def ring_to_reference(w):
    """The model with every parameter on the outer ring of cells set to the reference medium."""
    ref = O.reference_params(w.rho0, w.alpha0, w.beta0)
    m = w.model.copy()
    for p in range(5):
        m[p, 0, :] = m[p, -1, :] = m[p, :, 0] = m[p, :, -1] = ref[p]
    return m


SHAPES = [
    dict(nz=12, nx=10),                  # ragged, single tile
    dict(nz=5, nx=9, lz=16, lx=32),      # non-square FFT grid
    dict(nz=1, nx=8),                    # one row
    dict(nz=40, nx=24, vti=True),        # several row tiles, VTI background
    dict(nz=64, nx=64, lz=128, lx=128),  # several column tiles
    dict(nz=21, nx=30, lz=64, lx=512, vti=True),  # 512-long rows, ragged
    dict(nz=9, nx=256, lz=32, lx=512),   # 512-long rows at full width
    dict(nz=3, nx=300, lz=16, lx=1024),  # 1024-long rows (two rows per tile)
]
IDS = ["x".join(str(s[k]) for k in ("nz", "nx")) for s in SHAPES]


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES[:5], ids=IDS[:5])
def test_derivative_tables(precision, shape):
    """Dhat = h^2 / (lz lx) FFT of the six combined central-difference tables, column-major."""
    w = inputs.small_case(freqs=(3.0, 17.0), **shape)
    P = DeviceProblem(w, precision, with_space=False)
    orc = oracle_for(w)
    tol = 1e-10 if precision == dbi.C128 else 1e-6
    Dh = npy(P.Dhat)
    assert Dh.shape == (w.nf, 6, w.lx, w.lz)
    for f, om in enumerate(w.omegas):
        DG = O.green_derivative_lattice(w.nz, w.nx, w.h, om, w.alpha0, w.beta0, w.rho0)
        K = O.form_k_spectra(orc.G_lat[f], DG, w.lz, w.lx)
        # sigma11, sigma13, sigma33 columns of the 2 x 5 kernel, first row then second
        want = np.stack([K[0][2], K[1][2], K[0][3], K[1][3], K[0][4], K[1][4]]) * w.h * w.h / (w.lz * w.lx)
        for e in range(6):
            if not np.any(want[e]):  # one row: G13 and D3 G11 vanish on dz = 0 by parity
                assert not np.any(Dh[f, e]), (f, e)
            else:
                assert rel(Dh[f, e], want[e].T) < 10 * tol, (f, e)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_apply_k_matches_oracle(precision, shape):
    w = inputs.small_case(freqs=(4.0, 13.0), n_src=2, **shape)
    P = DeviceProblem(w, precision, with_space=False)
    orc = oracle_for(w)
    ud = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 31))
    u = npy(ud).astype(np.complex128)  # the input as the GPU sees it
    got = npy(P.apply_k(ud))
    fidx = w.problem_fidx()
    for q in range(P.B):
        want = orc.apply_k(u[q], w.model, fidx[q])
        # relative to the scattered part, so that the identity term does not hide an error
        assert np.linalg.norm(got[q] - want) <= TOL[precision] * np.linalg.norm(want - u[q]), q


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_forms_agree_when_the_ring_is_reference_medium(precision):
    """Summation by parts moves the difference from the stress onto G without boundary terms
    exactly when the stress vanishes on the outer ring: both GPU forms then give the same A u."""
    w = inputs.small_case(nz=40, nx=24, vti=True, freqs=(6.0, 11.0))
    P = DeviceProblem(w, precision, model=ring_to_reference(w), with_space=False)
    u = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 41))
    a_k, a_s, un = npy(P.apply_k(u)), npy(P.apply(u)), npy(u)
    assert np.linalg.norm(a_k - a_s) <= TOL[precision] * np.linalg.norm(a_s - un)
    # with the contrast up to the boundary the two forms differ by far more than rounding
    Q = DeviceProblem(w, precision, with_space=False)
    b_k, b_s = npy(Q.apply_k(u)), npy(Q.apply(u))
    assert np.linalg.norm(b_k - b_s) > 1e-3 * np.linalg.norm(b_s - un)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_solve_k_matches_oracle(precision):
    w = inputs.small_case(nz=20, nx=18, n_src=2, freqs=(7.0, 12.0), vti=True)
    P = DeviceProblem(w, precision)
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    u, iters, relres, code = P.solve_k(P.incident(), tol=tol, max_iter=500, check_every=4)
    assert bool((code == dbi.CONVERGED).all()) and float(relres.max()) <= tol
    orc = oracle_for(w)
    fidx, srcs = w.problem_fidx(), w.problem_src()
    got = npy(u)
    for q in range(P.B):
        u0 = orc.incident(fidx[q], w.src_cells[srcs[q]], w.src_force[srcs[q]])
        want = orc.solve_k(u0, w.model, fidx[q], tol=1e-13)
        assert rel(got[q], want) < (1e-8 if precision == dbi.C128 else 1e-5), q


def test_empty_batch_and_argument_errors():
    w = inputs.small_case(nz=8, nx=8, freqs=(5.0,))
    P = DeviceProblem(w, dbi.C64, with_space=False)
    empty = torch.empty((0, 2, w.nz, w.nx), dtype=P.cdt, device=P.device)
    out = dbi.ls_apply_k(P.grid, P.ref, P.m, P.omega, P.fidx[:0], P.Ghat, P.Dhat, empty)
    assert out.shape == empty.shape
    u = P.to_field(inputs.seeded_complex((P.B, 2, w.nz, w.nx), 3))
    lib = dbi.load()
    model = dbi._model(P.grid, P.ref, P.m, dbi.C64)
    batch = dbi._batch(P.omega, P.fidx)
    out = torch.empty_like(u)
    n = dbi.workspace_bytes(P.grid, P.B, dbi.C64, dbi.OP_APPLY_K)
    work = torch.empty(n, dtype=torch.uint8, device=P.device)
    stream = dbi._stream(P.device)
    rc = lib.ls_apply_k(ctypes.byref(model), ctypes.byref(batch), dbi._ptr(P.Ghat), None, dbi._ptr(u),
                        dbi._ptr(out), dbi.C64, dbi._ptr(work), n, stream)
    assert rc != 0 and b"Dhat" in lib.dbi_last_error()
    rc = lib.ls_apply_k(ctypes.byref(model), ctypes.byref(batch), dbi._ptr(P.Ghat), dbi._ptr(P.Dhat),
                        dbi._ptr(u), dbi._ptr(out), dbi.C64, dbi._ptr(work), n - 1, stream)
    assert rc != 0 and b"work buffer" in lib.dbi_last_error()
    torch.cuda.synchronize()


def test_form_difference_on_the_vti_256_workload():
    """The 256^2 VTI model (contrast up to the boundary, 8 frequencies 5-20 Hz): one problem per
    frequency against the oracle's form K, and the size of the form K - form S difference of the
    operator and of the solved wavefield, relative to the scattered field."""
    w = inputs.config2_batched_forward(n_src=1)
    P = DeviceProblem(w, dbi.C64)
    u0 = P.incident()
    a_k, a_s = npy(P.apply_k(u0)), npy(P.apply(u0))
    un = npy(u0)
    orc = oracle_for(w)
    fidx = w.problem_fidx()
    for q in (0, P.B - 1):
        want = orc.apply_k(un[q].astype(np.complex128), w.model, fidx[q])
        assert np.linalg.norm(a_k[q] - want) <= TOL[dbi.C64] * np.linalg.norm(want - un[q]), q
    op_diff = np.linalg.norm(a_k - a_s) / np.linalg.norm(a_s - un)
    uk, _, rk, ck = P.solve_k(u0, tol=1e-6, max_iter=3000)
    us, _, rs, cs = P.solve(u0, tol=1e-6, max_iter=3000)
    assert bool((ck == dbi.CONVERGED).all()) and bool((cs == dbi.CONVERGED).all())
    uk, us = npy(uk), npy(us)
    wf_diff = np.linalg.norm(uk - us) / np.linalg.norm(us - un)
    dk = np.stack([orc.sample(uk[b], w.rec_cells) for b in range(P.B)])
    ds = np.stack([orc.sample(us[b], w.rec_cells) for b in range(P.B)])
    data_diff = np.linalg.norm(dk - ds) / np.linalg.norm(ds)
    print(f"\nform K vs form S on {w.name}: operator {op_diff:.3e}, wavefield {wf_diff:.3e}, "
          f"receiver data {data_diff:.3e}")
    assert 0 < op_diff < 1 and 0 < wf_diff < 1

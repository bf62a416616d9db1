"""The 3D extension on the GPU (include/dbi.h, 3D section) against the 3D FP64 oracle: Green's
tables, incident fields, single operator passes on ragged and multi-tile grids in both
precisions, GMRES solves, and the size of the paper's modified 3D example (80 x 40 x 32 cells,
16 sources x 4 frequencies) with sampled true residuals under the oracle's operator."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.problem import DeviceProblem3D

o3 = O.o3d
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
    return o3.LSOracle3D(w.nz, w.ny, w.nx, w.h, w.lz, w.ly, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)


SHAPES = [
    dict(nz=4, ny=3, nx=5),                      # ragged, smallest FFT grid
    dict(nz=1, ny=2, nx=9),                      # one layer
    dict(nz=6, ny=5, nx=20, lz=16, ly=32, lx=64),  # oversized, non-cubic FFT grid
    dict(nz=9, ny=12, nx=30),                    # several CTAs per pass
    dict(nz=40, ny=2, nx=3),                     # tall columns: z transforms of length 128
    dict(nz=100, ny=1, nx=2),                    # and 256
    dict(nz=2, ny=30, nx=3),                     # y transforms of length 64
    dict(nz=1, ny=100, nx=2),                    # and 256
]
IDS = ["x".join(str(s[k]) for k in ("nz", "ny", "nx")) for s in SHAPES]


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES[:3], ids=IDS[:3])
def test_tables_and_incident_fields(precision, shape):
    w = inputs.small_case_3d(freqs=(6.0, 13.0), n_src=2, **shape)
    P = DeviceProblem3D(w, precision)
    orc = oracle_for(w)
    tol = 1e-10 if precision == dbi.C128 else 1e-6
    for f in range(w.nf):
        assert rel(npy(P.Gspace[f]), o3.embed_circulant_3d(orc.G_lat[f], w.lz, w.ly, w.lx)) < tol
        Gh = orc.G_hat[f] * w.h ** 3 / (w.lz * w.ly * w.lx)
        assert rel(npy(P.Ghat[f]), Gh) < 10 * tol
    u0 = npy(P.incident())
    fidx, srcs = w.problem_fidx(), w.problem_src()
    for q in range(P.B):
        want = orc.incident(fidx[q], w.src_cells[srcs[q]], w.src_force[srcs[q]])
        assert rel(u0[q], want) < tol


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_apply_matches_oracle(precision, shape):
    w = inputs.small_case_3d(freqs=(5.0, 11.0), n_src=2, **shape)
    P = DeviceProblem3D(w, precision, with_space=False)
    orc = oracle_for(w)
    ud = P.to_field(inputs.seeded_complex((P.B, 3, w.nz, w.ny, w.nx), 17))
    u = npy(ud).astype(np.complex128)
    got = npy(P.apply(ud))
    fidx = w.problem_fidx()
    for q in range(P.B):
        want = orc.apply(u[q], w.model, fidx[q])
        assert np.linalg.norm(got[q] - want) <= TOL[precision] * np.linalg.norm(want - u[q]), q


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_gmres_solve_matches_oracle(precision):
    w = inputs.small_case_3d(nz=5, ny=4, nx=6, freqs=(7.0, 12.0), n_src=2, amp=0.15)
    P = DeviceProblem3D(w, precision)
    tol = 1e-11 if precision == dbi.C128 else 1e-6
    u, iters, relres, code = P.solve(P.incident(), tol=tol, max_iter=500, check_every=4)
    assert bool((code == dbi.CONVERGED).all()) and float(relres.max()) <= tol
    orc = oracle_for(w)
    fidx, srcs = w.problem_fidx(), w.problem_src()
    for q in range(P.B):
        u0 = orc.incident(fidx[q], w.src_cells[srcs[q]], w.src_force[srcs[q]])
        want, _ = orc.solve(u0, w.model, fidx[q], tol=1e-13)
        assert rel(npy(u[q]), want) < (1e-8 if precision == dbi.C128 else 1e-5), q


def test_hess3d_sized_batch():
    """80 x 40 x 32 cells (FFT grid 256 x 128 x 64), 16 sources x 4 frequencies, complex64,
    GMRES(30) to 1e-5: every problem converges; sampled problems' true residuals under the
    oracle's operator stay near the tolerance."""
    w = inputs.hess3d_like()
    P = DeviceProblem3D(w, dbi.C64)
    u0 = P.incident()
    u, iters, relres, code = P.solve(u0, restart=30, tol=1e-5, max_iter=2000)
    assert bool((code == dbi.CONVERGED).all()), np.unique(npy(code), return_counts=True)
    print(f"\n3D batch {w.name}: GMRES steps mean {float(iters.float().mean()):.1f} max {int(iters.max())}")
    orc = oracle_for(w)
    fidx = w.problem_fidx()
    for q in (0, P.B - 1):
        x = npy(u[q]).astype(np.complex128)
        r = np.linalg.norm(orc.apply(x, w.model, fidx[q]) - npy(u0[q])) / np.linalg.norm(npy(u0[q]))
        assert r < 3e-5, (q, r)


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_frechet_and_adjoint_match_oracle(precision):
    w = inputs.small_case_3d(nz=4, ny=3, nx=5, freqs=(9.0,), n_src=2, amp=0.1, seed=31)
    P = DeviceProblem3D(w, precision)
    tol = 1e-12 if precision == dbi.C128 else 1e-7
    U_b, _, _, code = P.solve(P.incident(), tol=tol, max_iter=500)
    assert bool((code == dbi.CONVERGED).all())
    rng = np.random.default_rng(5)
    ref = o3.reference_params_3d(w.rho0, w.alpha0, w.beta0)
    dm = ref[:, None, None, None] * 0.01 * rng.standard_normal((6, w.nz, w.ny, w.nx))
    r = rng.standard_normal((P.B, len(w.rec_cells), 3)) + 1j * rng.standard_normal((P.B, len(w.rec_cells), 3))
    d, (it, _, cd) = P.frechet(U_b, P.to_model(dm), tol=tol)
    g, (it2, _, cd2) = P.adjoint(U_b, P.to_field(r), tol=tol)
    assert bool((cd == dbi.CONVERGED).all()) and bool((cd2 == dbi.CONVERGED).all())
    orc = oracle_for(w)
    Ub = npy(U_b).astype(np.complex128)
    fidx = list(w.problem_fidx())
    rec = [tuple(c) for c in w.rec_cells]
    want_d = o3.frechet_3d(orc, w.model, Ub, fidx, dm, rec, tol=1e-13)
    want_g = o3.adjoint_3d(orc, w.model, Ub, fidx, npy(P.to_field(r)).astype(np.complex128), rec, tol=1e-13)
    t = 1e-8 if precision == dbi.C128 else 1e-4
    assert rel(npy(d), want_d) < t
    assert rel(npy(g), want_g) < t
    # the GPU's own dot test
    lhs = float(np.real(np.vdot(npy(P.to_field(r)).astype(np.complex128), npy(d).astype(np.complex128))))
    rhs = float(np.sum(dm * npy(g)))
    assert abs(lhs - rhs) <= (1e-9 if precision == dbi.C128 else 1e-4) * abs(lhs)


@pytest.mark.parametrize("estimate_lambda", [False, True])
def test_normal_cg_matches_oracle(estimate_lambda):
    """Six CG steps of the 3D normal equation (complex128) against the oracle's, with a given
    lambda or lambda from power steps on the normal operator."""
    w = inputs.small_case_3d(nz=4, ny=3, nx=5, freqs=(9.0,), n_src=2, amp=0.1, seed=33)
    P = DeviceProblem3D(w, dbi.C128)
    U_b, _, _, code = P.solve(P.incident(), tol=1e-12, max_iter=500)
    rng = np.random.default_rng(6)
    dd = rng.standard_normal((P.B, len(w.rec_cells), 3)) + 1j * rng.standard_normal((P.B, len(w.rec_cells), 3))
    start = rng.standard_normal((6, w.nz, w.ny, w.nx))
    kw = dict(iters=6, tol=1e-12)
    if estimate_lambda:
        kw.update(lam=None, lambda_rel=1e-2, power_iters=4)
    else:
        kw.update(lam=3e-4)
    dm, lam, hist = P.normal_cg(U_b, P.to_field(dd), power_start=P.to_model(start) if estimate_lambda else None,
                                **kw)
    orc = oracle_for(w)
    rec = [tuple(c) for c in w.rec_cells]
    okw = dict(iters=6, tol=1e-13, lam=None if estimate_lambda else 3e-4, lam_rel=1e-2, power_start=start,
               power_iters=4)
    want, lam_o, hist_o = o3.normal_cg_3d(orc, w.model, npy(U_b), list(w.problem_fidx()), dd, rec, **okw)
    assert lam == pytest.approx(lam_o, rel=1e-8)
    assert np.allclose(hist, hist_o, rtol=1e-7)
    assert rel(npy(dm), want) < 1e-7

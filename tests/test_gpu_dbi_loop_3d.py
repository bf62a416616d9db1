"""The DBI loop on the 3D path (dbi_loop.dbi_inversion_3d): one update against the same steps
composed from the 3D FP64 oracle, and the loop over two frequencies reducing the data error at
each and the model error overall."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.dbi_loop import dbi_inversion_3d, observed_data_3d

o3 = O.o3d
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def case(freqs, seed=41):
    """Reference medium as the starting model; the true model adds +10 % in every parameter in a
    Gaussian anomaly."""
    w = inputs.small_case_3d(nz=5, ny=4, nx=6, freqs=freqs, n_src=3, amp=0.0, seed=seed)
    iz, iy, ix = np.meshgrid(np.arange(5), np.arange(4), np.arange(6), indexing="ij")
    bump = np.exp(-((iz - 2.5) ** 2 + (iy - 1.5) ** 2 + (ix - 3.0) ** 2) / (2 * 1.5 ** 2))
    return w, w.model.copy(), w.model * (1 + 0.1 * bump[None])


def test_one_update_matches_the_oracle_steps():
    w, m0, m_true = case((8.0,))
    d_obs = observed_data_3d(w, m_true, dbi.C128, tol=1e-12)
    res = dbi_inversion_3d(w, d_obs, m0, dbi.C128, max_iter=1, eps_d_stop=0.0, cg_iters=6, lambda_rel=1e-3,
                           m_true=m_true, tol=1e-12, power_iters=4)
    first = res.history[0]
    orc = o3.LSOracle3D(w.nz, w.ny, w.nx, w.h, w.lz, w.ly, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    srcs = w.problem_src()
    rec = [tuple(c) for c in w.rec_cells]

    def forward(m):
        U = np.stack([orc.solve(orc.incident(0, w.src_cells[s], w.src_force[s]), m, 0, tol=1e-13)[0] for s in srcs])
        return U, np.stack([o3.sample_3d(U[b], rec) for b in range(len(srcs))])

    _, d_o = forward(m_true)
    U_b, d_c = forward(m0)
    eps_d = np.linalg.norm(d_c - d_o) / np.linalg.norm(d_o)
    assert abs(first.eps_d - eps_d) < 1e-8 * eps_d
    start = np.random.default_rng(17).standard_normal((6, w.nz, w.ny, w.nx))
    dm, lam, _ = o3.normal_cg_3d(orc, m0, U_b, [0] * len(srcs), d_o - d_c, rec, iters=6, lam=None, lam_rel=1e-3,
                                 power_start=start, power_iters=4, tol=1e-13)
    assert first.lam == pytest.approx(lam, rel=1e-7)
    got = res.m.double().cpu().numpy()
    assert np.linalg.norm(got - (m0 + dm)) / np.linalg.norm(dm) < 1e-6
    assert res.history[1].eps_d < first.eps_d


def test_two_frequencies_reduce_data_and_model_error():
    w, m0, m_true = case((6.0, 11.0), seed=42)
    d_obs = observed_data_3d(w, m_true, dbi.C64, tol=1e-6)
    res = dbi_inversion_3d(w, d_obs, m0, dbi.C64, max_iter=2, cg_iters=10, lambda_rel=1e-3, m_true=m_true,
                           tol=1e-6, power_iters=4)
    h = res.history
    assert sorted({r.freq_hz for r in h}) == [6.0, 11.0]
    for f in (6.0, 11.0):
        recs = [r for r in h if r.freq_hz == f]
        assert recs[-1].eps_d < recs[0].eps_d, (f, [r.eps_d for r in recs])
    assert h[-1].eps_m < h[0].eps_m

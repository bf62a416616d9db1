"""The DBI loop with sequential frequencies (paper_2402_02116_gb300/dbi_loop.py): one update against
the same steps composed from the FP64 oracle, and the loop's behaviour over several updates and
frequencies (the data error falls at every frequency, the model error falls overall)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2402_02116_gb300 import build, dbi, inputs
from paper_2402_02116_gb300.dbi_loop import dbi_inversion, observed_data

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dbi.load()


def case(freqs, n=16, n_src=3, seed=91):
    """Homogeneous isotropic background (the reference medium); the true model adds a Gaussian
    anomaly of +10 % in every parameter."""
    w = inputs.small_case(nz=n, nx=n, n_src=n_src, freqs=freqs, amp=0.0, seed=seed)
    bump = inputs.gaussian_bump(n, n, 0.55 * n, 0.45 * n, n / 6.0)
    m_true = w.model * (1.0 + 0.1 * bump[None])
    return w, w.model.copy(), m_true


def test_one_update_matches_the_oracle_steps():
    w, m0, m_true = case((7.0,))
    d_obs = observed_data(w, m_true, dbi.C128, tol=1e-12)
    res = dbi_inversion(w, d_obs, m0, dbi.C128, max_iter=1, eps_d_stop=0.0, cg_iters=8, lambda_rel=1e-3,
                        m_true=m_true, tol=1e-12)
    first = res.history[0]
    assert first.lam is not None and first.lam > 0
    # the same update composed from the oracle's forward solve, sampling and normal CG
    orc = O.LSOracle(w.nz, w.nx, w.h, w.lz, w.lx, w.rho0, w.alpha0, w.beta0, w.omegas)
    fidx, srcs = w.problem_fidx(), w.problem_src()
    sc, fc = w.src_cells[srcs], w.src_force[srcs]
    U_t = orc.forward(m_true, fidx, sc, fc)
    d_o = np.stack([orc.sample(U_t[b], w.rec_cells) for b in range(len(fidx))])
    U_b = orc.forward(m0, fidx, sc, fc)
    d_c = np.stack([orc.sample(U_b[b], w.rec_cells) for b in range(len(fidx))])
    eps_d = np.linalg.norm(d_c - d_o) / np.linalg.norm(d_o)
    assert abs(first.eps_d - eps_d) < 1e-8 * eps_d
    dm, _, _ = orc.normal_cg(m0, U_b, fidx, d_o - d_c, w.rec_cells, iters=8, lam=first.lam)
    m1 = m0 + dm
    got = res.m.double().cpu().numpy()
    assert np.linalg.norm(got - m1) / np.linalg.norm(dm) < 1e-7
    # the update reduces the data error
    assert res.history[1].eps_d < first.eps_d


@pytest.mark.parametrize("precision", [dbi.C128, dbi.C64])
def test_sequential_frequencies_reduce_data_and_model_error(precision):
    w, m0, m_true = case((5.0, 9.0, 13.0), n=20, n_src=4, seed=92)
    tol = 1e-10 if precision == dbi.C128 else 1e-6
    d_obs = observed_data(w, m_true, precision, tol=tol)
    res = dbi_inversion(w, d_obs, m0, precision, max_iter=3, cg_iters=15, lambda_rel=1e-3, cooling=0.5,
                        m_true=m_true, tol=tol)
    h = res.history
    freqs = sorted({r.freq_hz for r in h})
    assert freqs == [5.0, 9.0, 13.0] and [r.freq_hz for r in h] == sorted(r.freq_hz for r in h)
    for f in freqs:
        recs = [r for r in h if r.freq_hz == f]
        assert recs[-1].eps_d < recs[0].eps_d, (f, [r.eps_d for r in recs])
        lams = [r.lam for r in recs if r.lam is not None]
        assert all(b == pytest.approx(0.5 * a) for a, b in zip(lams, lams[1:]))  # cooling
    assert h[-1].eps_m < h[0].eps_m
    assert bool(torch.isfinite(res.m).all())

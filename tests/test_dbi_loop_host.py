"""The DBI loop's control logic on the CPU (dbi_loop.dbi_inversion and dbi_inversion_3d), with a
linear stand-in for the per-frequency problem: the "background wavefield" is the model itself, the
data are d = J_f m for a fixed complex matrix per frequency, and the normal equation
(Re J^H J + lambda I) dm = Re J^H r is solved densely with lambda_max from the dense spectrum.
Checked: frequencies run from the lowest whatever their input order; a frequency stops when the
data error falls below eps_d_stop or after max_iter updates; lambda starts at lambda_rel lambda_max
and is multiplied by `cooling` after every update; the model error is recorded only with a true
model; a background solve that does not converge stops the loop with an error."""
import numpy as np
import pytest
import torch

from paper_2402_02116_gb300 import dbi, inputs
from paper_2402_02116_gb300.dbi_loop import dbi_inversion, dbi_inversion_3d

N_DATA = 24


class LinearProblem:
    """Per-frequency stand-in with the methods the loop calls."""

    created = []          # frequencies in the order the loop built their problems
    fail_solve = False

    def __init__(self, w, precision, model=None):
        self.freq = float(w.freqs_hz[0])
        self.shape = np.asarray(model).shape
        self.device = torch.device("cpu")
        self.cdt = dbi.complex_dtype(precision)
        self.J = self.matrix(self.freq, int(np.prod(self.shape)))
        LinearProblem.created.append(self.freq)

    @staticmethod
    def matrix(freq, n):
        rng = np.random.default_rng(int(round(freq * 1000)))
        return rng.standard_normal((N_DATA, n)) + 1j * rng.standard_normal((N_DATA, n))

    @staticmethod
    def lambda_max(J):
        return float(np.linalg.eigvalsh(np.real(J.conj().T @ J)).max())

    def incident(self):
        return None

    def to_model(self, arr):
        return torch.as_tensor(np.asarray(arr, dtype=np.float64))

    def solve(self, rhs, m=None, tol=None, **_):
        code = dbi.NOT_CONVERGED if LinearProblem.fail_solve else dbi.CONVERGED
        return (m.clone(), torch.tensor([3]), torch.tensor([1e-12]), torch.tensor([code]))

    def sample(self, u):
        return torch.as_tensor(self.J @ u.double().numpy().reshape(-1))

    def normal_cg(self, u_b, dd, iters=30, lam=None, lambda_rel=1e-3, power_iters=10, power_start=None,
                  m_b=None, tol=None):
        J = self.J
        lam_used = lambda_rel * self.lambda_max(J) if lam is None else lam
        H = np.real(J.conj().T @ J) + lam_used * np.eye(J.shape[1])
        dm = np.linalg.solve(H, np.real(J.conj().T @ dd.numpy()))
        return torch.as_tensor(dm.reshape(self.shape)), lam_used, []


def observed(freqs, m_true):
    return [torch.as_tensor(LinearProblem.matrix(f, m_true.size) @ m_true.reshape(-1)) for f in freqs]


def setup_2d(freqs):
    w = inputs.small_case(nz=3, nx=4, freqs=freqs)
    rng = np.random.default_rng(3)
    m_true = w.model * (1 + 0.05 * rng.standard_normal(w.model.shape))
    return w, m_true, observed(w.freqs_hz, m_true)


@pytest.fixture(autouse=True)
def _reset():
    LinearProblem.created = []
    LinearProblem.fail_solve = False


def run2d(w, d_obs, m0, **kw):
    return dbi_inversion(w, d_obs, m0, dbi.C128, problem=LinearProblem, device="cpu", **kw)


def test_frequencies_from_the_lowest_and_max_iter_updates_each():
    w, m_true, d_obs = setup_2d((12.0, 4.0, 8.0))
    res = run2d(w, d_obs, w.model, max_iter=3, eps_d_stop=0.0, lambda_rel=1e-2, cooling=0.5)
    assert LinearProblem.created == [4.0, 8.0, 12.0]
    assert [r.freq_hz for r in res.history] == [4.0] * 4 + [8.0] * 4 + [12.0] * 4
    for f in (4.0, 8.0, 12.0):
        recs = [r for r in res.history if r.freq_hz == f]
        assert [r.iteration for r in recs] == [0, 1, 2, 3]
        assert recs[-1].lam is None and all(r.lam is not None for r in recs[:-1])


def test_lambda_starts_at_lambda_rel_of_lambda_max_and_cools():
    w, m_true, d_obs = setup_2d((6.0, 9.0))
    res = run2d(w, d_obs, w.model, max_iter=4, eps_d_stop=0.0, lambda_rel=3e-2, cooling=0.25)
    for f in (6.0, 9.0):
        lams = [r.lam for r in res.history if r.freq_hz == f and r.lam is not None]
        lam0 = 3e-2 * LinearProblem.lambda_max(LinearProblem.matrix(f, w.model.size))
        assert lams[0] == pytest.approx(lam0, rel=1e-12)
        for a, b in zip(lams, lams[1:]):
            assert b == pytest.approx(0.25 * a, rel=1e-12)


def test_stops_when_the_data_error_falls_below_the_threshold():
    """With a small lambda the first update nearly fits the data (more unknowns than data), so every
    frequency stops after one update, with its last data error below eps_d_stop."""
    w, m_true, d_obs = setup_2d((5.0, 10.0))
    res = run2d(w, d_obs, w.model, max_iter=10, eps_d_stop=1e-3, lambda_rel=1e-9, m_true=m_true)
    for f in (5.0, 10.0):
        recs = [r for r in res.history if r.freq_hz == f]
        assert len(recs) == 2 and recs[0].eps_d > 1e-3 and recs[-1].eps_d < 1e-3
        assert all(r.eps_m is not None for r in recs)
    first = res.history[0]
    assert first.eps_m == pytest.approx(np.linalg.norm(w.model - m_true) / np.linalg.norm(m_true), rel=1e-12)


def test_model_error_only_with_a_true_model_and_the_update_is_applied():
    w, m_true, d_obs = setup_2d((7.0,))
    res = run2d(w, d_obs, w.model, max_iter=1, eps_d_stop=0.0, lambda_rel=1e-2)
    assert all(r.eps_m is None for r in res.history)
    J = LinearProblem.matrix(7.0, w.model.size)
    r0 = d_obs[0].numpy() - J @ w.model.reshape(-1)
    lam = 1e-2 * LinearProblem.lambda_max(J)
    dm = np.linalg.solve(np.real(J.conj().T @ J) + lam * np.eye(w.model.size), np.real(J.conj().T @ r0))
    assert np.allclose(res.m.numpy(), w.model + dm.reshape(w.model.shape), rtol=1e-12, atol=0)


def test_a_background_solve_that_does_not_converge_stops_the_loop():
    w, m_true, d_obs = setup_2d((7.0,))
    LinearProblem.fail_solve = True
    with pytest.raises(RuntimeError, match="did not converge"):
        run2d(w, d_obs, w.model, max_iter=2)


def test_the_3d_loop_follows_the_same_rules():
    w = inputs.small_case_3d(nz=2, ny=2, nx=3, freqs=(9.0, 3.0))
    rng = np.random.default_rng(4)
    m_true = w.model * (1 + 0.05 * rng.standard_normal(w.model.shape))
    d_obs = observed(w.freqs_hz, m_true)
    res = dbi_inversion_3d(w, d_obs, w.model, dbi.C128, max_iter=2, eps_d_stop=0.0, lambda_rel=1e-2, cooling=0.5,
                           m_true=m_true, problem=LinearProblem, device="cpu")
    assert LinearProblem.created == [3.0, 9.0]
    assert [(r.freq_hz, r.iteration) for r in res.history] == [(3.0, 0), (3.0, 1), (3.0, 2), (9.0, 0), (9.0, 1),
                                                               (9.0, 2)]
    lams = [r.lam for r in res.history if r.freq_hz == 3.0 and r.lam is not None]
    assert lams[1] == pytest.approx(0.5 * lams[0], rel=1e-12)
    assert res.history[-1].eps_d < res.history[3].eps_d

"""The seeded synthetic workloads (inputs.py) have the shapes and structure their recipes state:
grid and FFT sizes, sources, receivers and frequencies, the reference and background media (the
VTI background from Thomsen's delta), the bounds of the contrast, and determinism under the seed.
CPU only."""
import math

import numpy as np
import pytest

from paper_2402_02116_gb300 import inputs as I


def _pow2_at_least(n):
    return 1 << (n - 1).bit_length()


def test_vti_background_follows_thomsen():
    """rho 2200, C33 = rho alpha_v^2 (2500 m/s), C55 = C33 / 3, C11 = 1.2 C33 and
    (C13 + C55)^2 = (C33 - C55)(C33 (1 + 2 delta) - C55) with delta = 0.1."""
    rho, c11, c13, c33, c55 = I.vti_background(2, 3)[:, 1, 2]
    assert rho == 2200.0 and c33 == pytest.approx(2200.0 * 2500.0 ** 2, rel=1e-15)
    assert c55 == pytest.approx(c33 / 3, rel=1e-15) and c11 == pytest.approx(1.2 * c33, rel=1e-15)
    assert (c13 + c55) ** 2 == pytest.approx((c33 - c55) * (c33 * 1.2 - c55), rel=1e-14)


def test_config1():
    w = I.config1_tiny()
    assert (w.nz, w.nx, w.h, w.lz, w.lx) == (32, 32, 10.0, 64, 64)
    assert list(w.freqs_hz) == [10.0] and w.src_cells.tolist() == [[0, 16]] and w.src_force.tolist() == [[0.0, 1.0]]
    assert w.rec_cells.tolist() == [[0, j] for j in range(1, 32, 2)]
    assert (w.rho0, w.alpha0, w.beta0) == (2000.0, 2000.0, 1155.0)
    ratio = w.model / I.isotropic_model(32, 32, 2000.0, 2000.0, 1155.0)
    assert ratio.min() >= 1.0 and ratio.max() == pytest.approx(1.1, rel=1e-12)
    iz, ix = np.unravel_index(np.argmax(ratio[1]), ratio[1].shape)
    assert (iz, ix) == (16, 16)


def test_config2_the_benchmark_workload():
    w = I.config2_batched_forward()
    assert (w.nz, w.nx, w.h, w.lz, w.lx) == (256, 256, 5.0, 512, 512)
    assert np.allclose(w.freqs_hz, np.linspace(5.0, 20.0, 8)) and w.n_src == 32 and w.n_problems == 256
    assert np.all(w.src_cells[:, 0] == 0) and len(np.unique(w.src_cells[:, 1])) == 32
    assert w.rec_cells.tolist() == [[0, j] for j in range(0, 256, 2)]
    ratio = w.model / I.vti_background(256, 256)
    assert ratio.min() >= 0.85 - 1e-12 and ratio.max() <= 1.15 + 1e-12
    assert ratio.min() < 0.9 and ratio.max() > 1.1  # the contrast uses its range
    rho0, a0, b0 = w.rho0, w.alpha0, w.beta0  # isotropic reference from the background
    _, c11, _, c33, c55 = I.vti_background(1, 1)[:, 0, 0]
    assert rho0 == 2200.0 and rho0 * a0 * a0 == pytest.approx(0.5 * (c11 + c33)) and rho0 * b0 * b0 == pytest.approx(c55)


def test_config3_background_is_the_smoothed_true_model():
    w = I.config3_linear_dbi()
    assert (w.nz, w.nx, w.h, w.lz) == (128, 128, 10.0, 256) and list(w.freqs_hz) == [4.0, 8.0, 12.0, 16.0]
    assert w.n_src == 16 and len(w.rec_cells) == 64
    tv = lambda m: np.abs(np.diff(m, axis=-1)).sum() + np.abs(np.diff(m, axis=-2)).sum()  # noqa: E731
    ref = I.isotropic_model(128, 128, w.rho0, w.alpha0, w.beta0)
    for p in range(5):  # smoothing lowers the total variation and the peak deviation from the reference
        assert tv(w.model[p]) < tv(w.model_true[p])
        assert np.abs(w.model[p] - ref[p]).max() < np.abs(w.model_true[p] - ref[p]).max()
    assert np.abs(w.model_true / ref - 1).max() <= 0.4 and np.abs(w.model_true / ref - 1).max() > 0.05


def test_config4_misfit_workload():
    """512^2, h = 5 m, 64 sources x 3-18 Hz, 256 receivers; the misfit starts from the VTI
    background and the true model perturbs it by at most 10 % per parameter (reached)."""
    w = I.config4_misfit()
    assert (w.nz, w.nx, w.h, w.lz, w.lx) == (512, 512, 5.0, 1024, 1024)
    assert w.n_src == 64 and list(w.freqs_hz) == [3.0, 6.0, 9.0, 12.0, 15.0, 18.0] and len(w.rec_cells) == 256
    bg = I.vti_background(512, 512)
    assert np.array_equal(w.model, bg)
    p = np.abs(w.model_true / bg - 1).max(axis=(1, 2))
    assert np.allclose(p, 0.1, rtol=1e-12)


def test_fft_len():
    assert [I.fft_len(n) for n in (1, 8, 9, 256, 257, 384, 385, 512)] == [16, 16, 32, 512, 1024, 1024, 1024, 1024]
    assert [I.fft_len(n, radix3=True) for n in (256, 257, 384, 385, 512)] == [512, 768, 768, 1024, 1024]


def test_config5_uneven_batch():
    ws = I.config5_uneven()
    assert [w.lz for w in I.config5_uneven(radix3=False)] == [1024 if w.lz == 768 else w.lz for w in ws]
    assert len(ws) == 40
    assert sum(w.n_problems for w in ws) == 3074
    assert sum(w.n_problems * w.nz * w.nx for w in ws) == 289_759_232
    for w in ws:
        L = 768 if w.nz == 384 else _pow2_at_least(2 * w.nz - 1)  # 3 x 256 for the 384^2 members
        assert w.nz == w.nx and w.nz in (64, 128, 256, 384, 512) and w.lz == w.lx == L
        assert 1 <= w.n_src <= 32 and 1 <= len(w.freqs_hz) <= 8
        assert np.all(np.diff(w.freqs_hz) >= 0) and w.freqs_hz.min() >= 2.0 and w.freqs_hz.max() <= 25.0


def test_hess3d_like():
    w = I.hess3d_like()
    assert (w.nz, w.ny, w.nx, w.h) == (32, 40, 80, 25.0) and (w.lz, w.ly, w.lx) == (64, 128, 256)
    assert w.n_src == 16 and list(w.freqs_hz) == [3.0, 5.0, 7.0, 9.0] and w.n_problems == 64
    assert np.all(w.src_cells[:, 0] == 0) and np.all(w.src_force == [0.0, 0.0, 1.0])
    assert len(w.rec_cells) == 20 * 40 and np.all(w.rec_cells[:, 0] == 0)
    ratio = w.model / I.vti_background_3d(32, 40, 80)
    assert ratio.min() >= 0.85 - 1e-12 and ratio.max() <= 1.15 + 1e-12
    bg = I.vti_background_3d(1, 1, 1)[:, 0, 0, 0]
    assert bg[5] == bg[4]  # C66 = C55: the 2D background extended along y
    assert w.nz * w.h == 800.0 and w.ny * w.h == 1000.0 and w.nx * w.h == 2000.0


@pytest.mark.parametrize("make", [I.config2_batched_forward, I.config3_linear_dbi, I.hess3d_like])
def test_seeded_and_deterministic(make):
    a, b = make(), make()
    assert np.array_equal(a.model, b.model) and np.array_equal(a.src_cells, b.src_cells)
    assert math.isclose(float(np.sum(a.model)), float(np.sum(b.model)), rel_tol=0, abs_tol=0)


def test_the_paper_3d_acquisition():
    """100 sources and 400 receivers uniformly on the surface, 7 frequencies 3-15 Hz, on the same
    80 x 40 x 32 model as the benchmark's 3D workload."""
    w, base = I.hess3d_paper_acquisition(), I.hess3d_like()
    assert w.n_src == 100 and len(w.rec_cells) == 400 and list(w.freqs_hz) == [3.0, 5.0, 7.0, 9.0, 11.0, 13.0, 15.0]
    assert np.array_equal(w.model, base.model)
    for cells in (w.src_cells, w.rec_cells):
        assert np.all(cells[:, 0] == 0) and len({tuple(c) for c in cells.tolist()}) == len(cells)
        assert np.all((cells[:, 1] >= 0) & (cells[:, 1] < 40) & (cells[:, 2] >= 0) & (cells[:, 2] < 80))
    ys, xs = np.unique(w.rec_cells[:, 1]), np.unique(w.rec_cells[:, 2])
    assert len(ys) == 20 and len(xs) == 20 and np.ptp(np.diff(ys)) <= 1 and np.ptp(np.diff(xs)) <= 1
    # one frequency of it is one library call: B * 3 * nz = 100 * 3 * 32 within the 3D launch limit
    assert w.n_src * 3 * w.nz <= 65535


@pytest.mark.parametrize("make, shape, n_src, n_rec, freqs", [
    (I.reservoir_like, (45, 180), 45, 90, [3, 5, 7, 9, 11, 13, 15, 17, 19]),
    (I.hess2d_like, (43, 161), 40, 80, [3, 5, 7, 9, 11, 13, 15, 17]),
])
def test_the_paper_2d_example_geometries(make, shape, n_src, n_rec, freqs):
    """The reservoir (3600 m x 900 m) and 2D Hess (3220 m x 860 m) examples' grids of 20 m cells,
    surface acquisition and frequencies; the initial model is the smoothed true model."""
    w = make()
    assert (w.nz, w.nx, w.h) == (*shape, 20.0) and w.lz >= 2 * w.nz - 1 and w.lx >= 2 * w.nx - 1
    assert w.n_src == n_src and len(w.rec_cells) == n_rec and list(w.freqs_hz) == freqs
    for cells in (w.src_cells, w.rec_cells):
        assert np.all(cells[:, 0] == 0) and len(np.unique(cells[:, 1])) == len(cells)
    ratio = w.model_true / I.vti_background(w.nz, w.nx)
    assert ratio.min() >= 0.85 - 1e-12 and ratio.max() <= 1.15 + 1e-12
    tv = lambda m: np.abs(np.diff(m, axis=-1)).sum() + np.abs(np.diff(m, axis=-2)).sum()  # noqa: E731
    for p in range(5):
        assert tv(w.model[p]) < tv(w.model_true[p])

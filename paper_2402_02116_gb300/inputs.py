"""Seeded synthetic workloads for the 2D elastic distorted-Born problem.

This module only *describes* inputs: grids, the homogeneous isotropic reference medium,
absolute model fields (rho, C11, C13, C33, C55 per cell), sources, receivers, frequencies and
seeded random vectors. It holds none of the method's arithmetic (no Green's tensor, no
contrast, no stencil, no convolution), so both the CUDA path and the CPU oracle can consume
its output without sharing any computation.

Conventions: the grid is [nz][nx] with row index iz (depth, x3) and column index ix
(horizontal, x1); cell centres sit at (x1, x3) = (ix*h, iz*h). Parameter order is
(rho, C11, C13, C33, C55), the 2D P-SV restriction of the VTI stiffness matrix
(Section "Abbreviated subscript notation", Eq. 39). Problems are ordered
frequency-major: problem b = f * n_src + s.

The paper's own models (the 2D reservoir and the Hess VTI model of Section "Numerical
examples") are not available; the recipes below stand in for them with the same kinds of
structure (layers, localized anomalies, smooth random perturbations, VTI backgrounds).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PARAMS = ("rho", "C11", "C13", "C33", "C55")


@dataclasses.dataclass
class Workload:
    name: str
    nz: int
    nx: int
    h: float
    lz: int
    lx: int
    rho0: float          # homogeneous isotropic reference medium (Eq. 4)
    alpha0: float
    beta0: float
    model: np.ndarray    # [5][nz][nx] float64 absolute (rho, C11, C13, C33, C55) of the medium
    freqs_hz: np.ndarray  # [nf]
    src_cells: np.ndarray  # [n_src][2] int (iz, ix)
    src_force: np.ndarray  # [n_src][2] float (f1, f3)
    rec_cells: np.ndarray  # [n_rec][2] int (iz, ix)
    model_true: np.ndarray | None = None  # for inversion workloads: the model that made the data
    ref_vti: tuple | None = None  # (rho, C11, C13, C33, C55) of a homogeneous VTI reference, or None
    krylov_tol: float = 1e-5
    seed: int = 0

    @property
    def omegas(self) -> np.ndarray:
        return 2.0 * np.pi * np.asarray(self.freqs_hz, dtype=np.float64)

    @property
    def n_src(self) -> int:
        return int(self.src_cells.shape[0])

    @property
    def nf(self) -> int:
        return int(len(self.freqs_hz))

    @property
    def n_problems(self) -> int:
        return self.n_src * self.nf

    def problem_fidx(self) -> np.ndarray:
        """Frequency index of every problem (frequency-major order)."""
        return np.repeat(np.arange(self.nf, dtype=np.int32), self.n_src)

    def problem_src(self) -> np.ndarray:
        """Source index of every problem (frequency-major order)."""
        return np.tile(np.arange(self.n_src, dtype=np.int32), self.nf)


def isotropic_model(nz, nx, rho, alpha, beta) -> np.ndarray:
    """Absolute (rho, C11, C13, C33, C55) of a homogeneous isotropic medium."""
    m = np.empty((5, nz, nx), dtype=np.float64)
    m[0] = rho
    m[1] = rho * alpha * alpha
    m[2] = rho * (alpha * alpha - 2.0 * beta * beta)
    m[3] = rho * alpha * alpha
    m[4] = rho * beta * beta
    return m


def vti_background(nz, nx, rho=2200.0, alpha_v=2500.0, eps_ratio=1.2, delta=0.1) -> np.ndarray:
    """VTI background: C33 = rho*alpha_v^2, C55 = C33/3 (beta = alpha_v/sqrt 3), C11 = 1.2*C33,
    and C13 from Thomsen's delta, C13 = sqrt(2 delta C33 (C33 - C55) + (C33 - C55)^2) - C55."""
    c33 = rho * alpha_v ** 2
    c55 = rho * (alpha_v / math.sqrt(3.0)) ** 2
    c11 = eps_ratio * c33
    c13 = math.sqrt(2.0 * delta * c33 * (c33 - c55) + (c33 - c55) ** 2) - c55
    m = np.empty((5, nz, nx), dtype=np.float64)
    m[0], m[1], m[2], m[3], m[4] = rho, c11, c13, c33, c55
    return m


def isotropic_reference_for(m_bg: np.ndarray):
    """Homogeneous isotropic reference for a (possibly VTI) homogeneous background:
    rho0 = rho_b, rho0*alpha0^2 = (C11_b + C33_b)/2, rho0*beta0^2 = C55_b."""
    rho = float(m_bg[0].flat[0])
    c11, c33, c55 = float(m_bg[1].flat[0]), float(m_bg[3].flat[0]), float(m_bg[4].flat[0])
    alpha0 = math.sqrt(0.5 * (c11 + c33) / rho)
    beta0 = math.sqrt(c55 / rho)
    return rho, alpha0, beta0


def gaussian_bump(nz, nx, cz, cx, sigma):
    iz = np.arange(nz)[:, None]
    ix = np.arange(nx)[None, :]
    return np.exp(-((iz - cz) ** 2 + (ix - cx) ** 2) / (2.0 * sigma * sigma))


def surface_line(n, count, offset=0.5):
    """`count` evenly spaced column indices on a row of `n` cells."""
    return np.array([min(n - 1, int((k + offset) * n / count)) for k in range(count)], dtype=np.int64)


def _gauss_filter(a, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma, mode="nearest")


def config1_tiny(n=32) -> Workload:
    """Isotropic homogeneous background (2000, 1155, 2000), 32x32 cells, h = 10 m, FFT grid 64x64,
    one 10 Hz vertical point force at the top centre, 16 two-component receivers on the top row
    (odd columns), Gaussian inclusion (sigma = 4 cells) raising C11, C13, C33, C55 and rho by 10 %."""
    rho, a, b = 2000.0, 2000.0, 1155.0
    m_bg = isotropic_model(n, n, rho, a, b)
    g = gaussian_bump(n, n, n // 2, n // 2, 4.0 * n / 32.0)
    model = m_bg * (1.0 + 0.10 * g[None])
    return Workload(
        name=f"iso{n}x{n}_1src_1f", nz=n, nx=n, h=10.0, lz=2 * n, lx=2 * n,
        rho0=rho, alpha0=a, beta0=b, model=model,
        freqs_hz=np.array([10.0]),
        src_cells=np.array([[0, n // 2]]), src_force=np.array([[0.0, 1.0]]),
        rec_cells=np.array([[0, j] for j in range(1, n, 2)]),
        krylov_tol=1e-8, seed=1)


def _random_layers(rng, nz, nx, n_layers, amp):
    pert = np.zeros((5, nz, nx))
    depths = np.sort(rng.uniform(0.1 * nz, 0.9 * nz, size=n_layers)).astype(int)
    for k in range(n_layers):
        z0 = depths[k]
        z1 = depths[k + 1] if k + 1 < n_layers else nz
        pert[:, z0:z1, :] = rng.uniform(-amp, amp, size=5)[:, None, None]
    return pert


def _random_anomalies(rng, nz, nx, count, amp, sigma_range):
    pert = np.zeros((5, nz, nx))
    for _ in range(count):
        cz = rng.uniform(0.2 * nz, 0.8 * nz)
        cx = rng.uniform(0.2 * nx, 0.8 * nx)
        sig = rng.uniform(*sigma_range)
        sign = rng.choice([-1.0, 1.0], size=5)
        pert += (amp * sign)[:, None, None] * gaussian_bump(nz, nx, cz, cx, sig)[None]
    return pert


def config2_batched_forward(n=256, n_src=32, nf=8, seed=2) -> Workload:
    """VTI background (rho 2200, C11 = 1.2 C33, C13 from Thomsen delta = 0.1), n x n cells, h = 5 m,
    n_src surface point sources x nf frequencies 5-20 Hz, receivers on every 2nd column of the top
    row; contrast = 3 random horizontal layers + 4 Gaussian anomalies (sigma 5-20 cells), each
    +/-15 % per parameter, clipped to +/-15 %."""
    rng = np.random.default_rng(seed)
    m_bg = vti_background(n, n)
    rho0, a0, b0 = isotropic_reference_for(m_bg)
    scale = n / 256.0
    pert = _random_layers(rng, n, n, 3, 0.15)
    pert += _random_anomalies(rng, n, n, 4, 0.15, (5.0 * scale, 20.0 * scale))
    pert = np.clip(pert, -0.15, 0.15)
    model = m_bg * (1.0 + pert)
    cols = surface_line(n, n_src)
    return Workload(
        name=f"vti{n}x{n}_{n_src}src_{nf}f", nz=n, nx=n, h=5.0, lz=2 * n, lx=2 * n,
        rho0=rho0, alpha0=a0, beta0=b0, model=model,
        freqs_hz=np.linspace(5.0, 20.0, nf),
        src_cells=np.stack([np.zeros_like(cols), cols], axis=1),
        src_force=np.tile([0.0, 1.0], (n_src, 1)),
        rec_cells=np.array([[0, j] for j in range(0, n, 2)]),
        krylov_tol=1e-5, seed=seed)


def _paper_2d_example(name, nz, nx, n_src, n_rec, freqs, smooth, seed) -> Workload:
    """A stand-in with the geometry of one of the paper's 2D VTI examples (their models are not
    available): nz x nx cells of 20 m, n_src vertical forces and n_rec receivers evenly on the
    surface; true model = the config-2 VTI background with 3 random horizontal layers and 4
    Gaussian anomalies (sigma 3-10 cells), each +/-15 % per parameter, clipped to +/-15 %; initial
    model = the true model smoothed by a Gaussian of `smooth` cells, as the paper builds it."""
    rng = np.random.default_rng(seed)
    m_bg = vti_background(nz, nx)
    rho0, a0, b0 = isotropic_reference_for(m_bg)
    pert = _random_layers(rng, nz, nx, 3, 0.15) + _random_anomalies(rng, nz, nx, 4, 0.15, (3.0, 10.0))
    m_true = m_bg * (1.0 + np.clip(pert, -0.15, 0.15))
    m0 = np.stack([_gauss_filter(m_true[p], smooth) for p in range(5)])
    src, rec = surface_line(nx, n_src), surface_line(nx, n_rec)
    return Workload(
        name=name, nz=nz, nx=nx, h=20.0, lz=fft_len(nz), lx=fft_len(nx), rho0=rho0, alpha0=a0, beta0=b0,
        model=m0, model_true=m_true, freqs_hz=np.asarray(freqs, dtype=np.float64),
        src_cells=np.stack([np.zeros_like(src), src], axis=1), src_force=np.tile([0.0, 1.0], (n_src, 1)),
        rec_cells=np.stack([np.zeros_like(rec), rec], axis=1), krylov_tol=1e-5, seed=seed)


def reservoir_like(seed=7) -> Workload:
    """The geometry of the paper's 2D VTI reservoir example: 180 x 45 cells (3600 m x 900 m), 45
    sources, 90 receivers, 9 frequencies 3-19 Hz, initial model smoothed over 15 cells."""
    return _paper_2d_example("reservoir_like_180x45", 45, 180, 45, 90, np.arange(3.0, 20.0, 2.0), 15.0, seed)


def hess2d_like(seed=8) -> Workload:
    """The geometry of the paper's 2D VTI Hess example: 161 x 43 cells (3220 m x 860 m), 40 sources,
    80 receivers, 8 frequencies 3-17 Hz, initial model smoothed over 14 cells."""
    return _paper_2d_example("hess2d_like_161x43", 43, 161, 40, 80, np.arange(3.0, 18.0, 2.0), 14.0, seed)


def config3_linear_dbi(n=128, n_src=16, freqs=(4.0, 8.0, 12.0, 16.0), seed=3) -> Workload:
    """Isotropic reference (2000, 1155, 2000); true model = reference + 4 seeded Gaussian anomalies
    (+/-10 % per parameter); the DBI background is the true model smoothed by a Gaussian of 8 cells
    (the paper starts from smoothed true models). n x n cells, h = 10 m, 16 sources x 4 frequencies,
    receivers on every 2nd column of the top row."""
    rng = np.random.default_rng(seed)
    rho, a, b = 2000.0, 2000.0, 1155.0
    m_ref = isotropic_model(n, n, rho, a, b)
    scale = n / 128.0
    pert = _random_anomalies(rng, n, n, 4, 0.10, (4.0 * scale, 12.0 * scale))
    m_true = m_ref * (1.0 + pert)
    m_b = np.stack([_gauss_filter(m_true[p], 8.0 * scale) for p in range(5)])
    cols = surface_line(n, n_src)
    return Workload(
        name=f"iso{n}x{n}_{n_src}src_{len(freqs)}f_dbi", nz=n, nx=n, h=10.0, lz=2 * n, lx=2 * n,
        rho0=rho, alpha0=a, beta0=b, model=m_b, model_true=m_true,
        freqs_hz=np.asarray(freqs, dtype=np.float64),
        src_cells=np.stack([np.zeros_like(cols), cols], axis=1),
        src_force=np.tile([0.0, 1.0], (n_src, 1)),
        rec_cells=np.array([[0, j] for j in range(0, n, 2)]),
        krylov_tol=1e-6, seed=seed)


def config4_misfit(n=512, n_src=64, nf=6, seed=4) -> Workload:
    """VTI background as config 2, n x n cells, h = 5 m, n_src sources x nf frequencies 3-18 Hz,
    receivers on every 2nd column of the top row; true model = background x (1 + p) with p white
    noise smoothed by a Gaussian of 20 cells and scaled to max |p| = 10 % per parameter. The model
    handed to the misfit is the background; `model_true` made the observed data."""
    rng = np.random.default_rng(seed)
    m_bg = vti_background(n, n)
    rho0, a0, b0 = isotropic_reference_for(m_bg)
    corr = 20.0 * n / 512.0
    pert = np.empty((5, n, n))
    for p in range(5):
        w = _gauss_filter(rng.standard_normal((n, n)), corr)
        pert[p] = 0.10 * w / np.max(np.abs(w))
    cols = surface_line(n, n_src)
    return Workload(
        name=f"vti{n}x{n}_{n_src}src_{nf}f_misfit", nz=n, nx=n, h=5.0, lz=2 * n, lx=2 * n,
        rho0=rho0, alpha0=a0, beta0=b0, model=m_bg.copy(), model_true=m_bg * (1.0 + pert),
        freqs_hz=np.linspace(3.0, 18.0, nf),
        src_cells=np.stack([np.zeros_like(cols), cols], axis=1),
        src_force=np.tile([0.0, 1.0], (n_src, 1)),
        rec_cells=np.array([[0, j] for j in range(0, n, 2)]),
        krylov_tol=1e-6, seed=seed)


def config5_uneven(sizes=(64, 128, 256, 384, 512), n_members=40, max_src=32, max_f=8, f_range=(2.0, 25.0),
                   h=5.0, seed=5, radix3=True) -> list:
    """Uneven batch: n_members independent problems, each with a square grid drawn from `sizes`,
    1..max_src surface sources, 1..max_f frequencies drawn in f_range (sorted), an isotropic
    (rho 2000, alpha 2000, beta 1155) or VTI background (as config 2) and 1-4 Gaussian anomalies
    (sigma N/32 .. N/8 cells) of +/-15 % with a random sign per parameter. The FFT grid of each is
    the smallest complex64 length >= 2N - 1 (fft_len: 384 cells -> 768; with radix3=False the
    smallest power of two, 384 cells -> 1024)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_members):
        n = int(rng.choice(sizes))
        n_src = int(rng.integers(1, max_src + 1))
        nf = int(rng.integers(1, max_f + 1))
        freqs = np.sort(rng.uniform(f_range[0], f_range[1], nf))
        vti = bool(rng.integers(0, 2))
        if vti:
            m_bg = vti_background(n, n)
            rho0, a0, b0 = isotropic_reference_for(m_bg)
        else:
            rho0, a0, b0 = 2000.0, 2000.0, 1155.0
            m_bg = isotropic_model(n, n, rho0, a0, b0)
        count = int(rng.integers(1, 5))
        pert = _random_anomalies(rng, n, n, count, 0.15, (n / 32.0, n / 8.0))
        model = m_bg * (1.0 + np.clip(pert, -0.15, 0.15))
        cols = surface_line(n, n_src)
        L = fft_len(n, radix3)
        out.append(Workload(
            name=f"{'vti' if vti else 'iso'}{n}x{n}_{n_src}src_{nf}f", nz=n, nx=n, h=h, lz=L, lx=L,
            rho0=rho0, alpha0=a0, beta0=b0, model=model, freqs_hz=freqs,
            src_cells=np.stack([np.zeros_like(cols), cols], axis=1),
            src_force=np.tile([0.0, 1.0], (n_src, 1)),
            rec_cells=np.array([[0, j] for j in range(0, n, 2)]),
            krylov_tol=1e-5, seed=seed))
    return out


def fft_len(n: int, radix3: bool = False) -> int:
    """Smallest power of two >= max(16, 2n - 1): an FFT length that holds every offset of n cells.
    With radix3, 768 (= 3 x 256, a complex64 length of the library) when 512 < 2n - 1 <= 768."""
    p = 16
    while p < 2 * n - 1:
        p *= 2
    return 768 if radix3 and p == 1024 and 2 * n - 1 <= 768 else p


def small_case(nz=12, nx=10, h=10.0, seed=11, n_src=2, freqs=(8.0, 14.0), amp=0.1, vti=False,
               lz=None, lx=None) -> Workload:
    """A small, non-square case with a ragged contrast for parity and pin tests."""
    rng = np.random.default_rng(seed)
    if vti:
        m_bg = vti_background(nz, nx)
        rho0, a0, b0 = isotropic_reference_for(m_bg)
    else:
        rho0, a0, b0 = 2000.0, 2000.0, 1155.0
        m_bg = isotropic_model(nz, nx, rho0, a0, b0)
    pert = amp * (2.0 * rng.random((5, nz, nx)) - 1.0)
    model = m_bg * (1.0 + pert)
    cols = surface_line(nx, n_src)
    return Workload(
        name=f"small{nz}x{nx}", nz=nz, nx=nx, h=h,
        lz=lz if lz is not None else fft_len(nz), lx=lx if lx is not None else fft_len(nx),
        rho0=rho0, alpha0=a0, beta0=b0, model=model,
        freqs_hz=np.asarray(freqs, dtype=np.float64),
        src_cells=np.stack([np.zeros_like(cols), cols], axis=1),
        src_force=np.tile([0.3, 1.0], (n_src, 1)),
        rec_cells=np.array([[0, j] for j in range(0, nx, 2)] + [[nz - 1, 1]]),
        krylov_tol=1e-10, seed=seed)


def seeded_complex(shape, seed) -> np.ndarray:
    """Complex128 array with independent standard-normal real and imaginary parts."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def seeded_real(shape, seed) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape)


CONFIGS = {
    "c1": config1_tiny,
    "c2": config2_batched_forward,
    "c3": config3_linear_dbi,
    "c4": config4_misfit,
}


# ---------------------------------------------------------------------------------------------
# 3D workloads (the paper's 3D extension): fields [3][nz][ny][nx], models [6][nz][ny][nx] of
# (rho, C11, C13, C33, C55, C66); isotropic reference
# ---------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload3D:
    name: str
    nz: int
    ny: int
    nx: int
    h: float
    lz: int
    ly: int
    lx: int
    rho0: float
    alpha0: float
    beta0: float
    model: np.ndarray      # [6][nz][ny][nx]
    freqs_hz: np.ndarray
    src_cells: np.ndarray  # [n_src][3] (iz, iy, ix)
    src_force: np.ndarray  # [n_src][3]
    rec_cells: np.ndarray  # [n_rec][3]
    krylov_tol: float = 1e-5
    seed: int = 0

    @property
    def omegas(self) -> np.ndarray:
        return 2.0 * np.pi * np.asarray(self.freqs_hz, dtype=np.float64)

    @property
    def nf(self) -> int:
        return int(len(self.freqs_hz))

    @property
    def n_src(self) -> int:
        return int(self.src_cells.shape[0])

    @property
    def n_problems(self) -> int:
        return self.n_src * self.nf

    def problem_fidx(self) -> np.ndarray:
        return np.repeat(np.arange(self.nf, dtype=np.int32), self.n_src)

    def problem_src(self) -> np.ndarray:
        return np.tile(np.arange(self.n_src, dtype=np.int64), self.nf)


def vti_background_3d(nz, ny, nx, rho=2200.0, alpha_v=2500.0, eps_ratio=1.2, delta=0.1) -> np.ndarray:
    """The 2D VTI background extended along y with C66 = C55 (as the paper's modified 3D model)."""
    m2 = vti_background(1, 1, rho, alpha_v, eps_ratio, delta)
    vals = [float(m2[p, 0, 0]) for p in range(5)] + [float(m2[4, 0, 0])]
    return np.broadcast_to(np.asarray(vals)[:, None, None, None], (6, nz, ny, nx)).copy()


def _surface_grid(ny, nx, count):
    k = int(round(math.sqrt(count)))
    ys, xs = surface_line(ny, k), surface_line(nx, max(1, count // k))
    return np.array([[0, y, x] for y in ys for x in xs][:count], dtype=np.int64)


def small_case_3d(nz=4, ny=3, nx=5, h=10.0, seed=21, n_src=2, freqs=(8.0,), amp=0.1, lz=None, ly=None,
                  lx=None) -> Workload3D:
    """A small 3D case: isotropic reference (2000, 2000, 1155), the medium perturbed by +-amp per
    parameter and cell, vertical point forces on the surface."""
    rng = np.random.default_rng(seed)
    rho0, a0, b0 = 2000.0, 2000.0, 1155.0
    a2, b2 = a0 * a0, b0 * b0
    ref = np.array([rho0, rho0 * a2, rho0 * (a2 - 2 * b2), rho0 * a2, rho0 * b2, rho0 * b2])
    model = ref[:, None, None, None] * (1.0 + amp * (2.0 * rng.random((6, nz, ny, nx)) - 1.0))
    src = _surface_grid(ny, nx, n_src)
    return Workload3D(
        name=f"small3d_{nz}x{ny}x{nx}", nz=nz, ny=ny, nx=nx, h=h,
        lz=lz or fft_len(nz), ly=ly or fft_len(ny), lx=lx or fft_len(nx), rho0=rho0, alpha0=a0, beta0=b0,
        model=model, freqs_hz=np.asarray(freqs, dtype=np.float64), src_cells=src,
        src_force=np.tile([0.0, 0.3, 1.0], (len(src), 1)),
        rec_cells=np.array([[0, y, x] for y in range(0, ny, 2) for x in range(0, nx, 2)], dtype=np.int64),
        krylov_tol=1e-10, seed=seed)


def hess3d_like(nz=32, ny=40, nx=80, h=25.0, n_src=16, freqs=(3.0, 5.0, 7.0, 9.0), seed=6, n_rec=None) -> Workload3D:
    """The size of the paper's modified 3D VTI example (2000 m x 1000 m x 800 m at h = 25 m:
    80 x 40 x 32 cells): the VTI background extended along y (C66 = C55), three horizontal layers
    and four Gaussian anomalies of +-15 % per parameter; isotropic reference; vertical forces on a
    4 x 4 surface grid; receivers on every 2nd surface cell, or on an even surface grid of n_rec.
    (The paper's Hess model itself is not available.)"""
    rng = np.random.default_rng(seed)
    m_bg = vti_background_3d(nz, ny, nx)
    pert = np.zeros((6, nz, ny, nx))
    bounds = np.sort(rng.integers(nz // 5, nz, size=3))
    for k, z0 in enumerate(bounds):
        pert[:, z0:] += rng.uniform(-0.15, 0.15, size=(6, 1, 1, 1)) / (k + 1)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(4):
        c = rng.uniform([nz * 0.2, ny * 0.2, nx * 0.2], [nz * 0.8, ny * 0.8, nx * 0.8])
        sig = rng.uniform(3.0, 8.0)
        bump = np.exp(-((iz - c[0]) ** 2 + (iy - c[1]) ** 2 + (ix - c[2]) ** 2) / (2 * sig * sig))
        pert += rng.choice([-0.15, 0.15], size=(6, 1, 1, 1)) * bump
    model = m_bg * (1.0 + np.clip(pert, -0.15, 0.15))
    rho = float(m_bg[0, 0, 0, 0])
    a0 = math.sqrt(0.5 * (m_bg[1, 0, 0, 0] + m_bg[3, 0, 0, 0]) / rho)
    b0 = math.sqrt(m_bg[4, 0, 0, 0] / rho)
    src = _surface_grid(ny, nx, n_src)
    return Workload3D(
        name=f"hess3d_like_{nz}x{ny}x{nx}_{n_src}src_{len(freqs)}f", nz=nz, ny=ny, nx=nx, h=h,
        lz=fft_len(nz), ly=fft_len(ny), lx=fft_len(nx), rho0=rho, alpha0=a0, beta0=b0, model=model,
        freqs_hz=np.asarray(freqs, dtype=np.float64), src_cells=src,
        src_force=np.tile([0.0, 0.0, 1.0], (len(src), 1)),
        rec_cells=(np.array([[0, y, x] for y in range(0, ny, 2) for x in range(0, nx, 2)], dtype=np.int64)
                   if n_rec is None else _surface_grid(ny, nx, n_rec)),
        krylov_tol=1e-5, seed=seed)


def hess3d_paper_acquisition(seed=6) -> Workload3D:
    """The acquisition of the paper's 3D example on the hess3d_like model: 100 vertical forces on a
    10 x 10 surface grid, 400 receivers on a 20 x 20 surface grid, 7 frequencies 3-15 Hz (700
    wavefields; the DBI loop takes them one frequency, 100 wavefields, at a time)."""
    return hess3d_like(n_src=100, freqs=(3.0, 5.0, 7.0, 9.0, 11.0, 13.0, 15.0), seed=seed, n_rec=400)

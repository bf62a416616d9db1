"""Pins of the oracle's paper-literal form (Eq. 9: the derivative on the Green's tensor), CPU only.

The form is pinned by properties that do not retype its code: its direct sum equals its FFT
evaluation (the embedding of its nine tables); summation by parts makes it equal to the
divergence form of Eq. 6 exactly when the stress vanishes on the outer ring of D, and only then;
the derivative tables have the parities that the parities of G_11, G_13, G_33 imply, with x and z
in their places; and at explicit coordinates they are the central differences of the closed form.
"""
import numpy as np
import pytest

import oracle as O


def case(nz=9, nx=7, seed=5, ring_zero=False):
    rng = np.random.default_rng(seed)
    rho0, a0, b0 = 2000.0, 2000.0, 1155.0
    ref = O.reference_params(rho0, a0, b0)
    model = ref[:, None, None] * (1.0 + 0.1 * (2.0 * rng.random((5, nz, nx)) - 1.0))
    if ring_zero:
        for p in range(5):
            model[p, 0, :] = model[p, -1, :] = model[p, :, 0] = model[p, :, -1] = ref[p]
    u = rng.standard_normal((2, nz, nx)) + 1j * rng.standard_normal((2, nz, nx))
    return model, u, (rho0, a0, b0)


def oracle(nz, nx, h=10.0, lz=None, lx=None, freq=9.0):
    lz = lz or 2 * nz
    lx = lx or 2 * nx
    return O.LSOracle(nz, nx, h, lz, lx, 2000.0, 2000.0, 1155.0, [2 * np.pi * freq])


def test_direct_sum_equals_fft():
    nz, nx, h = 6, 5, 10.0
    w = 2 * np.pi * 11.0
    G = O.green_lattice(nz, nx, h, w, 2000.0, 1155.0, 2000.0)
    DG = O.green_derivative_lattice(nz, nx, h, w, 2000.0, 1155.0, 2000.0)
    rng = np.random.default_rng(1)
    src = rng.standard_normal((5, nz, nx)) + 1j * rng.standard_normal((5, nz, nx))
    direct = O.form_k_direct(src, G, DG, h)
    for lz, lx in ((2 * nz, 2 * nx), (16, 32)):
        fft = O.form_k_fft(src, O.form_k_spectra(G, DG, lz, lx), h)
        assert np.linalg.norm(fft - direct) <= 1e-12 * np.linalg.norm(direct)


def test_equals_divergence_form_when_the_stress_vanishes_on_the_ring():
    model, u, _ = case(ring_zero=True)
    orc = oracle(*u.shape[1:])
    a_k = orc.apply_k(u, model, 0)
    a_s = orc.apply(u, model, 0)
    assert np.linalg.norm(a_k - a_s) <= 1e-12 * np.linalg.norm(a_s - u)


def test_differs_from_divergence_form_when_the_contrast_reaches_the_boundary():
    model, u, _ = case(ring_zero=False)
    orc = oracle(*u.shape[1:])
    a_k = orc.apply_k(u, model, 0)
    a_s = orc.apply(u, model, 0)
    rel = np.linalg.norm(a_k - a_s) / np.linalg.norm(a_s - u)
    assert rel > 1e-3
    # the difference is the convolution of G with sources on the ring: a contrast confined to
    # the interior gives none (previous test), so removing the ring's stiffness contrast alone
    # removes the whole difference
    model_i = model.copy()
    ref = O.reference_params(2000.0, 2000.0, 1155.0)
    for p in range(1, 5):
        model_i[p, 0, :] = model_i[p, -1, :] = model_i[p, :, 0] = model_i[p, :, -1] = ref[p]
    assert np.linalg.norm(orc.apply_k(u, model_i, 0) - orc.apply(u, model_i, 0)) <= \
        1e-12 * np.linalg.norm(a_s - u)


def test_derivative_tables_have_the_parities_of_G():
    nz, nx, h, w = 7, 6, 10.0, 2 * np.pi * 7.0
    DG = O.green_derivative_lattice(nz, nx, h, w, 2000.0, 1155.0, 2000.0)
    fz = lambda a: a[::-1, :]   # dz -> -dz
    fx = lambda a: a[:, ::-1]   # dx -> -dx
    # G11, G33 are even in x and z, G13 odd in both; d/dx flips the x parity, d/dz the z parity
    parity = {0: (-1, +1), 1: (+1, -1), 2: (-1, +1),   # D1 G11, D1 G13, D1 G33: (x, z) parities
              3: (+1, -1), 4: (-1, +1), 5: (+1, -1)}   # D3 G11, D3 G13, D3 G33
    for k, (px, pz) in parity.items():
        t = DG[k]
        assert np.allclose(fx(t), px * t, rtol=1e-12, atol=1e-12 * np.abs(t).max()), k
        assert np.allclose(fz(t), pz * t, rtol=1e-12, atol=1e-12 * np.abs(t).max()), k


@pytest.mark.parametrize("dz,dx", [(3, -2), (-4, 5), (0, 3), (2, 0)])
def test_derivatives_are_central_differences_of_the_closed_form(dz, dx):
    nz, nx, h, w = 7, 7, 10.0, 2 * np.pi * 6.0
    a, b, rho = 2000.0, 1155.0, 2000.0
    DG = O.green_derivative_lattice(nz, nx, h, w, 2000.0, 1155.0, 2000.0)
    iz, ix = dz + nz - 1, dx + nx - 1
    g = lambda y1, y3: np.array(O.green_2d(np.array([y1]), np.array([y3]), w, a, b, rho))[:, 0]
    y1, y3 = dx * h, dz * h
    d1 = (g(y1 + h, y3) - g(y1 - h, y3)) / (2 * h)
    d3 = (g(y1, y3 + h) - g(y1, y3 - h)) / (2 * h)
    assert np.allclose(DG[0:3, iz, ix], d1, rtol=1e-12)
    assert np.allclose(DG[3:6, iz, ix], d3, rtol=1e-12)

"""Pins for the oracle's spectral operators (Sec. III-B1), CPU only.

Each check compares against a closed form: trigonometric polynomials with
|k_j| < N_j/2 are differentiated exactly by the Fourier method, single modes
are eigenfunctions of every diagonal operator, and the Leray projection has
the algebraic properties of an orthogonal projection onto divergence-free
fields.
"""

import numpy as np
import pytest

from oracle import spectral as sp
from oracle.problem import inner
from paper_1608_03630_gb300 import synth

SHAPE = (16, 20, 12)


def coords(shape=SHAPE):
    return synth.grid_coords(shape)


def test_fft_sign_convention_matches_naive_dft():
    # The multiplier i*k for d/dx assumes F[f](k) = sum f exp(-i k x).
    rng = np.random.default_rng(0)
    f = rng.standard_normal((4, 6, 5))
    naive = np.zeros(f.shape, dtype=complex)
    for k1 in range(4):
        for k2 in range(6):
            for k3 in range(5):
                s = 0.0
                for i1 in range(4):
                    for i2 in range(6):
                        for i3 in range(5):
                            s += f[i1, i2, i3] * np.exp(-2j * np.pi * (
                                k1 * i1 / 4 + k2 * i2 / 6 + k3 * i3 / 5))
                naive[k1, k2, k3] = s
    assert np.allclose(sp.fft(f), naive, atol=1e-12)


def test_gradient_exact_on_trig_polynomial():
    x1, x2, x3 = coords()
    f = np.sin(2 * x1) * np.cos(3 * x2) * np.sin(x3) + np.cos(5 * x3)
    g = sp.gradient(f)
    e1 = 2 * np.cos(2 * x1) * np.cos(3 * x2) * np.sin(x3)
    e2 = -3 * np.sin(2 * x1) * np.sin(3 * x2) * np.sin(x3)
    e3 = np.sin(2 * x1) * np.cos(3 * x2) * np.cos(x3) - 5 * np.sin(5 * x3)
    for got, exp in zip(g, (e1, e2, e3)):
        assert np.abs(got - exp).max() < 1e-12


def test_divergence_exact():
    x1, x2, x3 = coords()
    v = np.stack([np.sin(x1) * np.cos(x3), np.cos(2 * x2) * np.sin(x1), np.sin(3 * x3)])
    exp = np.cos(x1) * np.cos(x3) - 2 * np.sin(2 * x2) * np.sin(x1) + 3 * np.cos(3 * x3)
    assert np.abs(sp.divergence(v) - exp).max() < 1e-12


def test_nyquist_reading():
    # cos(N/2 x) is (-1)^i on the grid: the odd derivative is zero (k' = 0 at
    # the Nyquist entry), the even one keeps |k|^2 = (N/2)^2.
    x1, _, _ = coords()
    f = np.cos(SHAPE[0] // 2 * x1)
    assert np.abs(sp.gradient(f)).max() < 1e-12
    assert np.abs(sp.laplacian(f) + (SHAPE[0] // 2) ** 2 * f).max() < 1e-10


@pytest.mark.parametrize('kind,power', [('H2', 2), ('H1', 1), ('H1DIV', 1)])
def test_regularisation_symbol_on_modes(kind, power):
    x1, x2, x3 = coords()
    f = np.cos(2 * x1 + 3 * x2 - x3)
    v = np.stack([f, 2 * f, -f])
    av = sp.apply_regularisation(v, kind)
    assert np.abs(av - (4 + 9 + 1) ** power * v).max() < 1e-9


def test_laplacian_and_biharmonic():
    x1, x2, x3 = coords()
    f = np.sin(x1) * np.sin(2 * x2) + np.cos(4 * x3)
    lap = -(1 + 4) * np.sin(x1) * np.sin(2 * x2) - 16 * np.cos(4 * x3)
    assert np.abs(sp.laplacian(f) - lap).max() < 1e-11
    bih = sp.apply_symbol(f, sp.regularisation_symbol(SHAPE, 'H2'))
    assert np.abs(bih - (25 * np.sin(x1) * np.sin(2 * x2) + 256 * np.cos(4 * x3))).max() < 1e-9


def test_gaussian_on_single_mode():
    x1, x2, x3 = coords()
    f = np.cos(3 * x1 - 2 * x3)
    s = (0.3, 0.2, 0.5)
    exp = np.exp(-0.5 * ((0.3 * 3) ** 2 + (0.5 * 2) ** 2)) * f
    assert np.abs(sp.gaussian_smooth(f, s) - exp).max() < 1e-13


def test_leray_properties():
    x1, x2, x3 = coords()
    rng = np.random.default_rng(1)
    v = synth.bandlimited(SHAPE, 5, 11)
    w = synth.bandlimited(SHAPE, 5, 12)
    pv = sp.leray(v)
    # div P v = 0 exactly, P^2 = P, <P v, w> = <v, P w>
    assert np.abs(sp.divergence(pv)).max() < 1e-12
    assert np.abs(sp.leray(pv) - pv).max() < 1e-12
    assert abs(inner(pv, w) - inner(v, sp.leray(w))) < 1e-10 * abs(inner(v, w)) + 1e-12
    # gradients are annihilated, curls are kept
    phi = np.sin(x1 + 2 * x2) * np.cos(x3)
    assert np.abs(sp.leray(sp.gradient(phi))).max() < 1e-12
    a = np.stack([np.sin(2 * x2), np.cos(x3) * np.sin(x1), np.sin(x1 + x2)])
    ga = [sp.gradient(a[c]) for c in range(3)]  # ga[c][j] = d_j a_c
    curl = np.stack([ga[2][1] - ga[1][2], ga[0][2] - ga[2][0], ga[1][0] - ga[0][1]])
    assert np.abs(sp.leray(curl) - curl).max() < 1e-12
    del rng


def test_preconditioner_inverts_regularisation():
    v = synth.bandlimited(SHAPE, 6, 21)
    v = v - v.mean(axis=(1, 2, 3), keepdims=True)
    beta = 3e-3
    for kind in ('H2', 'H1'):
        av = beta * sp.apply_regularisation(v, kind)
        z = sp.preconditioner(av, beta, kind, incompressible=False)
        assert np.abs(z - v).max() < 1e-9
    # k = 0 reading: M(0) = 1/beta
    c = np.ones((3,) + SHAPE)
    assert np.allclose(sp.preconditioner(c, beta, 'H2', False), c / beta)
    # incompressible: z = M P r
    pv = sp.leray(v)
    z = sp.preconditioner(beta * sp.apply_regularisation(v, 'H2'), beta, 'H2', True)
    assert np.abs(z - pv).max() < 1e-9


def test_inner_product_is_the_l2_integral():
    x1, x2, x3 = coords()
    f = np.sin(x1) + np.cos(2 * x3)
    # int_{[0,2pi)^3} (sin x1 + cos 2x3)^2 = (2 pi)^3 (1/2 + 1/2)
    assert abs(inner(f, f) - (2 * np.pi) ** 3) < 1e-9


def test_resample_reproduces_band_limited_fields():
    """A trigonometric polynomial with modes |k| < min(N, M)/2 sampled on one
    grid and resampled equals its samples on the other (closed form); the
    Nyquist planes of the finer grid are dropped."""
    def field(shape):
        x1, x2, x3 = np.meshgrid(*[2 * np.pi * np.arange(n) / n for n in shape], indexing='ij')
        return (0.3 + np.sin(x1) * np.cos(2 * x2) + 0.5 * np.cos(3 * x3 - x1)
                + 0.25 * np.sin(x1 + x2 + x3))

    for a, b in (((8, 10, 12), (16, 12, 20)), ((16, 12, 20), (8, 10, 12)), ((9, 8, 8), (8, 8, 9))):
        assert np.abs(sp.resample(field(a), b) - field(b)).max() < 1e-12
    # a Nyquist mode of the 8-grid is not kept (8 -> 16: cos(4 x) is dropped)
    x = 2 * np.pi * np.arange(8) / 8
    f = np.cos(4 * x)[:, None, None] * np.ones((8, 8, 8))
    assert np.abs(sp.resample(f, (16, 16, 16))).max() < 1e-12
    # vector input
    v = np.stack([field((8, 8, 8)), 2 * field((8, 8, 8))])
    assert np.abs(sp.resample(v, (12, 12, 12))[1] - 2 * field((12, 12, 12))).max() < 1e-12

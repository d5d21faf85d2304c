"""Pins for the oracle's tricubic Lagrange interpolation (Sec. III-C2), CPU only."""

import os
from fractions import Fraction

import numpy as np

from oracle import interp as ip
from paper_1608_03630_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'lagrange_weights.txt')


def read_golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith('#'):
                continue
            rows.append([float(Fraction(t)) for t in line.split()])
    return np.array(rows)


def test_weights_match_textbook_values():
    g = read_golden()
    w = ip.lagrange_weights(g[:, 0])
    for j in range(4):
        assert np.abs(w[j] - g[:, 1 + j]).max() < 1e-15


def test_weights_match_polyfit_through_four_nodes():
    # the interpolant of node data y is the unique cubic through (n, y_n)
    rng = np.random.default_rng(3)
    for _ in range(5):
        y = rng.standard_normal(4)
        coef = np.polyfit([-1.0, 0.0, 1.0, 2.0], y, 3)
        xi = rng.uniform(0, 1, 7)
        w = ip.lagrange_weights(xi)
        got = sum(w[j] * y[j] for j in range(4))
        assert np.abs(got - np.polyval(coef, xi)).max() < 1e-12


def test_exact_on_tensor_cubics_away_from_the_wrap():
    shape = (12, 14, 16)
    i1, i2, i3 = [np.arange(n, dtype=float) for n in shape]
    p = lambda s: 0.3 - 0.2 * s + 0.05 * s * s - 0.004 * s ** 3
    q = lambda s: 1.0 + 0.1 * s - 0.02 * s ** 3 / 10
    r = lambda s: -0.5 + 0.03 * s * s + 0.001 * s ** 3
    f = p(i1)[:, None, None] * q(i2)[None, :, None] * r(i3)[None, None, :]
    rng = np.random.default_rng(4)
    pos = [rng.uniform(1.0, n - 3.0, 500) for n in shape]  # stencils inside
    got = ip.interp(f, pos)
    exp = p(pos[0]) * q(pos[1]) * r(pos[2])
    assert np.abs(got - exp).max() < 1e-11 * np.abs(exp).max()


def test_exact_at_nodes_with_wrap():
    shape = (9, 10, 11)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(shape)
    idx = [rng.integers(-40, 40, 300) for _ in range(3)]
    got = ip.interp(f, [i.astype(float) for i in idx])
    exp = f[np.mod(idx[0], 9), np.mod(idx[1], 10), np.mod(idx[2], 11)]
    assert np.abs(got - exp).max() < 1e-14


def test_constants_everywhere_including_wrap():
    f = np.full((7, 8, 9), 2.5)
    rng = np.random.default_rng(6)
    pos = [rng.uniform(-30, 30, 400) for _ in range(3)]
    assert np.abs(ip.interp(f, pos) - 2.5).max() < 1e-13


def test_periodicity_of_the_interpolant():
    shape = (8, 9, 10)
    f = np.random.default_rng(7).standard_normal(shape)
    rng = np.random.default_rng(8)
    pos = [rng.uniform(0, n, 200) for n in shape]
    shifted = [pos[0] + 3 * shape[0], pos[1] - 2 * shape[1], pos[2] + shape[2]]
    assert np.abs(ip.interp(f, pos) - ip.interp(f, shifted)).max() < 1e-12


def test_fourth_order_convergence_on_smooth_field():
    def field(x1, x2, x3):
        return np.sin(x1 + 2 * x2) * np.cos(x3) + np.exp(np.sin(x2 - x3)) * 0.3

    rng = np.random.default_rng(9)
    xs = [rng.uniform(0, 2 * np.pi, 3000) for _ in range(3)]
    errs = []
    for n in (32, 64, 128):
        shape = (n, n, n)
        f = field(*synth.grid_coords(shape))
        h = 2 * np.pi / n
        got = ip.interp(f, [x / h for x in xs])
        errs.append(np.abs(got - field(*xs)).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) >= 3.8, (errs, rates)

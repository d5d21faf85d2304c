"""Pins for the oracle's semi-Lagrangian transport (Sec. III-B2), CPU only.

Closed forms: the exact characteristic foot of v = (s sin x1, 0, 0), the
analytic solution of a shear flow, the identity map for v = 0, conservation
of constants.  Invariants of the continuous equations that the discretisation
must approach under refinement: d/dt <lam, rho> = 0 for the state/adjoint pair
(so a wrong source sign or direction in the adjoint fails), int lam dt
conservation, and det grad y = 1 for a divergence-free velocity.
"""

import numpy as np
import pytest

from oracle import spectral as sp
from oracle import transport as tr
from oracle.problem import inner
from paper_1608_03630_gb300 import synth


def test_departure_zero_and_constant_velocity():
    shape = (8, 10, 12)
    d = tr.departure(np.zeros((3,) + shape), 0.25)
    assert np.abs(d).max() == 0.0
    c = np.array([0.7, -1.3, 2.9])
    v = np.ones((3,) + shape) * c[:, None, None, None]
    d = tr.departure(v, 0.25)
    h = tr.grid_spacing(shape)
    for j in range(3):
        assert np.abs(d[j] + 0.25 * c[j] / h[j]).max() < 1e-12


def test_departure_shear_is_exact():
    shape = (16, 24, 8)
    x1, x2, x3 = synth.grid_coords(shape)
    s = 1.7
    v = np.stack([s * np.sin(x2), 0 * x1, 0 * x1])
    d = tr.departure(v, 0.5)
    h = tr.grid_spacing(shape)
    assert np.abs(d[0] + 0.5 * s * np.sin(x2) / h[0]).max() < 1e-12
    assert np.abs(d[1]).max() == 0.0 and np.abs(d[2]).max() == 0.0


def test_departure_is_second_order_rk():
    # v = (s sin x1, 0, 0): the foot of the characteristic through x after a
    # time dt backward is X = 2 atan2(sin(x/2) e^{-s dt}, cos(x/2)).
    shape = (256, 4, 4)
    x1, _, _ = synth.grid_coords(shape)
    s = 1.0
    v = np.stack([s * np.sin(x1), 0 * x1, 0 * x1])
    h = tr.grid_spacing(shape)[0]
    errs = []
    for dt in (0.2, 0.1, 0.05):
        d = tr.departure(v, dt)
        exact = 2.0 * np.arctan2(np.sin(x1 / 2) * np.exp(-s * dt), np.cos(x1 / 2))
        errs.append(np.abs(x1 + h * d[0] - exact).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert min(ratios) > 6.5, (errs, ratios)  # third-order local error


def test_zero_velocity_is_identity():
    shape = (8, 9, 10)
    rng = np.random.default_rng(1)
    rho0 = rng.standard_normal(shape)
    d = tr.departure(np.zeros((3,) + shape), 0.25)
    rho = tr.state_solve(rho0, d, 4)
    assert all(np.array_equal(r, rho0) for r in rho)
    lam = tr.adjoint_solve(rho0, d, np.zeros(shape), 4)
    assert all(np.abs(l - rho0).max() < 1e-15 for l in lam)


def test_constants_are_transported_unchanged():
    shape = (12, 12, 12)
    v = 0.8 * synth.bandlimited(shape, 3, 5)
    d = tr.departure(v, 0.25)
    rho = tr.state_solve(np.full(shape, 1.25), d, 4)
    assert np.abs(rho[-1] - 1.25).max() < 1e-13


def test_shear_flow_analytic_solution_fourth_order():
    s = 0.9
    f = lambda a, b, c: np.sin(a) * np.cos(c) + 0.5 * np.cos(2 * a + b)
    errs = []
    for n in (16, 32, 64):
        shape = (n, n, 8)
        x1, x2, x3 = synth.grid_coords(shape)
        v = np.stack([s * np.sin(x2), 0 * x1, 0 * x1])
        d = tr.departure(v, 0.25)
        rho = tr.state_solve(f(x1, x2, x3), d, 4)
        errs.append(np.abs(rho[-1] - f(x1 - s * np.sin(x2), x2, x3)).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 3.5, (errs, rates)


def _duality_drift(n, nt=4):
    shape = (n, n, n)
    v = 0.6 * synth.bandlimited(shape, 2, 7)
    rho0 = synth.bandlimited(shape, 3, 8, ncomp=None)
    lam1 = synth.bandlimited(shape, 3, 9, ncomp=None)
    d_fwd = tr.departure(v, 1.0 / nt)
    d_adj = tr.departure(-v, 1.0 / nt)
    divv = sp.divergence(v)
    rho = tr.state_solve(rho0, d_fwd, nt)
    lam = tr.adjoint_solve(lam1, d_adj, divv, nt)
    pairs = [inner(lam[j], rho[j]) for j in range(nt + 1)]
    mass = [inner(lam[j], np.ones(shape)) for j in range(nt + 1)]
    scale = np.sqrt(inner(lam1, lam1) * inner(rho0, rho0))
    return (max(abs(p - pairs[-1]) for p in pairs) / scale,
            max(abs(m - mass[-1]) for m in mass) / scale)


def test_adjoint_is_dual_to_the_state():
    # d/dt <lam, rho> = 0 and d/dt int lam = 0 for the continuous pair; the
    # discrete drift is small and the mass drift is second order in dt.
    dual4, mass4 = _duality_drift(32, 4)
    dual8, mass8 = _duality_drift(32, 8)
    assert max(dual4, mass4, dual8, mass8) < 5e-3, (dual4, mass4, dual8, mass8)
    assert mass8 < mass4 / 3.0, (mass4, mass8)


def test_duality_pin_catches_a_wrong_adjoint_source_sign(monkeypatch):
    good, _ = _duality_drift(16)
    orig = tr.adjoint_step

    def flipped(nu, d_adj, divv, dt):
        return orig(nu, d_adj, None if divv is None else -divv, dt)

    monkeypatch.setattr(tr, 'adjoint_step', flipped)
    bad, _ = _duality_drift(16)
    assert bad > 20 * good, (good, bad)


def test_incremental_state_is_the_linearised_state():
    # rho~(1) approaches the directional derivative of rho(1) under refinement
    # (optimise-then-discretise: equal only up to discretisation error).
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        v = 0.5 * synth.bandlimited(shape, 2, 17)
        vt = synth.bandlimited(shape, 2, 18)
        rho0 = synth.bandlimited(shape, 3, 19, ncomp=None)
        nt = 4
        d = tr.departure(v, 1.0 / nt)
        rho = tr.state_solve(rho0, d, nt)
        grad_rho = [sp.gradient(r) for r in rho]
        rt = tr.incremental_state_solve(vt, grad_rho, d, nt)[-1]
        eps = 1e-5
        rp = tr.state_solve(rho0, tr.departure(v + eps * vt, 1.0 / nt), nt)[-1]
        rm = tr.state_solve(rho0, tr.departure(v - eps * vt, 1.0 / nt), nt)[-1]
        fd = (rp - rm) / (2 * eps)
        errs.append(np.sqrt(inner(rt - fd, rt - fd) / inner(fd, fd)))
    assert errs[1] < 0.05 and errs[1] < errs[0], errs


@pytest.mark.slow
def test_divergence_free_velocity_preserves_volume():
    shape = (64, 64, 64)
    v = synth.vstar(shape, 0.5)
    assert np.abs(sp.divergence(v)).max() < 1e-12
    d = tr.departure(v, 0.25)
    u = tr.deformation_displacement(v, d, 4)
    det = tr.jacobian_determinant(u)
    assert np.abs(det - 1.0).max() < 1e-2, np.abs(det - 1).max()


def test_compressible_map_has_unit_mean_jacobian():
    # a periodic diffeomorphism maps the torus onto itself: mean det = 1,
    # while the pointwise det departs from 1 by O(div v).
    shape = (24, 24, 24)
    v = 0.4 * synth.bandlimited(shape, 2, 27)
    d = tr.departure(v, 0.25)
    det = tr.jacobian_determinant(tr.deformation_displacement(v, d, 4))
    assert abs(det.mean() - 1.0) < 1e-3
    assert np.abs(det - 1.0).max() > 0.05
    assert det.min() > 0.0

"""Pins for the oracle's objective, gradient, GN Hessian and solver, CPU only.

Closed forms at v = 0 (Sec. II-B): rho(t) = rho_T, lam = rho_R - rho_T, so
g(0) = P[(rho_R - rho_T) grad rho_T]; rho~(t) = -t v~.grad rho_T, lam~ =
v~.grad rho_T, so H(0) v~ = beta A v~ + P[(v~.grad rho_T) grad rho_T] -- exact
for the discrete scheme too (on-grid points, trapezoid exact for constants).
At v != 0 the optimise-then-discretise gradient and Hessian agree with
finite differences and with symmetry only up to discretisation error, which
must shrink under refinement.  PCG is checked against a dense solve.
"""

import numpy as np
import pytest

from oracle import problem as pr
from oracle import solver as so
from oracle import spectral as sp
from oracle import transport as tr
from paper_1608_03630_gb300 import synth


def smooth_pair(shape, seed=31):
    rho_T = synth.bandlimited(shape, 3, seed, ncomp=None)
    rho_R = synth.bandlimited(shape, 3, seed + 1, ncomp=None)
    return rho_T, rho_R


@pytest.mark.parametrize('incompressible', [False, True])
def test_gradient_at_zero_closed_form(incompressible):
    shape = (16, 18, 20)
    rho_T, rho_R = smooth_pair(shape)
    P = pr.Problem(rho_T, rho_R, 4, 1e-2, 'H2', incompressible)
    g, J = P.gradient(np.zeros((3,) + shape))
    b = (rho_R - rho_T) * sp.gradient(rho_T)
    exp = sp.leray(b) if incompressible else b
    assert np.abs(g - exp).max() < 1e-12 * np.abs(exp).max()
    r = rho_T - rho_R
    assert abs(J - 0.5 * pr.inner(r, r)) < 1e-14 * J


@pytest.mark.parametrize('kind,incompressible', [('H2', False), ('H1DIV', True)])
def test_hessian_at_zero_closed_form(kind, incompressible):
    shape = (16, 18, 20)
    rho_T, rho_R = smooth_pair(shape)
    beta = 3e-3
    P = pr.Problem(rho_T, rho_R, 4, beta, kind, incompressible)
    P.gradient(np.zeros((3,) + shape))
    w = synth.bandlimited(shape, 6, 41)
    if incompressible:
        w = sp.leray(w)
    gr = sp.gradient(rho_T)
    exp = beta * sp.apply_regularisation(w, kind) + P.project(np.sum(w * gr, 0) * gr)
    got = P.hessian_matvec(w)
    assert np.abs(got - exp).max() < 1e-12 * np.abs(exp).max()
    assert pr.inner(w, got) > 0.0


def _fd_gradient_error(n, seed=51):
    shape = (n, n, n)
    rho_T, rho_R = smooth_pair(shape, seed)
    P = pr.Problem(rho_T, rho_R, 4, 1e-2, 'H2', False)
    v = 0.4 * synth.bandlimited(shape, 2, seed + 2)
    w = synth.bandlimited(shape, 2, seed + 3)
    g, _ = P.gradient(v)
    eps = 1e-4
    fd = (P.objective(v + eps * w) - P.objective(v - eps * w)) / (2 * eps)
    return abs(pr.inner(g, w) - fd) / abs(fd)


def test_gradient_matches_finite_differences():
    e16 = _fd_gradient_error(16)
    e32 = _fd_gradient_error(32)
    assert e32 < 5e-2 and e32 < e16, (e16, e32)


def _asymmetry(n, nt, seed=61):
    shape = (n, n, n)
    rho_T, rho_R = smooth_pair(shape, seed)
    P = pr.Problem(rho_T, rho_R, nt, 1e-3, 'H2', False)
    P.gradient(0.4 * synth.bandlimited(shape, 2, seed + 2))
    a = synth.bandlimited(shape, 3, seed + 3)
    b = synth.bandlimited(shape, 3, seed + 4)
    ha, hb = P.hessian_matvec(a), P.hessian_matvec(b)
    return abs(pr.inner(ha, b) - pr.inner(a, hb)) / np.sqrt(pr.inner(ha, ha) * pr.inner(b, b))


def test_hessian_symmetric_up_to_discretisation():
    a16 = _asymmetry(16, 4)
    a32 = _asymmetry(32, 8)
    assert a16 < 1e-2 and a32 < a16 / 2, (a16, a32)


def test_hessian_energy_identity():
    # <v~, H v~> = beta <v~, A v~> + ||rho~(1)||^2 for the continuous GN Hessian
    shape = (32, 32, 32)
    rho_T, rho_R = smooth_pair(shape, 71)
    P = pr.Problem(rho_T, rho_R, 4, 1e-3, 'H2', False)
    P.gradient(0.4 * synth.bandlimited(shape, 2, 73))
    w = synth.bandlimited(shape, 3, 74)
    lhs = pr.inner(w, P.hessian_matvec(w))
    rt = P.incremental_state(w)[-1]
    rhs = 1e-3 * pr.inner(w, sp.apply_regularisation(w, 'H2')) + pr.inner(rt, rt)
    assert abs(lhs - rhs) < 2e-2 * rhs, (lhs, rhs)


def test_incompressible_gradient_is_divergence_free():
    shape = (16, 16, 16)
    rho_T, rho_R = smooth_pair(shape, 81)
    P = pr.Problem(rho_T, rho_R, 4, 1e-3, 'H1DIV', True)
    g, _ = P.gradient(sp.leray(0.4 * synth.bandlimited(shape, 2, 83)))
    assert np.abs(sp.divergence(g)).max() < 1e-12 * np.abs(g).max()


def test_pcg_matches_a_dense_solve():
    rng = np.random.default_rng(5)
    shape = (3, 2, 2, 2)
    m = rng.standard_normal((24, 24))
    a = m @ m.T + 24 * np.eye(24)
    d = np.diag(a).copy()
    rhs = rng.standard_normal(shape)
    mv = lambda x: (a @ x.ravel()).reshape(shape)
    pc = lambda x: (x.ravel() / d).reshape(shape)
    s, its, flag = so.pcg(mv, pc, rhs, 1e-12, 200)
    assert flag == 'converged'
    assert np.abs(s.ravel() - np.linalg.solve(a, rhs.ravel())).max() < 1e-9


def test_gauss_newton_on_the_sinusoid_problem():
    shape = (32, 32, 32)
    rho_T, rho_R, _ = synth.sinusoid_problem(shape, 0.5)
    P = pr.Problem(rho_T, rho_R, 4, 1e-2, 'H2', False)
    v, st = so.gauss_newton(P, np.zeros((3,) + shape), gtol=1e-2, max_gn=3)
    J = [h[0] for h in st['history']]
    assert all(J[i + 1] < J[i] for i in range(len(J) - 1))
    assert st['gnorm_rel'] < 1e-2
    assert st['mismatch_rel'] < 1.0


def test_sinusoid_problem_is_consistent_with_the_transport():
    # rho_T is rho_R moved back along the flow of v*; the discrete forward
    # solve with v* must bring it back to rho_R up to discretisation error.
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        rho_T, rho_R, vs = synth.sinusoid_problem(shape, 0.5)
        nt = 8
        rho = tr.state_solve(rho_T, tr.departure(vs, 1.0 / nt), nt)
        errs.append(np.abs(rho[-1] - rho_R).max())
    assert errs[1] < 2e-3 and errs[1] < errs[0], errs


def test_closed_form_pin_catches_wrong_quadrature_weights(monkeypatch):
    # plant a mistake in the oracle: rectangle weights dt on all nt+1 levels
    shape = (12, 12, 12)
    rho_T, rho_R = smooth_pair(shape)
    monkeypatch.setattr(tr, 'trapezoid_weights', lambda nt: np.full(nt + 1, 1.0 / nt))
    P = pr.Problem(rho_T, rho_R, 4, 1e-2, 'H2', False)
    g, _ = P.gradient(np.zeros((3,) + shape))
    b = (rho_R - rho_T) * sp.gradient(rho_T)
    assert np.abs(g - b).max() > 0.1 * np.abs(b).max()


def test_fd_pin_catches_a_wrong_adjoint_final_condition(monkeypatch):
    # plant a mistake in the oracle: lam(1) = rho(1) - rho_R
    orig = tr.adjoint_solve
    monkeypatch.setattr(tr, 'adjoint_solve',
                        lambda lam1, d, divv, nt: orig(-lam1, d, divv, nt))
    assert _fd_gradient_error(16) > 0.5

"""Pins for the oracle's full Newton Hessian (Eq. (hessian) with the terms in
lam kept), CPU only.

Closed form at v = 0 (Sec. II-B): rho = rho_T, lam = r := rho_R - rho_T (both
constant in time), rho~(t) = -t a with a = v~.grad rho_T, and the incremental
adjoint -d_t lam~ = div(r v~) with lam~(1) = a gives
lam~(t) = a + (1 - t) div(r v~).  Then
    b~ = int_0^1 (lam~ grad rho_T + r grad rho~) dt
       = a grad rho_T + 1/2 div(r v~) grad rho_T - 1/2 r grad a,
and H(0) v~ = beta A v~ + P b~.  The discrete scheme reproduces it exactly:
at v = 0 the semi-Lagrangian points are the grid points, the predictor-
corrector is exact for sources constant in time, and the trapezoid rule is
exact for integrands linear in t.  The same closed form is symmetric in
(v~, w) (integrate div by parts), so H(0) is symmetric to rounding.

At v != 0 the full Newton Hessian is the derivative of the gradient: central
finite differences of the oracle's gradient must agree with the full Newton
matvec up to discretisation error, which shrinks under refinement, while the
Gauss-Newton matvec, which drops the lam terms, stays off by those terms.
"""

import numpy as np
import pytest

from oracle import problem as pr
from oracle import spectral as sp
from paper_1608_03630_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _zero_point(kind, incompressible, shape=(16, 20, 24), beta=1e-2):
    rho_T = synth.bandlimited(shape, 3, 61, ncomp=None)
    rho_R = synth.bandlimited(shape, 3, 62, ncomp=None)
    P = pr.Problem(rho_T, rho_R, 4, beta, kind, incompressible, newton=True)
    P.gradient(np.zeros((3,) + shape))
    return P, rho_T, rho_R


def _closed_form(P, rho_T, rho_R, w):
    gr = sp.gradient(rho_T)
    r = rho_R - rho_T
    a = np.sum(w * gr, 0)
    bt = a * gr + 0.5 * sp.divergence(r * w) * gr - 0.5 * r * sp.gradient(a)
    return P.beta * P.regularisation(w) + P.project(bt)


@pytest.mark.parametrize('kind,incompressible', [('H2', False), ('H1DIV', True)])
def test_full_newton_hessian_at_zero_closed_form(kind, incompressible):
    P, rho_T, rho_R = _zero_point(kind, incompressible)
    w = synth.bandlimited(P.shape, 4, 63)
    if incompressible:
        w = sp.leray(w)
    got = P.hessian_matvec(w)
    exp = _closed_form(P, rho_T, rho_R, w)
    assert rel(got, exp) < 1e-12
    # the lam terms are of the size of the Gauss-Newton part here
    assert rel(P.hessian_matvec(w, full=False), got) > 0.1


def test_full_newton_hessian_at_zero_is_symmetric():
    P, _, _ = _zero_point('H2', False)
    w1 = synth.bandlimited(P.shape, 4, 63)
    w2 = synth.bandlimited(P.shape, 4, 64)
    a = pr.inner(P.hessian_matvec(w1), w2)
    b = pr.inner(w1, P.hessian_matvec(w2))
    assert abs(a - b) < 1e-12 * abs(a)


def _fd_errors(n, nt, beta=1e-3, eps=1e-4):
    """Relative errors of the full and the Gauss-Newton data term against
    central differences of the gradient, at v = 0.3 v* of the sinusoid
    problem (beta A w, exact on both sides, removed)."""
    shape = (n, n, n)
    rho_T, rho_R, vs = synth.sinusoid_problem(shape, 0.5)
    P = pr.Problem(rho_T, rho_R, nt, beta, 'H2', False)
    v = 0.3 * vs
    w = synth.bandlimited(shape, 2, 71)
    P.gradient(v)
    hf = P.hessian_matvec(w, full=True)
    hg = P.hessian_matvec(w, full=False)
    gp, _ = P.gradient(v + eps * w)
    gm, _ = P.gradient(v - eps * w)
    bA = beta * P.regularisation(w)
    fd = (gp - gm) / (2 * eps) - bA
    return rel(hf - bA, fd), rel(hg - bA, fd)


def test_full_newton_hessian_matches_finite_differences_of_the_gradient():
    f16, g16 = _fd_errors(16, 4)
    f32, g32 = _fd_errors(32, 8)
    assert f16 < 0.05 and f32 < 0.01          # measured 3.3e-2, 4.5e-3
    assert f32 < f16 / 3                       # discretisation error shrinks
    assert g16 > 3 * f16 and g32 > 10 * f32   # GN drops the lam terms


def test_closed_form_pin_catches_a_wrong_sign_of_the_lam_source(monkeypatch):
    """A mistake planted in the oracle: the incremental adjoint's source
    div(lam v~) with the wrong sign must fail the closed-form pin."""
    P, rho_T, rho_R = _zero_point('H2', False)
    w = synth.bandlimited(P.shape, 4, 63)
    exp = _closed_form(P, rho_T, rho_R, w)
    real_div = pr._sp.divergence
    monkeypatch.setattr(pr._sp, 'divergence', lambda v: -real_div(v))
    assert rel(P.hessian_matvec(w), exp) > 1e-2

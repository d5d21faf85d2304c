"""Pins of the oracle's two-level preconditioner and flexible PCG, CPU only.

* Restriction to a coarse grid keeps the Fourier modes |k_j| < n_c/2: a
  trigonometric polynomial inside that band restricts to its own samples on
  the coarse grid, and prolongation returns it exactly; equal grids are the
  identity.
* Without a data term (rho_T = rho_R constant, so grad rho = 0) the Hessian
  is beta A on both grids, the inner PCG with (beta A)^-1 converges in one
  step, and M^-1 r = (beta A)^-1 P r in closed form.
* With the coarse grid equal to the fine one and an exact inner solve the
  preconditioner is H^-1: at v = 0 (where the Gauss-Newton Hessian is exactly
  symmetric) flexible PCG then takes one iteration to the exact Newton step.
* Flexible PCG with a fixed SPD preconditioner makes the same iterates as
  PCG (the two direction coefficients agree in exact arithmetic).
* A coarse Hessian with its own time steps (nt_c): with an exact inner solve
  at v = 0 the operator is symmetric, and it equals the coarse correction
  assembled by hand from a coarse problem with nt_c steps.
"""

import numpy as np

from oracle import precond as opc
from oracle import problem as opr
from oracle import solver as oso
from oracle import spectral as osp
from paper_1608_03630_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def zero_mean(r):
    """Without a data term the Hessian beta A vanishes on constants, so the
    test residuals carry no k = 0 mode."""
    return r - r.mean(axis=(1, 2, 3), keepdims=True)


def trig(shape):
    x = synth.grid_coords(shape)
    return np.sin(2 * x[0]) * np.cos(3 * x[1]) + np.cos(x[2]) - 0.5 * np.sin(x[0] + 2 * x[2])


def test_restriction_samples_band_limited_fields_and_prolongation_inverts_it():
    fine, coarse = (32, 24, 20), (16, 12, 10)
    f = trig(fine)
    fc = opc.restrict(f, coarse)
    assert np.abs(fc - trig(coarse)).max() < 1e-12
    assert np.abs(opc.prolong(fc, fine) - f).max() < 1e-12
    assert np.abs(opc.restrict(f, fine) - f).max() < 1e-13
    # a mode outside the coarse band is removed
    x = synth.grid_coords(fine)
    g = np.cos(9 * x[0])
    assert np.abs(opc.restrict(g, coarse)).max() < 1e-12
    assert np.abs(opc.low_pass(f + g, coarse) - f).max() < 1e-12


def test_without_a_data_term_the_preconditioner_is_the_inverse_regularisation():
    shape, beta = (16, 16, 16), 1e-2
    for kind, inc in (('H2', False), ('H1DIV', True)):
        const = np.full(shape, 0.3)
        P = opr.Problem(const, const, 4, beta, kind, inc)
        T = opc.TwoLevel(P, (8, 8, 8), inner_tol=1e-12, inner_max=20)
        v = 0.2 * synth.bandlimited(shape, 2, 5)
        P.gradient(P.project(v))
        T.linearize(P.project(v))
        r = zero_mean(synth.bandlimited(shape, 6, 6))
        z = T.apply(r)
        assert rel(z, osp.preconditioner(r, beta, kind, inc)) < 1e-12, kind


def test_coarse_equal_to_fine_with_an_exact_inner_solve_inverts_the_hessian():
    shape = (16, 16, 16)
    rho_T = synth.bandlimited(shape, 3, 61, ncomp=None)
    rho_R = synth.bandlimited(shape, 3, 62, ncomp=None)
    P = opr.Problem(rho_T, rho_R, 4, 1e-3, 'H2', False)
    TP = opc.TwoLevelProblem(P, shape, inner_tol=1e-11, inner_max=400)
    g, _ = TP.gradient(np.zeros((3,) + shape))
    s, its, flag = oso.fpcg(P.hessian_matvec, TP.precond, -g, 1e-8 * np.sqrt(opr.inner(g, g)),
                            10)
    assert its == 1 and flag == 'converged'
    assert rel(P.hessian_matvec(s), -g) < 1e-8
    # the one-level preconditioner needs many iterations for the same system
    _, its1, _ = oso.pcg(P.hessian_matvec, P.precond, -g, 1e-8 * np.sqrt(opr.inner(g, g)), 400)
    assert its1 > 10


def test_flexible_pcg_equals_pcg_for_a_fixed_preconditioner():
    rng = np.random.default_rng(4)
    shape = (3, 4, 4, 4)
    n = int(np.prod(shape))
    m = rng.standard_normal((n, n))
    A = m @ m.T / n + 0.1 * np.eye(n)
    d = np.diag(A).reshape(shape)
    b = rng.standard_normal(shape)
    mv = lambda x: (A @ x.ravel()).reshape(shape)
    pc = lambda r: r / d
    s1, i1, f1 = oso.pcg(mv, pc, b, 1e-10, 200)
    s2, i2, f2 = oso.fpcg(mv, pc, b, 1e-10, 200)
    assert i1 == i2 and f1 == f2 == 'converged'
    assert np.abs(s1 - s2).max() < 1e-8 * np.abs(s1).max()


def test_closed_form_pin_catches_a_dropped_high_mode_part(monkeypatch):
    """A mistake planted in the oracle: the modes outside the coarse band
    left unpreconditioned must fail the no-data-term closed form."""
    shape, beta = (16, 16, 16), 1e-2
    const = np.full(shape, 0.3)
    P = opr.Problem(const, const, 4, beta, 'H2', False)
    T = opc.TwoLevel(P, (8, 8, 8), inner_tol=1e-12, inner_max=20)
    P.gradient(np.zeros((3,) + shape))
    T.linearize(np.zeros((3,) + shape))
    r = zero_mean(synth.bandlimited(shape, 6, 6))
    expected = osp.preconditioner(r, beta, 'H2', False)
    monkeypatch.setattr(opc._sp, 'preconditioner', lambda rr, *a: 0.0 * rr)
    assert rel(T.apply(r), expected) > 1e-2


def test_coarse_time_steps_give_a_symmetric_operator_built_from_that_coarse_problem():
    """At v = 0 the state does not move and the Gauss-Newton Hessian does not
    depend on the number of steps (its time integrand is linear in t, which
    the trapezoid rule integrates exactly), so there the operator must be
    symmetric; away from v = 0 it must equal the coarse correction assembled
    by hand from a coarse problem with nt_c steps, and differ from the one
    with the fine number of steps."""
    shape, coarse, beta = (16, 16, 16), (8, 8, 8), 1e-3
    rho_T = synth.bandlimited(shape, 3, 71, ncomp=None)
    rho_R = synth.bandlimited(shape, 3, 72, ncomp=None)
    P = opr.Problem(rho_T, rho_R, 4, beta, 'H2', False)
    a = synth.bandlimited(shape, 5, 73)
    b = synth.bandlimited(shape, 5, 74)
    zero = np.zeros((3,) + shape)
    P.gradient(zero)
    T2 = opc.TwoLevel(P, coarse, inner_tol=1e-12, inner_max=300, nt_c=2)
    T2.linearize(zero)
    assert T2.coarse.nt == 2
    ma, mb = T2.apply(a), T2.apply(b)
    # symmetric up to the inner solve's error (residual 1e-12 relative, times
    # the coarse Hessian's condition number, about 1e4 at beta = 1e-3)
    assert abs(opr.inner(ma, b) - opr.inner(a, mb)) < 1e-6 * abs(opr.inner(ma, b))
    # away from v = 0: the same correction from a coarse problem with two
    # steps, by hand
    v = 0.8 * synth.bandlimited(shape, 2, 75)
    P.gradient(v)
    T2.linearize(v)
    ma = T2.apply(a)
    C = opr.Problem(opc.restrict(rho_T, coarse), opc.restrict(rho_R, coarse), 2, beta, 'H2',
                    False)
    C.gradient(opc.restrict(v, coarse))
    rl = opc.restrict(a, coarse)
    y, _, _ = oso.pcg(C.hessian_matvec, C.precond, rl, 1e-12 * np.sqrt(opr.inner(rl, rl)), 300)
    expected = opc.prolong(y, shape) + osp.preconditioner(a - opc.low_pass(a, coarse), beta, 'H2',
                                                          False)
    assert rel(ma, expected) < 1e-9
    # and it differs from the operator with the fine number of steps
    T4 = opc.TwoLevel(P, coarse, inner_tol=1e-12, inner_max=300)
    T4.linearize(v)
    assert rel(T4.apply(a), ma) > 1e-4

"""Pins of the oracle's inexact Gauss-Newton-Krylov loop (Sec. III-A) on
model objectives whose behaviour is known in closed form.

* Convex quadratic J(v) = 1/2 <v, A v> - <b, v> with the exact Hessian A:
  after a PCG step s with residual r = -g - A s, the new gradient is
  g + A s = -r exactly, so the quadratic forcing term fixes the decrease:
  ||g_{k+1}|| <= min(1/2, ||g_k|| / ||g_0||) ||g_k||, and the full step
  always passes the Armijo test (J(v + s) - J(v) = <g, s> + 1/2 <s, A s>
  <= 1/2 <g, s> < c <g, s> for a CG step, c = 1e-4).
* Pseudo-Huber J(v) = sum sqrt(1 + v^2) h^3 (curvature at most 1) with a
  model Hessian that is too flat (0.1 I): the full step -10 g overshoots
  the minimum at 0, so the line search must halve it until sufficient
  decrease holds.
"""

import numpy as np

from oracle import problem as opr
from oracle import solver as so

SHAPE = (3, 4, 4, 4)
H3 = (2 * np.pi) ** 3 / 64.0   # cell volume of the 4^3 grid in the inner product


class Quadratic:
    def __init__(self, seed):
        rng = np.random.default_rng(seed)
        n = int(np.prod(SHAPE))
        m = rng.standard_normal((n, n))
        # SPD in the <.,.>_h metric: A = (M M^T / n + I) acting on the raw vector
        self.A = m @ m.T / n + np.eye(n)
        self.b = rng.standard_normal(SHAPE)
        self.rho_T = np.zeros(SHAPE[1:])
        self.rho_R = np.ones(SHAPE[1:])
        self.lin = {'rho': [self.rho_R]}

    def project(self, v):
        return v

    def apply(self, v):
        return (self.A @ v.ravel()).reshape(SHAPE)

    def objective(self, v):
        return 0.5 * opr.inner(v, self.apply(v)) - opr.inner(self.b, v)

    def gradient(self, v):
        # Riesz representative in <.,.>_h: grad J = A v - b
        return self.apply(v) - self.b, self.objective(v)

    def hessian_matvec(self, w):
        return self.apply(w)

    def precond(self, r):
        return r / np.diag(self.A).reshape(SHAPE)


class PseudoHuber:
    def __init__(self, seed):
        rng = np.random.default_rng(seed)
        self.v0 = 30.0 * rng.standard_normal(SHAPE)
        self.rho_T = np.zeros(SHAPE[1:])
        self.rho_R = np.ones(SHAPE[1:])
        self.lin = {'rho': [self.rho_R]}

    def project(self, v):
        return v

    def objective(self, v):
        return H3 * float(np.sum(np.sqrt(1.0 + v * v)))

    def gradient(self, v):
        return v / np.sqrt(1.0 + v * v), H3 * float(np.sum(np.sqrt(1.0 + v * v)))

    def hessian_matvec(self, w):
        return 0.1 * w

    def precond(self, r):
        return 10.0 * r


def test_quadratic_forcing_fixes_the_gradient_decrease():
    P = Quadratic(3)
    hist = []
    v, st = so.gauss_newton(P, np.zeros(SHAPE), gtol=1e-10, max_gn=20,
                            log=lambda k, J, rel, its, alpha, flag: hist.append(alpha))
    g = [h[1] for h in st['history']]
    assert st['gnorm_rel'] <= 1e-10
    assert all(a == 1.0 for a in hist)   # every full step passes Armijo
    for k in range(len(g) - 1):
        eta = min(0.5, g[k] / g[0])
        assert g[k + 1] <= eta * g[k] * (1 + 1e-9), (k, g[k + 1] / g[k], eta)
    # the minimiser of the quadratic
    x = np.linalg.solve(P.A, P.b.ravel()).reshape(SHAPE)
    assert np.abs(v - x).max() < 1e-8 * np.abs(x).max()


def test_objective_decreases_and_newton_steps_count_matches_the_forcing():
    # quadratic forcing gives q-superlinear decrease: from the first step on
    # the ratio ||g_{k+1}|| / ||g_k|| shrinks with ||g_k|| / ||g_0||
    P = Quadratic(11)
    _, st = so.gauss_newton(P, np.zeros(SHAPE), gtol=1e-8, max_gn=20)
    J = [h[0] for h in st['history']]
    assert all(J[i + 1] < J[i] for i in range(len(J) - 1))
    assert st['gn_iters'] <= 6


def test_armijo_halves_an_overshooting_step():
    P = PseudoHuber(5)
    alphas = []
    v, st = so.gauss_newton(P, P.v0, gtol=1e-6, max_gn=40,
                            log=lambda k, J, rel, its, alpha, flag: alphas.append(alpha))
    J = [h[0] for h in st['history']]
    assert all(J[i + 1] < J[i] for i in range(len(J) - 1))
    # the flat model overshoots: some steps were halved, and every accepted
    # step decreased J (sufficient decrease with <g, s> < 0)
    assert min(alphas) < 1.0
    assert not st.get('line_search_failed', False)
    assert st['gnorm_rel'] <= 1e-6
    assert np.abs(v).max() < 1e-5


def test_pins_catch_a_wrong_step_sign(monkeypatch):
    # a planted mistake: PCG's solution with the wrong sign (an ascent
    # direction).  The line search then finds no acceptable step and the
    # solve stops short of the tolerance, which both pins above check.
    orig = so.pcg

    def wrong_pcg(*a, **k):
        s, its, flag = orig(*a, **k)
        return -s, its, flag

    monkeypatch.setattr(so, 'pcg', wrong_pcg)
    for P, v0 in ((Quadratic(3), np.zeros(SHAPE)), (PseudoHuber(5), PseudoHuber(5).v0)):
        _, st = so.gauss_newton(P, v0, gtol=1e-6, max_gn=20)
        assert st.get('line_search_failed', False)
        assert st['gnorm_rel'] > 1e-6


class RegularisedQuadratic(Quadratic):
    """J_beta(v) = 1/2 <v, (A + beta B) v> - <b, v>: a data term plus a
    regularisation weighted by beta, minimiser (A + beta B)^-1 b."""

    def __init__(self, seed, beta):
        super().__init__(seed)
        rng = np.random.default_rng(seed + 100)
        n = self.A.shape[0]
        self.A = self.A - np.eye(n) + 1e-3 * np.eye(n)   # nearly singular data term
        self.B = np.diag(1.0 + rng.uniform(0.0, 10.0, n))
        self.beta = beta

    def apply(self, v):
        return ((self.A + self.beta * self.B) @ v.ravel()).reshape(SHAPE)

    def precond(self, r):
        return r / (self.beta * np.diag(self.B)).reshape(SHAPE)

    def minimiser(self):
        return np.linalg.solve(self.A + self.beta * self.B, self.b.ravel()).reshape(SHAPE)


def test_resumed_solve_with_the_reference_norm_repeats_the_uninterrupted_one():
    """gnorm_ref: a solve stopped after two Newton steps and resumed from its
    iterate with the original ||g_0|| takes exactly the remaining steps."""
    P = RegularisedQuadratic(7, 1e-2)
    v_all, st_all = so.gauss_newton(P, np.zeros(SHAPE), gtol=1e-9, max_gn=20)
    v2, st2 = so.gauss_newton(P, np.zeros(SHAPE), gtol=1e-9, max_gn=2)
    v_rest, st_rest = so.gauss_newton(P, v2, gtol=1e-9, max_gn=20, gnorm_ref=st2['gnorm0'])
    assert st2['gn_iters'] + st_rest['gn_iters'] == st_all['gn_iters']
    assert st2['pcg_per_step'] + st_rest['pcg_per_step'] == st_all['pcg_per_step']
    assert np.abs(v_rest - v_all).max() <= 1e-12 * np.abs(v_all).max()


def test_beta_schedule():
    assert np.allclose(so.beta_schedule(1e-1, 1e-4, 10.0), [1e-1, 1e-2, 1e-3, 1e-4])
    assert so.beta_schedule(1.0, 0.3, 10.0) == [1.0, 0.3]
    assert so.beta_schedule(1e-3, 1e-3, 10.0) == [1e-3]


def test_continuation_ends_at_the_target_minimiser():
    """Continuation from beta = 1 to 1e-4 reaches the minimiser of the target
    objective (to the stopping tolerance), the single-stage schedule is the
    plain solve, and the weight is restored afterwards."""
    P = RegularisedQuadratic(9, 1e-4)
    x = P.minimiser()
    v, st = so.continuation(P, np.zeros(SHAPE), 1.0, 10.0, gtol=1e-10, max_gn=30)
    assert [s['beta'] for s in st['stages']] == so.beta_schedule(1.0, 1e-4, 10.0)
    assert P.beta == 1e-4
    assert np.abs(v - x).max() < 1e-7 * np.abs(x).max()
    assert st['gn_iters'] == sum(s['gn_iters'] for s in st['stages'])
    v1, st1 = so.continuation(P, np.zeros(SHAPE), 1e-4, 10.0, gtol=1e-10, max_gn=30)
    v0, st0 = so.gauss_newton(P, np.zeros(SHAPE), gtol=1e-10, max_gn=30)
    assert np.array_equal(v1, v0) and st1['pcg_iters'] == st0['pcg_iters']
    # every stage stops at the first stage's reference norm: the final
    # gradient is below gtol times the gradient at v = 0
    assert st['gnorm'] <= 1e-10 * st['stages'][0]['gnorm0'] * (1 + 1e-9)

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

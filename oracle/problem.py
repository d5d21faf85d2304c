"""Objective, gradient and Gauss-Newton Hessian matvec (oracle, FP64).

Test infrastructure.  Follows Sec. II-B ("Formulation"):

  J[v] = 1/2 ||rho(1) - rho_R||^2 + beta/2 <v, A v>          Eq. (varopt)
  g(v) = beta A v + P b,  b = int_0^1 lam grad rho dt         Eq. (gradient)
  H v~ = beta A v~ + P b~,  b~ = int_0^1 lam~ grad rho dt     Eq. (hessian), GN
  full Newton: lam~ from Eq. (inc-adj) with div(lam v~) kept and
  b~ = int_0^1 (lam~ grad rho + lam grad rho~) dt              Eq. (hessian)

For the compressible problem P -> I (Sec. II-B, after Eq. (gradient)) and the
adjoint carries the source lam div v; for the incompressible problem v is kept
in the range of P, div v = 0, and the adjoint needs interpolation only.

Inner products are the discrete L2 product <a, b>_h = (2 pi)^3 / n * sum a b.
"""

import numpy as np

from . import spectral as _sp
from . import transport as _tr


def inner(a, b):
    """Discrete L2 inner product on [0, 2 pi)^3 for scalar or vector fields."""
    n = a.shape[-1] * a.shape[-2] * a.shape[-3]
    return (_sp.TWO_PI ** 3) / n * float(np.sum(a * b))


class Problem:
    """One registration problem: images, time steps, regularisation, variant.

    rho_T, rho_R: (N1, N2, N3) arrays.  kind: 'H2', 'H1' or 'H1DIV'.
    presmooth: apply the one-cell Gaussian to both images first (Sec. III-B1).
    newton: hessian_matvec applies the full Newton Hessian (Eq. (hessian) with
    the terms in lam) instead of the Gauss-Newton one.
    """

    def __init__(self, rho_T, rho_R, nt, beta, kind='H2', incompressible=False,
                 presmooth=False, newton=False):
        self.shape = rho_T.shape
        self.nt = int(nt)
        self.dt = 1.0 / self.nt
        self.beta = float(beta)
        self.kind = kind
        self.incompressible = bool(incompressible)
        self.newton = bool(newton)   # full Newton Hessian instead of Gauss-Newton
        rt = np.array(rho_T, dtype=np.float64)
        rr = np.array(rho_R, dtype=np.float64)
        if presmooth:
            h = _tr.grid_spacing(self.shape)
            rt = _sp.gaussian_smooth(rt, h)
            rr = _sp.gaussian_smooth(rr, h)
        self.rho_T = rt
        self.rho_R = rr
        self.lin = None  # quantities at the linearisation point

    # -- pieces --------------------------------------------------------
    def project(self, v):
        return _sp.leray(v) if self.incompressible else v

    def regularisation(self, v):
        return _sp.apply_regularisation(v, self.kind)

    def _divv(self, v):
        return None if self.incompressible else _sp.divergence(v)

    # -- Eq. (varopt) --------------------------------------------------
    def objective(self, v):
        """J[v]: forward state solve, mismatch and regularisation."""
        d_fwd = _tr.departure(v, self.dt)
        rho = _tr.state_solve(self.rho_T, d_fwd, self.nt)
        r = rho[-1] - self.rho_R
        return 0.5 * inner(r, r) + 0.5 * self.beta * inner(v, self.regularisation(v))

    # -- Eq. (gradient) ------------------------------------------------
    def gradient(self, v):
        """Returns (g, J) and stores the linearisation point for matvecs.

        Steps: semi-Lagrangian points of v and -v; state history; grad rho at
        every time level; adjoint backward from lam(1) = rho_R - rho(1);
        b by the time quadrature; g = beta A v + P b.
        """
        nt = self.nt
        d_fwd = _tr.departure(v, self.dt)
        d_adj = _tr.departure(-v, self.dt)
        divv = self._divv(v)
        rho = _tr.state_solve(self.rho_T, d_fwd, nt)
        grad_rho = [_sp.gradient(r) for r in rho]
        lam = _tr.adjoint_solve(self.rho_R - rho[-1], d_adj, divv, nt)
        b = _tr.time_integral(lam, grad_rho)
        av = self.regularisation(v)
        g = self.beta * av + self.project(b)
        r = rho[-1] - self.rho_R
        J = 0.5 * inner(r, r) + 0.5 * self.beta * inner(v, av)
        self.lin = dict(v=np.array(v), d_fwd=d_fwd, d_adj=d_adj, divv=divv,
                        rho=rho, grad_rho=grad_rho, lam=lam, b=b)
        return g, J

    # -- Eq. (hessian), Gauss-Newton -----------------------------------
    def incremental_state(self, vt):
        lin = self.lin
        return _tr.incremental_state_solve(vt, lin['grad_rho'], lin['d_fwd'], self.nt)

    def hessian_matvec(self, vt, full=None):
        """Hessian matvec at the last gradient's v.

        rho~ from Eq. (inc-state) (Algorithm 2), lam~(1) = -rho~(1)
        (Eq. (inc-adj-fc)), H v~ = beta A v~ + P b~.  Gauss-Newton (the
        default, full=False): lam~ from Eq. (inc-adj) without the div(lam v~)
        term and b~ = int lam~ grad rho dt (Sec. II-B drops both terms that
        involve lam).  Full Newton (full=True, or the problem's `newton`):
        lam~ with the source div(lam v~), where lam is the adjoint of the
        linearisation point at the time levels, and b~ = int (lam~ grad rho +
        lam grad rho~) dt, grad rho~ spectral on every level.
        """
        if self.lin is None:
            raise RuntimeError('hessian_matvec before gradient')
        full = self.newton if full is None else full
        lin = self.lin
        rt = self.incremental_state(vt)
        src = None
        if full:
            src = [_sp.divergence(lin['lam'][j] * vt) for j in range(self.nt + 1)]
        lt = _tr.adjoint_solve(-rt[-1], lin['d_adj'], lin['divv'], self.nt, src)
        bt = _tr.time_integral(lt, lin['grad_rho'])
        if full:
            bt = bt + _tr.time_integral(lin['lam'], [_sp.gradient(r) for r in rt])
        return self.beta * self.regularisation(vt) + self.project(bt)

    def precond(self, r):
        """Inverse-regularisation spectral preconditioner (Sec. III-A)."""
        return _sp.preconditioner(r, self.beta, self.kind, self.incompressible)

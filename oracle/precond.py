"""Two-level spectral preconditioner (oracle, FP64).

Test infrastructure.  Sec. III-A: the spectral preconditioner (beta A)^-1 is
mesh independent but not beta independent, and Sec. I (limitations) names
grid continuation and multilevel preconditioning as the remedy; Sec. IV-C
(Table 5) shows the Hessian matvecs growing as beta falls.  The paper builds
no such preconditioner; this module states the two-level reading used here.

Every field is its Fourier series on the periodic grid (Sec. III-B1), so a
coarse grid of n_c points per axis holds exactly the modes
L = {k : |k_j| < n_c,j / 2 on every axis} (the whole axis when n_c = n), and
restriction / prolongation between the grids are exact on L (normalised
coefficients are the same numbers on both grids).  The preconditioner is

    M^-1 r = Pi_L H_c^-1 Pi_L r + (beta A)^-1 P (I - Pi_L) r,

with H_c the Gauss-Newton Hessian of the same problem on the coarse grid
(images restricted to L, linearised at the restriction of the current v),
inverted approximately by PCG with the coarse spectral preconditioner to a
relative tolerance, and the inverse regularisation operator on the modes
outside L.  An inexact inner solve makes M^-1 vary with r, so the outer
Krylov method is flexible CG (solver.fpcg).
"""

import numpy as np

from . import spectral as _sp
from .problem import Problem, inner
from .solver import pcg


def _axis_map(n, nc):
    """Indices (fine, coarse) of the modes |k| < nc/2 along one axis in FFT
    order; the whole axis when nc == n."""
    if nc == n:
        idx = np.arange(n)
        return idx, idx
    k = _sp.wavenumbers(n)
    fine = np.nonzero(2 * np.abs(k) < nc)[0]
    coarse = np.where(k[fine] >= 0, k[fine], k[fine] + nc).astype(int)
    return fine, coarse


def restrict(f, shape_c):
    """The field of the modes in L on the coarse grid (scalar or vector)."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 4:
        return np.stack([restrict(c, shape_c) for c in f])
    shape = f.shape
    fh = np.fft.fftn(f) / f.size
    gh = np.zeros(tuple(shape_c), dtype=complex)
    (f1, c1), (f2, c2), (f3, c3) = [_axis_map(n, m) for n, m in zip(shape, shape_c)]
    gh[np.ix_(c1, c2, c3)] = fh[np.ix_(f1, f2, f3)]
    return np.real(np.fft.ifftn(gh) * np.prod(shape_c))


def prolong(fc, shape):
    """The coarse field's modes in L placed on the fine grid (zero elsewhere)."""
    fc = np.asarray(fc, dtype=np.float64)
    if fc.ndim == 4:
        return np.stack([prolong(c, shape) for c in fc])
    shape_c = fc.shape
    gh = np.fft.fftn(fc) / fc.size
    fh = np.zeros(tuple(shape), dtype=complex)
    (f1, c1), (f2, c2), (f3, c3) = [_axis_map(n, m) for n, m in zip(shape, shape_c)]
    fh[np.ix_(f1, f2, f3)] = gh[np.ix_(c1, c2, c3)]
    return np.real(np.fft.ifftn(fh) * np.prod(shape))


def low_pass(f, shape_c):
    """Pi_L f on the fine grid."""
    return prolong(restrict(f, shape_c), f.shape[-3:])


class TwoLevel:
    """The two-level preconditioner of a Problem with a coarse grid shape_c.

    linearize(v) sets the coarse Hessian's linearisation point to the
    restriction of v; apply(r) returns M^-1 r.  inner_tol is the inner PCG's
    relative residual tolerance, inner_max its iteration cap (inner_tol = 0
    runs exactly inner_max iterations unless the residual vanishes).  nt_c:
    the coarse Hessian's semi-Lagrangian time steps (None: the fine nt); a
    coarse grid moves a point across fewer cells per step, so it may take
    fewer steps -- any nt_c gives an SPD H_c, so M^-1 stays a valid
    preconditioner for the flexible outer iteration.
    """

    def __init__(self, problem, shape_c, inner_tol=0.1, inner_max=10, nt_c=None):
        self.P = problem
        self.shape_c = tuple(shape_c)
        self.inner_tol = float(inner_tol)
        self.inner_max = int(inner_max)
        self.coarse = Problem(restrict(problem.rho_T, shape_c), restrict(problem.rho_R, shape_c),
                              int(nt_c) if nt_c else problem.nt, problem.beta, problem.kind,
                              problem.incompressible)
        self.inner_iters = 0

    def linearize(self, v):
        self.coarse.beta = self.P.beta
        self.coarse.gradient(restrict(v, self.shape_c))

    def apply(self, r):
        # the Krylov residuals of the incompressible problem lie in the range
        # of P already; projecting keeps the inner solve there for any r
        rl = self.coarse.project(restrict(r, self.shape_c))
        tol = self.inner_tol * np.sqrt(inner(rl, rl))
        y, its, _ = pcg(self.coarse.hessian_matvec, self.coarse.precond, rl, tol,
                        self.inner_max)
        self.inner_iters += its
        shape = r.shape[1:]
        high = r - low_pass(r, self.shape_c)
        return prolong(y, shape) + _sp.preconditioner(high, self.P.beta, self.P.kind,
                                                      self.P.incompressible)


class TwoLevelProblem:
    """A Problem whose preconditioner is the two-level operator: gradient()
    also relinearises the coarse Hessian, precond() applies M^-1.  For
    solver.gauss_newton(..., flexible=True)."""

    def __init__(self, problem, shape_c, inner_tol=0.1, inner_max=10, nt_c=None):
        self.base = problem
        self.two = TwoLevel(problem, shape_c, inner_tol, inner_max, nt_c)

    def __getattr__(self, name):
        return getattr(self.base, name)

    def gradient(self, v):
        out = self.base.gradient(v)
        self.two.linearize(v)
        return out

    def precond(self, r):
        return self.two.apply(r)

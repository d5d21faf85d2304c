"""Semi-Lagrangian transport solves (oracle, FP64).  Test infrastructure.

Sec. III-B2 ("Time").  A field nu transported by the stationary velocity v
with a source f,  d_t nu + v . grad nu = f,  advances one step dt by

  * the RK2 semi-Lagrangian point, Eq. (sml-trajectory):
        X* = x - dt v(x),     X = x - (dt/2) (v(x) + v(X*));
  * the predictor-corrector along the characteristic, Eq. (sml-advection):
        nu_0 = nu(X, t),  f_0 = f(X, t),  nu_* = nu_0 + dt f_0,
        f_* = f(nu_*, x, t + dt),  nu(x, t + dt) = nu_0 + (dt/2)(f_0 + f_*).

Off-grid values come from the tricubic interpolant (oracle.interp).  The
adjoint equations run in tau = 1 - t with the velocity -v, so their points are
the semi-Lagrangian points of -v.  dt = 1/nt throughout.

Points are kept as displacements X - x in grid units (3, N1, N2, N3).
"""

import numpy as np

from . import interp as _interp
from . import spectral as _spectral


def grid_spacing(shape):
    return tuple(_spectral.TWO_PI / n for n in shape)


def departure(v, dt):
    """RK2 semi-Lagrangian points of v, Eq. (sml-trajectory).

    v: (3, N1, N2, N3) velocity in physical units.  Returns X - x in grid
    units.  The points depend on v only (Sec. III-C2): they are computed once
    per velocity and reused by every transport solve with that velocity.
    """
    shape = v.shape[1:]
    h = grid_spacing(shape)
    g = _interp.grid_index(shape)
    star = tuple(g[j] - dt * v[j] / h[j] for j in range(3))
    v_star = [_interp.interp(v[j], star) for j in range(3)]
    return np.stack([-(dt / 2.0) * (v[j] + v_star[j]) / h[j] for j in range(3)])


def state_solve(rho0, d_fwd, nt):
    """Forward state, Eq. (varopt:state): d_t rho + v . grad rho = 0, rho(0) = rho_T.

    No source, so each step is one interpolation at the points of v.  All
    nt + 1 time levels are returned (the method stores the whole history,
    Sec. III-B2).
    """
    rho = [np.array(rho0, dtype=np.float64)]
    for _ in range(nt):
        rho.append(_interp.interp_at_displacement(rho[-1], d_fwd))
    return rho


def adjoint_step(nu, d_adj, divv, dt, src_old=None, src_new=None):
    """One tau-step of -d_t lam - div(v lam) = 0 (Eq. (adjoint)).

    In tau = 1 - t this is d_tau lam + (-v) . grad lam = lam div v: transport
    by -v with the source f(lam, x) = lam div v(x).  With divv None the
    velocity is divergence free and the source vanishes (Sec. III-C2: the
    state and adjoint then need only interpolations).

    Eq. (sml-advection) evaluates the source at the semi-Lagrangian point as
    f_0(X) = f(nu_0(X), X) = nu_0(X) * (div v)(X): the interpolated field times
    div v interpolated at X (an interpolation "for the f terms that depend on
    the semi-Lagrangian point").  Then nu_* = nu_0 + dt f_0,
    f_* = nu_* div v(x), lam_new = nu_0 + dt/2 (f_0 + f_*).

    src_old, src_new: an additional known source s(x, tau) at the level the
    step starts from and at the level it reaches (the full-Newton incremental
    adjoint of Eq. (inc-adj) carries s = div(lam v~)); f gains s, with
    s_old interpolated at X like every term that belongs to the
    semi-Lagrangian point and s_new taken at the grid point.
    """
    nu0 = _interp.interp_at_displacement(nu, d_adj)
    f0 = np.zeros_like(nu0) if divv is None else nu0 * _interp.interp_at_displacement(divv, d_adj)
    if src_old is not None:
        f0 = f0 + _interp.interp_at_displacement(src_old, d_adj)
    nu_star = nu0 + dt * f0
    f_star = np.zeros_like(nu0) if divv is None else nu_star * divv
    if src_new is not None:
        f_star = f_star + src_new
    return nu0 + (dt / 2.0) * (f0 + f_star)


def adjoint_solve(lam_final, d_adj, divv, nt, src=None):
    """Adjoint (or incremental adjoint) backward in time.

    lam_final is the value at t = 1.  Returns [lam(t_0), ..., lam(t_nt)].
    Used for Eq. (adjoint) with lam(1) = rho_R - rho(1), and for Eq. (inc-adj)
    with lam~(1) = -rho~(1): the Gauss-Newton Hessian drops div(lam v~), so
    the incremental adjoint is the same equation (Sec. II-B).  For the full
    Newton Hessian, src = [s(t_0), ..., s(t_nt)] is the known source
    s = div(lam v~) of Eq. (inc-adj) on the time levels: in tau the equation
    reads d_tau lam~ + (-v) . grad lam~ = lam~ div v + div(lam v~).
    """
    dt = 1.0 / nt
    lam = [None] * (nt + 1)
    lam[nt] = np.array(lam_final, dtype=np.float64)
    for j in range(nt - 1, -1, -1):
        if src is None:
            lam[j] = adjoint_step(lam[j + 1], d_adj, divv, dt)
        else:
            lam[j] = adjoint_step(lam[j + 1], d_adj, divv, dt, src[j + 1], src[j])
    return lam


def incremental_state_solve(vt, grad_rho, d_fwd, nt):
    """Incremental state, Eq. (inc-state), one step as in Algorithm 2.

    d_t rho~ + v . grad rho~ = f(x, t),  f = -v~ . grad rho(t),  rho~(0) = 0.
    The source does not depend on rho~, so per step
        rho~_{j+1}(x) = rho~_j(X) + (dt/2) (f_j(X) + f_{j+1}(x)),
    with f_j formed on the grid and interpolated at X (Algorithm 2).  Reading of
    a garble in Algorithm 2 (it writes the state rho where the incremental
    state is meant, and grad rho_* for the corrector): the corrector uses
    grad rho at the new time level t_{j+1}, an input of the algorithm.

    grad_rho: list of nt + 1 arrays (3, N1, N2, N3).  Returns all levels.
    """
    dt = 1.0 / nt
    f = [-np.sum(vt * grad_rho[j], axis=0) for j in range(nt + 1)]
    rt = [np.zeros_like(f[0])]
    for j in range(nt):
        nu0 = _interp.interp_at_displacement(rt[j], d_fwd)
        f0 = _interp.interp_at_displacement(f[j], d_fwd)
        rt.append(nu0 + (dt / 2.0) * (f0 + f[j + 1]))
    return rt


def trapezoid_weights(nt):
    """Time-quadrature weights on t_j = j/nt: the paper is silent; reading:
    the trapezoidal rule (w_0 = w_nt = dt/2, w_j = dt otherwise)."""
    dt = 1.0 / nt
    w = np.full(nt + 1, dt)
    w[0] = w[nt] = dt / 2.0
    return w


def time_integral(lam, grad_rho):
    """b = int_0^1 lam grad rho dt (Eq. (gradient)); also b~ (Eq. (hessian))."""
    nt = len(lam) - 1
    w = trapezoid_weights(nt)
    b = np.zeros_like(grad_rho[0])
    for j in range(nt + 1):
        b += w[j] * lam[j] * grad_rho[j]
    return b


def deformation_displacement(v, d_fwd, nt):
    """u = y(x, 1) - x from Eq. (euler-def), d_t y + v . grad y = 0, y(0) = x.

    With y = x + u: d_t u + v . grad u = -v, u(0) = 0; a transport with the
    known, time-independent source f = -v, advanced by Eq. (sml-advection).
    """
    dt = 1.0 / nt
    u = np.zeros_like(v)
    for _ in range(nt):
        nxt = np.empty_like(u)
        for c in range(3):
            nu0 = _interp.interp_at_displacement(u[c], d_fwd)
            f0 = _interp.interp_at_displacement(-v[c], d_fwd)
            nxt[c] = nu0 + (dt / 2.0) * (f0 - v[c])
        u = nxt
    return u


def jacobian_determinant(u):
    """det(grad y) = det(I + grad u), derivatives spectral (Sec. II-A)."""
    gu = np.stack([_spectral.gradient(u[c]) for c in range(3)])  # gu[c, j] = d_j u_c
    m = gu + np.eye(3)[:, :, None, None, None]
    return (m[0, 0] * (m[1, 1] * m[2, 2] - m[1, 2] * m[2, 1])
            - m[0, 1] * (m[1, 0] * m[2, 2] - m[1, 2] * m[2, 0])
            + m[0, 2] * (m[1, 0] * m[2, 1] - m[1, 1] * m[2, 0]))

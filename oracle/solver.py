"""Inexact Gauss-Newton-Krylov solve (oracle, FP64).  Test infrastructure.

Sec. III-A: Newton steps from PCG on H s = -g, preconditioned by the inverse
regularisation operator, solved inexactly to a tolerance tied to the relative
gradient norm; globalised by an Armijo line search.  Sec. IV-A3: Gauss-Newton,
gradient tolerance 1e-2 relative, "quadratic forcing".

Readings (the paper does not give these constants):
* forcing: eta_k = min(0.5, ||g_k|| / ||g_0||) (quadratic forcing);
* PCG starts from s = 0 and stops when the unpreconditioned residual satisfies
  ||r|| <= eta_k ||g_k|| (norms in <.,.>_h), or after max_pcg iterations;
* if PCG meets p.Hp <= 0 (the discretised GN Hessian is only symmetric up to
  discretisation error), it stops and returns the current iterate, or the
  preconditioned steepest-descent direction on the first iteration;
* Armijo: alpha = 1, 1/2, 1/4, ... (at most armijo_max trials); accept when
  J(v + alpha s) <= J(v) + c alpha <g, s>, c = 1e-4;
* stop when ||g_k|| <= gtol ||g_0|| or after max_gn iterations (50 in the
  paper's brain runs, Sec. IV-C).
"""

import numpy as np

from .problem import inner


def pcg(matvec, precond, rhs, tol_abs, max_iter):
    """Preconditioned CG for H s = rhs from s = 0.  Returns (s, iters, flag)."""
    s = np.zeros_like(rhs)
    r = rhs.copy()
    z = precond(r)
    p = z.copy()
    rz = inner(r, z)
    if np.sqrt(inner(r, r)) <= tol_abs:
        return s, 0, 'converged'
    for it in range(1, max_iter + 1):
        q = matvec(p)
        pq = inner(p, q)
        if pq <= 0.0:
            if it == 1:
                return p, it, 'negative_curvature'
            return s, it, 'negative_curvature'
        alpha = rz / pq
        s = s + alpha * p
        r = r - alpha * q
        if np.sqrt(inner(r, r)) <= tol_abs:
            return s, it, 'converged'
        z = precond(r)
        rz_new = inner(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return s, max_iter, 'max_iter'


def gauss_newton(problem, v0, gtol=1e-2, max_gn=50, max_pcg=500,
                 armijo_c=1e-4, armijo_max=10, log=None):
    """Inexact GN-Krylov with Armijo line search.  Returns (v, stats)."""
    v = problem.project(np.array(v0, dtype=np.float64))
    g, J = problem.gradient(v)
    g0 = np.sqrt(inner(g, g))
    gn = g0
    stats = dict(gn_iters=0, pcg_iters=0, matvecs=0, J0=J, J=J, gnorm0=g0,
                 gnorm=g0, history=[(J, g0)])
    r0 = problem.rho_T - problem.rho_R
    m0 = np.sqrt(inner(r0, r0))
    for k in range(max_gn):
        if gn <= gtol * g0 or g0 == 0.0:
            break
        eta = min(0.5, gn / g0)
        s, its, flag = pcg(problem.hessian_matvec, problem.precond, -g,
                           eta * gn, max_pcg)
        stats['pcg_iters'] += its
        stats['matvecs'] += its
        slope = inner(g, s)
        alpha = 1.0
        accepted = False
        for _ in range(armijo_max):
            vt = v + alpha * s
            Jt = problem.objective(vt)
            if Jt <= J + armijo_c * alpha * slope:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            stats['line_search_failed'] = True
            break
        v = vt
        g, J = problem.gradient(v)
        gn = np.sqrt(inner(g, g))
        stats['gn_iters'] = k + 1
        stats['history'].append((J, gn))
        if log is not None:
            log(k + 1, J, gn / g0, its, alpha, flag)
    stats['J'] = J
    stats['gnorm'] = gn
    stats['gnorm_rel'] = gn / g0 if g0 > 0 else 0.0
    rho1 = problem.lin['rho'][-1]
    r1 = rho1 - problem.rho_R
    stats['mismatch_rel'] = np.sqrt(inner(r1, r1)) / m0 if m0 > 0 else 0.0
    return v, stats

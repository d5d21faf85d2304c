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


def fpcg(matvec, precond, rhs, tol_abs, max_iter):
    """Flexible preconditioned CG for H s = rhs from s = 0 (the direction
    update beta = -alpha <z_new, q> / <r, z>, q = H p).  Same return
    convention as solver.pcg: (s, iters, flag)."""
    s = np.zeros_like(rhs)
    r = rhs.copy()
    if np.sqrt(inner(r, r)) <= tol_abs:
        return s, 0, 'converged'
    z = precond(r)
    p = z.copy()
    rz = inner(r, z)
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
        bk = -alpha * inner(z, q) / rz
        rz = inner(r, z)
        p = z + bk * p
    return s, max_iter, 'max_iter'


def gauss_newton(problem, v0, gtol=1e-2, max_gn=50, max_pcg=500,
                 armijo_c=1e-4, armijo_max=10, log=None, gnorm_ref=None, flexible=False):
    """Inexact GN-Krylov with Armijo line search.  Returns (v, stats).

    gnorm_ref: the reference ||g_0|| of the stop test ||g|| <= gtol ||g_0||
    and of the forcing term eta = min(0.5, ||g|| / ||g_0||); None takes the
    gradient norm at v0 (the paper's solves start from v = 0).  A solve
    resumed from one of its own iterates with the original ||g_0|| takes the
    same steps as the uninterrupted solve.  flexible: the Newton steps by
    flexible PCG (for a preconditioner that varies with its argument, such
    as the two-level one of oracle.precond).
    """
    v = problem.project(np.array(v0, dtype=np.float64))
    g, J = problem.gradient(v)
    gn = np.sqrt(inner(g, g))
    g0 = gn if gnorm_ref is None else float(gnorm_ref)
    stats = dict(gn_iters=0, pcg_iters=0, matvecs=0, J0=J, J=J, gnorm0=g0,
                 gnorm=gn, history=[(J, gn)], pcg_per_step=[])
    r0 = problem.rho_T - problem.rho_R
    m0 = np.sqrt(inner(r0, r0))
    for k in range(max_gn):
        if gn <= gtol * g0 or g0 == 0.0:
            break
        eta = min(0.5, gn / g0)
        krylov = fpcg if flexible else pcg
        s, its, flag = krylov(problem.hessian_matvec, problem.precond, -g, eta * gn, max_pcg)
        stats['pcg_iters'] += its
        stats['matvecs'] += its
        stats['pcg_per_step'].append(its)
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


def beta_schedule(beta_start, beta, factor):
    """Continuation values of the regularisation weight: beta_start,
    beta_start / factor, ... while above beta, then beta itself."""
    out = []
    b = float(beta_start)
    while b > beta * (1.0 + 1e-12):
        out.append(b)
        b /= factor
    out.append(float(beta))
    return out


def continuation(problem, v0, beta_start, factor=10.0, gtol=1e-2, **kw):
    """Parameter continuation on beta (Sec. III-A: the problem is highly
    nonlinear, so the solver starts from a larger regularisation weight and
    lowers it to the target).  Reading (the paper gives no schedule): beta is
    divided by `factor` from beta_start down to the problem's beta, each
    stage a Gauss-Newton solve warm-started from the last one, every stage
    stopped at ||g|| <= gtol ||g(v0)|| with ||g(v0)|| from the first stage
    (at v0 = 0 the gradient -- P[(rho_R - rho_T) grad rho_T] -- does not
    depend on beta, so every stage stops at the same absolute norm).
    Returns (v, stats) with per-stage statistics in stats['stages'].
    """
    target = problem.beta
    v = np.array(v0, dtype=np.float64)
    stages, ref = [], kw.pop('gnorm_ref', None)
    try:
        for b in beta_schedule(beta_start, target, factor):
            problem.beta = b
            v, st = gauss_newton(problem, v, gtol=gtol, gnorm_ref=ref, **kw)
            if ref is None:
                ref = st['gnorm0']
            st['beta'] = b
            stages.append(st)
    finally:
        problem.beta = target
    total = dict(stages[-1])
    total['stages'] = stages
    for key in ('gn_iters', 'pcg_iters', 'matvecs'):
        total[key] = sum(st[key] for st in stages)
    return v, total

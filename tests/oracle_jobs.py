"""Oracle reference computations that take minutes, run in worker processes.

Test infrastructure.  The FP64 oracle at 128^3 takes about a minute per
gradient or Hessian matvec on one host core, so the references of the
128^3 parity tests are computed in a pool of spawned worker processes that
starts when the test session has collected them (tests/conftest.py) and runs
while the rest of the GPU suite does.  The workers import only ``oracle`` and
the seeded input generator ``synth``; nothing here touches the GPU.

Every job returns its inputs as the GPU receives them (images rounded to
FP32, velocities and directions as normalised half-spectrum coefficients
rounded to complex64) and the oracle's results on exactly those inputs, as
normalised half-spectrum coefficients in complex128.
"""

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np

FUTURES = {}
_POOL = None


def to_hat(f):
    """Normalised half spectrum F f / n of a (..., n1, n2, n3) real field."""
    n = f.shape[-1] * f.shape[-2] * f.shape[-3]
    return np.fft.rfftn(f, axes=(-3, -2, -1)) / n


def from_hat(fh, shape):
    """The real field whose normalised half spectrum is fh."""
    n = shape[0] * shape[1] * shape[2]
    return np.fft.irfftn(fh * n, s=shape, axes=(-3, -2, -1))


def rounded_hat(f):
    """(complex64 coefficients the GPU receives, the FP64 field they define)."""
    h32 = to_hat(f).astype(np.complex64)
    return h32, from_hat(h32.astype(np.complex128), f.shape[-3:])


def herm_weights(shape):
    """Parseval weights of the half spectrum: 1 on the k3 = 0 (and Nyquist)
    planes, 2 elsewhere."""
    m3 = shape[2] // 2 + 1
    w = np.full(m3, 2.0)
    w[0] = 1.0
    if shape[2] % 2 == 0:
        w[-1] = 1.0
    return w


def rel_hat(got, ref, shape):
    """Relative L2 error of normalised half-spectrum coefficients (the
    physical-space relative L2, by Parseval)."""
    w = herm_weights(shape)
    d = np.abs(np.asarray(got).astype(np.complex128) - ref) ** 2
    return float(np.sqrt(np.sum(d * w) / np.sum(np.abs(ref) ** 2 * w)))


def sinusoid_case(shape, scale, kind, incompressible, beta, nt, vscale, dir_seeds, dir_kmax=8):
    """Gradient and Hessian matvecs of the sinusoid problem (v* x scale) at
    v = vscale v*, on band-limited directions (|k| <= dir_kmax, Leray-projected
    when incompressible)."""
    from oracle import problem as opr
    from oracle import spectral as osp
    from paper_1608_03630_gb300 import synth
    rho_T, rho_R, vs = synth.sinusoid_problem(shape, scale)
    rho_T = rho_T.astype(np.float32).astype(np.float64)
    rho_R = rho_R.astype(np.float32).astype(np.float64)
    v = vscale * vs
    if incompressible:
        v = osp.leray(v)
    v_hat, v = rounded_hat(v)
    P = opr.Problem(rho_T, rho_R, nt, beta, kind, incompressible)
    g, J = P.gradient(v)
    out = dict(rho_T=rho_T.astype(np.float32), rho_R=rho_R.astype(np.float32), v_hat=v_hat,
               g_hat=to_hat(g), J=J, w_hat=[], h_hat=[], w=[], h=[])
    for s in dir_seeds:
        w = synth.bandlimited(shape, dir_kmax, s)
        if incompressible:
            w = osp.leray(w)
        w_hat, w = rounded_hat(w)
        h = P.hessian_matvec(w)
        out['w_hat'].append(w_hat)
        out['h_hat'].append(to_hat(h))
        out['w'].append(w.astype(np.float32))
        out['h'].append(h)
    return out


JOBS = {
    # the 128^3 sinusoid problem, nt = 4, v* x 1.0; compressible H2 beta = 1e-2
    'c128_h2_a': (sinusoid_case, ((128, 128, 128), 1.0, 'H2', False, 1e-2, 4, 0.5, (1001,))),
    'c128_h2_b': (sinusoid_case, ((128, 128, 128), 1.0, 'H2', False, 1e-2, 4, 0.5, (1002, 1003))),
    # the same problem, incompressible: Leray projection, H1-div, beta = 1e-3
    'c128_div_a': (sinusoid_case, ((128, 128, 128), 1.0, 'H1DIV', True, 1e-3, 4, 0.5, (1001,))),
    'c128_div_b': (sinusoid_case, ((128, 128, 128), 1.0, 'H1DIV', True, 1e-3, 4, 0.5,
                                   (1002, 1003))),
    # interior tensor-copy blocks (x3 = 128 > the 64-wide box), beta = 1e-3
    'tma_64x64x128': (sinusoid_case, ((64, 64, 128), 1.0, 'H2', False, 1e-3, 4, 0.5,
                                      (1101, 1102))),
}


def start(names=None):
    """Submit the named jobs (default: all) to a pool of spawned workers."""
    global _POOL
    if _POOL is None:
        names = list(JOBS) if names is None else list(names)
        _POOL = cf.ProcessPoolExecutor(max_workers=len(names),
                                       mp_context=mp.get_context('spawn'))
        for name in names:
            fn, args = JOBS[name]
            FUTURES[name] = _POOL.submit(fn, *args)
    return FUTURES


def result(name, timeout=3600):
    """The job's result, starting the pool first if nothing started it."""
    if name not in FUTURES:
        start()
    return FUTURES[name].result(timeout=timeout)


def shutdown():
    """Cancel pending jobs and stop the workers (a session that ends early
    does not wait for references nobody will read)."""
    global _POOL
    if _POOL is not None:
        procs = list(getattr(_POOL, '_processes', {}).values())
        _POOL.shutdown(wait=False, cancel_futures=True)
        for p in procs:
            if p.is_alive():
                p.terminate()
        _POOL = None

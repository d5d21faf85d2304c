"""Spectral operators on the periodic grid (oracle, FP64).  Test infrastructure.

Discretisation (Sec. III-B1, "Space"): the domain is [0, 2*pi)^3 with
N_i points per axis at x = 2*pi*i/N_i; every field is a trigonometric
polynomial with wavenumbers -N/2 <= k <= N/2 - 1 (FFT order).  All
derivatives are applied by an FFT, a diagonal scaling of the spectral
coefficients and an inverse FFT.

Readings (the paper prints the expansion as exp(-k.x) with k in N^3 -- read as
exp(i k.x), k in Z^3 -- and does not say how the Nyquist mode is treated):

* first (odd) derivatives use k' = k with the Nyquist entry |k_j| = N_j/2 set to
  zero, so that the derivative of a real field stays real and div(P v) = 0
  holds exactly on the grid;
* even operators (Laplacian, biharmonic) use the full k, Nyquist included;
* the Leray projection uses k': P(k) = I - k' k'^T / |k'|^2, and P = I where
  k' = 0.

Every function takes and returns real arrays of shape (N1, N2, N3) (scalar)
or (3, N1, N2, N3) (vector).  This module is plain: full complex FFTs, no
half-spectrum tricks.
"""

import numpy as np

TWO_PI = 2.0 * np.pi


def wavenumbers(n):
    """Integer wavenumbers in FFT order: 0, 1, ..., n/2-1, -n/2, ..., -1."""
    return np.fft.fftfreq(n, d=1.0 / n)


def odd_wavenumbers(n):
    """Wavenumbers for first derivatives: the Nyquist entry (n even) is zero."""
    k = wavenumbers(n)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return k


def kgrid(shape):
    """Broadcastable wavenumber arrays (k1, k2, k3) with the full k."""
    n1, n2, n3 = shape
    return (wavenumbers(n1)[:, None, None],
            wavenumbers(n2)[None, :, None],
            wavenumbers(n3)[None, None, :])


def kgrid_odd(shape):
    """Broadcastable wavenumber arrays (k1', k2', k3') for first derivatives."""
    n1, n2, n3 = shape
    return (odd_wavenumbers(n1)[:, None, None],
            odd_wavenumbers(n2)[None, :, None],
            odd_wavenumbers(n3)[None, None, :])


def ksq(shape):
    """|k|^2 with the full wavenumbers (symbol of -Laplacian)."""
    k1, k2, k3 = kgrid(shape)
    return k1 * k1 + k2 * k2 + k3 * k3


def fft(f):
    return np.fft.fftn(f)


def ifft(fh):
    return np.real(np.fft.ifftn(fh))


def gradient(f):
    """grad f, Sec. III-B1: multiply the coefficients by i k'_j."""
    fh = fft(f)
    kp = kgrid_odd(f.shape)
    return np.stack([ifft(1j * kp[j] * fh) for j in range(3)])


def divergence(v):
    """div v = sum_j d_j v_j, each derivative spectral with i k'_j."""
    kp = kgrid_odd(v.shape[1:])
    acc = np.zeros(v.shape[1:], dtype=complex)
    for j in range(3):
        acc += 1j * kp[j] * fft(v[j])
    return ifft(acc)


def apply_symbol(f, symbol):
    """Inverse FFT of symbol(k) * FFT(f), for a scalar field."""
    return ifft(symbol * fft(f))


def laplacian(f):
    """Lap f: symbol -|k|^2."""
    return apply_symbol(f, -ksq(f.shape))


def regularisation_symbol(shape, kind):
    """Symbol A(k) of the regularisation operator.

    kind 'H2' -- A = |k|^4, the biharmonic Lap^2 that comes from the seminorm
                 ||Lap v||^2 of the objective, Eq. (varopt).
    kind 'H1' -- A = |k|^2 (-Lap; from ||grad v||^2).  Not defined in the
                 paper; reading of the H1 variant.
    kind 'H1DIV' -- A = |k|^2 applied to the Leray-projected velocity.  With
                 div v = 0 enforced by P, a penalty on div v vanishes
                 identically, so the operator equals H1 (reading).
    """
    s = ksq(shape)
    if kind == 'H2':
        return s * s
    if kind in ('H1', 'H1DIV'):
        return s
    raise ValueError(kind)


def apply_regularisation(v, kind):
    """A v for a vector field, component by component."""
    sym = regularisation_symbol(v.shape[1:], kind)
    return np.stack([apply_symbol(v[j], sym) for j in range(3)])


def leray(v):
    """Leray projection P v = (I - grad Lap^{-1} div) v, Eq. (gradient).

    In Fourier space P(k) = I - k' k'^T / |k'|^2; P(k) = I where k' = 0.
    """
    kp = kgrid_odd(v.shape[1:])
    vh = [fft(v[j]) for j in range(3)]
    kk = kp[0] ** 2 + kp[1] ** 2 + kp[2] ** 2
    dot = kp[0] * vh[0] + kp[1] * vh[1] + kp[2] * vh[2]
    safe = np.where(kk > 0, kk, 1.0)
    coef = np.where(kk > 0, dot / safe, 0.0)
    return np.stack([ifft(vh[j] - kp[j] * coef) for j in range(3)])


def preconditioner(r, beta, kind, incompressible):
    """Spectral preconditioner: the inverse regularisation operator, Sec. III-A.

    z = F^{-1}[ M(k) P(k) F r ] with M(k) = 1 / (beta A(k)) for k != 0.  A(0) = 0
    makes the paper's "inverse of the biharmonic" singular at k = 0; reading:
    M(0) = 1 / beta.  For the compressible problem P -> I.
    """
    shape = r.shape[1:]
    a = regularisation_symbol(shape, kind)
    m = np.where(a > 0, 1.0 / (beta * np.where(a > 0, a, 1.0)), 1.0 / beta)
    rr = leray(r) if incompressible else r
    return np.stack([apply_symbol(rr[j], m) for j in range(3)])


def gaussian_smooth(f, sigma):
    """Spectral Gaussian filter exp(-sum_j sigma_j^2 k_j^2 / 2), Sec. III-B1.

    sigma is a 3-tuple in physical units; the method pre-smooths its input
    images with sigma_j = h_j = 2 pi / N_j (one grid cell).
    """
    k1, k2, k3 = kgrid(f.shape)
    g = np.exp(-0.5 * ((sigma[0] * k1) ** 2 + (sigma[1] * k2) ** 2
                       + (sigma[2] * k3) ** 2))
    return apply_symbol(f, g)


def resample(f, shape_out):
    """Trigonometric resampling of f (scalar (N1, N2, N3) or (c, N1, N2, N3))
    to the grid shape_out (Sec. III-B1: a field is its Fourier series on the
    grid).  Reading: the coefficients with |k_j| < min(N_j, M_j)/2 on every
    axis are kept and all others, the Nyquist planes included, are dropped, so
    the result is real and a field band-limited to the kept modes is
    reproduced exactly on the new points."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 4:
        return np.stack([resample(c, shape_out) for c in f])
    nin = f.shape
    fh = np.fft.fftn(f) / f.size
    gh = np.zeros(tuple(shape_out), dtype=complex)
    keep = []
    for a, b in zip(nin, shape_out):
        k = wavenumbers(a)
        lim = min(a, b)
        idx_in = np.nonzero(2 * np.abs(k) < lim)[0]
        idx_out = np.where(k[idx_in] >= 0, k[idx_in], k[idx_in] + b).astype(int)
        keep.append((idx_in, idx_out))
    (i1, o1), (i2, o2), (i3, o3) = keep
    gh[np.ix_(o1, o2, o3)] = fh[np.ix_(i1, i2, i3)]
    return np.real(np.fft.ifftn(gh) * np.prod(shape_out))

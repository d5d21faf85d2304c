"""Seeded synthetic inputs for the registration problems.

This module only makes input data: images and velocity fields on the grid,
from NumPy's PCG64 generator (``numpy.random.default_rng(seed)``).  It holds
none of the method's arithmetic (no semi-Lagrangian step, no tricubic
interpolation, no operator of the solver), so the FP64 oracle and the CUDA
library can both be fed from it without sharing code.

Problems
--------
* ``sinusoid_problem`` -- the smooth synthetic problem of Sec. IV-A1 in the
  form used here: reference rho_R = (sin^2 x1 + sin^2 x2 + sin^2 x3) / 3 and
  the analytic divergence-free velocity
  v* = s (sin x3 cos x2 sin x2, sin x1 cos x3 sin x3, sin x2 cos x1 sin x1).
  The template is rho_R moved backward along v*: rho_T(x) = rho_R(phi_1(x)),
  with phi_t the flow of v* (d phi / dt = v*(phi), phi_0 = x), integrated
  pointwise with classical RK4 on the analytic formulas.  A forward transport
  of rho_T by v* then returns rho_R, and no grid operator was used to make the
  pair (no inverse crime).
* ``phantom_problem`` -- a brain-like phantom standing in for the NIREP MRI
  volumes of Sec. IV-A1, which are not available here: three nested
  ellipsoids (intensities 0.2 / 0.5 / 0.9, background 0), the template given
  by the same analytic phantom evaluated at x + u(x) for a random band-limited
  displacement u (|k| <= 6, max |u| = 8 voxels), both smoothed by a Gaussian of
  1.5 voxels and given additive N(0, 0.01^2) noise.
* ``bandlimited`` -- random real fields with Fourier support |k|_2 <= kmax and
  unit RMS per component (search directions, test velocities).
* ``phantom_problem_torch`` -- the phantom recipe above in torch on any
  device, seeded through ``torch.Generator`` (a different random stream from
  the NumPy version: same distribution, not the same draws), for the
  thousands of pairs that train the learned initial velocity.
"""

import numpy as np

TWO_PI = 2.0 * np.pi


def grid_coords(shape):
    """Physical coordinates x_j = 2 pi i_j / N_j as three (N1,N2,N3) arrays."""
    axes = [TWO_PI * np.arange(n, dtype=np.float64) / n for n in shape]
    return np.meshgrid(*axes, indexing='ij')


def sin2_image(x1, x2, x3):
    return (np.sin(x1) ** 2 + np.sin(x2) ** 2 + np.sin(x3) ** 2) / 3.0


def vstar_at(x1, x2, x3, scale):
    """The analytic velocity v*(x) (each component free of its own coordinate,
    so div v* = 0 exactly)."""
    return (scale * np.sin(x3) * np.cos(x2) * np.sin(x2),
            scale * np.sin(x1) * np.cos(x3) * np.sin(x3),
            scale * np.sin(x2) * np.cos(x1) * np.sin(x1))


def vstar(shape, scale):
    x = grid_coords(shape)
    return np.stack(vstar_at(*x, scale))


def flow_of_vstar(shape, scale, steps=64):
    """phi_1(x) for every grid point: RK4 on d phi/dt = v*(phi), unit time."""
    p = [c.copy() for c in grid_coords(shape)]
    h = 1.0 / steps
    for _ in range(steps):
        k1 = vstar_at(*p, scale)
        k2 = vstar_at(*[p[j] + 0.5 * h * k1[j] for j in range(3)], scale)
        k3 = vstar_at(*[p[j] + 0.5 * h * k2[j] for j in range(3)], scale)
        k4 = vstar_at(*[p[j] + h * k3[j] for j in range(3)], scale)
        p = [p[j] + (h / 6.0) * (k1[j] + 2 * k2[j] + 2 * k3[j] + k4[j])
             for j in range(3)]
    return p


def sinusoid_problem(shape, scale=0.5):
    """(rho_T, rho_R, v*) for the smooth synthetic problem, float64."""
    rho_R = sin2_image(*grid_coords(shape))
    rho_T = sin2_image(*flow_of_vstar(shape, scale))
    return rho_T, rho_R, vstar(shape, scale)


def bandlimited(shape, kmax, seed, ncomp=3):
    """Real random fields with |k|_2 <= kmax and unit RMS per component.

    Real white noise -> real-to-complex FFT -> keep |k|_2 <= kmax -> inverse,
    so the coefficients are complex normal and Hermitian by construction.
    Returns (ncomp, N1, N2, N3), or (N1, N2, N3) when ncomp is None.
    """
    rng = np.random.default_rng(seed)
    n = 1 if ncomp is None else ncomp
    k1 = np.fft.fftfreq(shape[0], 1.0 / shape[0])[:, None, None]
    k2 = np.fft.fftfreq(shape[1], 1.0 / shape[1])[None, :, None]
    k3 = np.fft.rfftfreq(shape[2], 1.0 / shape[2])[None, None, :]
    mask = (k1 ** 2 + k2 ** 2 + k3 ** 2) <= kmax * kmax
    out = np.empty((n,) + tuple(shape))
    for c in range(n):
        w = rng.standard_normal(shape)
        f = np.fft.irfftn(np.fft.rfftn(w) * mask, s=shape, axes=(0, 1, 2))
        out[c] = f / np.sqrt(np.mean(f * f))
    return out[0] if ncomp is None else out


def _gaussian_blur(f, sigma_vox):
    """Periodic Gaussian blur of sigma_vox voxels (input synthesis only)."""
    shape = f.shape
    k1 = np.fft.fftfreq(shape[0])[:, None, None]
    k2 = np.fft.fftfreq(shape[1])[None, :, None]
    k3 = np.fft.rfftfreq(shape[2])[None, None, :]
    g = np.exp(-0.5 * (TWO_PI * sigma_vox) ** 2 * (k1 ** 2 + k2 ** 2 + k3 ** 2))
    return np.fft.irfftn(np.fft.rfftn(f) * g, s=shape, axes=(0, 1, 2))


def _ellipsoid_params(seed):
    rng = np.random.default_rng(seed)
    centre = np.pi + rng.uniform(-0.05 * np.pi, 0.05 * np.pi, size=3)
    axes = np.array([0.75, 0.85, 0.70]) * np.pi * rng.uniform(0.95, 1.05, size=3)
    return centre, axes


def _phantom_at(x1, x2, x3, centre, axes):
    """Nested ellipsoids: outer shell 0.2, middle 0.5, inner 0.9, else 0."""
    out = np.zeros(np.shape(x1))
    d = [np.mod(c - c0 + np.pi, TWO_PI) - np.pi for c, c0 in zip((x1, x2, x3), centre)]
    for scale, value in ((1.0, 0.2), (0.72, 0.5), (0.45, 0.9)):
        r2 = sum((d[j] / (scale * axes[j])) ** 2 for j in range(3))
        out = np.where(r2 <= 1.0, value, out)
    return out


def phantom_problem(shape, seed, max_disp_vox=8.0, kmax=6, sigma_vox=1.5,
                    noise=0.01):
    """(rho_T, rho_R, u) for the phantom problem, float64.

    u is the band-limited displacement (physical units) used to warp the
    template; the seeds are seed (geometry), seed+1 (u), seed+2 (noise on
    rho_R) and seed+3 (noise on rho_T).
    """
    centre, axes = _ellipsoid_params(seed)
    u = bandlimited(shape, kmax, seed + 1)
    h = TWO_PI / max(shape)
    mag = np.sqrt(np.sum(u * u, axis=0)).max()
    u *= max_disp_vox * h / mag
    x = grid_coords(shape)
    rho_R = _gaussian_blur(_phantom_at(*x, centre, axes), sigma_vox)
    rho_T = _gaussian_blur(_phantom_at(*[x[j] + u[j] for j in range(3)],
                                       centre, axes), sigma_vox)
    if noise > 0:
        rho_R = rho_R + noise * np.random.default_rng(seed + 2).standard_normal(shape)
        rho_T = rho_T + noise * np.random.default_rng(seed + 3).standard_normal(shape)
    return rho_T, rho_R, u


def phantom_problem_torch(shape, seed, device='cpu', max_disp_vox=8.0, kmax=6, sigma_vox=1.5,
                          noise=0.01):
    """(rho_T, rho_R, u) of the phantom recipe as float32 torch tensors on
    `device`: ellipsoid geometry from NumPy's generator at `seed` (as
    ``phantom_problem``), the displacement and the noise from a torch
    generator seeded with `seed`."""
    import torch
    f64 = torch.float64
    centre, axes = _ellipsoid_params(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    n1, n2, n3 = shape
    k1 = torch.fft.fftfreq(n1, 1.0 / n1, dtype=f64, device=device)[:, None, None]
    k2 = torch.fft.fftfreq(n2, 1.0 / n2, dtype=f64, device=device)[None, :, None]
    k3 = torch.fft.rfftfreq(n3, 1.0 / n3, dtype=f64, device=device)[None, None, :]
    mask = (k1 ** 2 + k2 ** 2 + k3 ** 2) <= kmax * kmax
    u = []
    for _ in range(3):
        w = torch.randn(shape, generator=gen, dtype=f64, device=device)
        f = torch.fft.irfftn(torch.fft.rfftn(w) * mask, s=shape)
        u.append(f / torch.sqrt(torch.mean(f * f)))
    u = torch.stack(u)
    u *= max_disp_vox * (TWO_PI / max(shape)) / torch.sqrt(torch.sum(u * u, dim=0)).max()
    ax = [TWO_PI * torch.arange(n, dtype=f64, device=device) / n for n in shape]
    x = torch.meshgrid(*ax, indexing='ij')

    def phantom(p):
        out = torch.zeros(shape, dtype=f64, device=device)
        d = [torch.remainder(p[j] - float(centre[j]) + np.pi, TWO_PI) - np.pi for j in range(3)]
        for scale, value in ((1.0, 0.2), (0.72, 0.5), (0.45, 0.9)):
            r2 = sum((d[j] / (scale * float(axes[j]))) ** 2 for j in range(3))
            out = torch.where(r2 <= 1.0, torch.full_like(out, value), out)
        return out

    g = torch.exp(-0.5 * (TWO_PI * sigma_vox) ** 2 *
                  ((k1 / n1) ** 2 + (k2 / n2) ** 2 + (k3 / n3) ** 2))

    def blur(f):
        return torch.fft.irfftn(torch.fft.rfftn(f) * g, s=shape)

    rho_R = blur(phantom(x))
    rho_T = blur(phantom([x[j] + u[j] for j in range(3)]))
    if noise > 0:
        rho_R = rho_R + noise * torch.randn(shape, generator=gen, dtype=f64, device=device)
        rho_T = rho_T + noise * torch.randn(shape, generator=gen, dtype=f64, device=device)
    return rho_T.float(), rho_R.float(), u.float()

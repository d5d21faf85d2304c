"""Tricubic Lagrange interpolation on the periodic grid (oracle, FP64).

Test infrastructure.  Sec. III-C2 ("Interpolation"): every off-grid value
is built from the 4^3 = 64 grid values around the point.  The paper names the
scheme only "tricubic"; reading: the tensor product of 1-D cubic Lagrange
polynomials on the four nodes {-1, 0, 1, 2} around the cell that holds the
point, with periodic wrap of the grid indices.

Positions are given in grid units: position p_j along axis j means the
physical coordinate p_j * h_j, h_j = 2 pi / N_j.  For p = i + xi with
i = floor(p) and xi in [0, 1):

    value = sum_{a,b,c in {-1,0,1,2}} l_a(xi_1) l_b(xi_2) l_c(xi_3)
                                      f[(i_1+a) mod N_1, (i_2+b) mod N_2, (i_3+c) mod N_3]
"""

import numpy as np

NODES = (-1, 0, 1, 2)


def lagrange_weights(xi):
    """The four cubic Lagrange basis polynomials on nodes -1, 0, 1, 2.

    l_m(xi) = prod_{n != m} (xi - n) / (m - n).  Returns a list of four arrays
    (for nodes -1, 0, 1, 2) with the shape of xi.
    """
    w = []
    for m in NODES:
        num = np.ones_like(xi)
        den = 1.0
        for n in NODES:
            if n != m:
                num = num * (xi - n)
                den = den * (m - n)
        w.append(num / den)
    return w


def interp(field, pos):
    """Interpolate a scalar grid field at positions pos = (p1, p2, p3).

    field: (N1, N2, N3) array.  pos: three arrays of one common shape, in grid
    units (any real value: the periodic wrap is a proper modulo, so points
    more than one cell away, CFL > 1, are fine).
    """
    shape = field.shape
    idx = []
    wts = []
    for j in range(3):
        p = np.asarray(pos[j], dtype=np.float64)
        base = np.floor(p)
        xi = p - base
        base = base.astype(np.int64)
        idx.append([np.mod(base + a, shape[j]) for a in NODES])
        wts.append(lagrange_weights(xi))
    out = np.zeros(np.shape(pos[0]), dtype=np.float64)
    for a in range(4):
        for b in range(4):
            for c in range(4):
                w = wts[0][a] * wts[1][b] * wts[2][c]
                out += w * field[idx[0][a], idx[1][b], idx[2][c]]
    return out


def grid_index(shape):
    """Integer grid coordinates (i1, i2, i3) as float arrays of the grid shape."""
    return np.meshgrid(np.arange(shape[0], dtype=np.float64),
                       np.arange(shape[1], dtype=np.float64),
                       np.arange(shape[2], dtype=np.float64), indexing='ij')


def interp_at_displacement(field, disp):
    """Interpolate a grid field at x_i + disp_i for every grid point.

    disp: (3, N1, N2, N3) displacements in grid units.
    """
    g = grid_index(field.shape)
    return interp(field, (g[0] + disp[0], g[1] + disp[1], g[2] + disp[2]))

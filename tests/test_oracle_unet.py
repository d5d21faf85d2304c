"""Pins for the oracle U-Net (CPU): convolution against a direct loop, and
every backward formula against central finite differences of the forward."""

import numpy as np

from oracle import unet as un


def naive_conv(x, w, b):
    k = w.shape[0]
    p = k // 2
    D, H, W, Ci = x.shape
    Co = w.shape[4]
    y = np.zeros((D, H, W, Co))
    for z in range(D):
        for yy in range(H):
            for xx in range(W):
                acc = b.copy()
                for dz in range(k):
                    for dy in range(k):
                        for dx in range(k):
                            zz, y2, x2 = z + dz - p, yy + dy - p, xx + dx - p
                            if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                acc = acc + x[zz, y2, x2] @ w[dz, dy, dx]
                y[z, yy, xx] = acc
    return y


def test_conv_matches_a_direct_loop():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((4, 5, 3, 2))
    for k in (3, 1):
        w = rng.standard_normal((k, k, k, 2, 3))
        b = rng.standard_normal(3)
        assert np.abs(un.conv(x, w, b) - naive_conv(x, w, b)).max() < 1e-12


def _fd(f, a, eps=1e-6, n=12, seed=1):
    """Central differences of the scalar f at n random entries of a."""
    rng = np.random.default_rng(seed)
    idx = [tuple(rng.integers(0, s) for s in a.shape) for _ in range(n)]
    out = []
    for i in idx:
        old = a[i]
        a[i] = old + eps
        fp = f()
        a[i] = old - eps
        fm = f()
        a[i] = old
        out.append((i, (fp - fm) / (2 * eps)))
    return out


def test_layer_backwards_match_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 4, 4, 3))
    w = rng.standard_normal((3, 3, 3, 3, 2))
    b = rng.standard_normal(2)
    c = rng.standard_normal((4, 4, 4, 2))
    loss = lambda: float(np.sum(un.conv(x, w, b) * c))
    dx, dw, db = un.conv_backward(x, w, c)
    for arr, grad in ((x, dx), (w, dw), (b, db)):
        for i, fd in _fd(loss, arr):
            assert abs(grad[i] - fd) < 1e-6 * max(1.0, abs(fd))
    c2 = rng.standard_normal((2, 2, 2, 3))
    for i, fd in _fd(lambda: float(np.sum(un.avgpool2(x) * c2)), x):
        assert abs(un.avgpool2_backward(c2)[i] - fd) < 1e-8
    c3 = rng.standard_normal((8, 8, 8, 3))
    for i, fd in _fd(lambda: float(np.sum(un.upsample2(x) * c3)), x):
        assert abs(un.upsample2_backward(c3)[i] - fd) < 1e-8


def test_network_gradient_matches_finite_differences():
    ch = (2, 4, 4)
    p = un.init_params(ch, seed=3)
    rng = np.random.default_rng(4)
    for k in p:
        if k.endswith('.b'):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((8, 8, 8, 2))
    t = rng.standard_normal((8, 8, 8, 3))

    def loss():
        y, _ = un.forward(p, x, ch)
        return un.mse(y, t)[0]

    y, cache = un.forward(p, x, ch)
    _, dy = un.mse(y, t)
    g = un.backward(p, cache, dy, ch)
    for name in ('enc0.0.w', 'enc1.1.b', 'enc2.0.w', 'dec1.0.w', 'dec0.1.b', 'head.w'):
        for i, fd in _fd(loss, p[name], n=6, seed=sum(map(ord, name))):
            assert abs(g[name][i] - fd) < 1e-5 * max(1e-3, abs(fd)), (name, i, g[name][i], fd)

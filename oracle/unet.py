"""3-D U-Net for the learned initial velocity (oracle, FP64).  Test infrastructure.

The network maps the image pair (rho_T, rho_R), resampled to an R^3 grid, to a
velocity field on the same grid; the registration solve then starts from the
(spectrally upsampled) prediction.  This module is the plain FP64 reference of
every layer, forward and backward, used to check the CUDA kernels; it follows
the usual definitions and pins itself against finite differences in the
tests.

Layout: activations are channels-last arrays (D, H, W, C).  Convolutions are
3 x 3 x 3 with zero padding 1 (weights (3, 3, 3, Cin, Cout)) or 1 x 1 x 1
(weights (1, 1, 1, Cin, Cout)), bias (Cout,).

Architecture (levels L = len(ch), channels ch = (16, 32, 64, 128)):
  encoder level l:  x -> conv3 -> relu -> conv3 -> relu = skip_l  (-> avgpool2 for l < L)
  decoder level l (from L-1 down to 1): upsample2 (nearest) -> concat(skip_l) ->
                    conv3 -> relu -> conv3 -> relu
  head: conv1 (ch[0] -> 3).
Loss: mean squared error against the target velocity.
"""

import numpy as np


# ------------------------------------------------------------------ layers

def conv(x, w, b):
    """y[z,y,x,o] = b[o] + sum_{dz,dy,dx,i} w[dz,dy,dx,i,o] x[z+dz-p, y+dy-p, x+dx-p, i]."""
    k = w.shape[0]
    p = k // 2
    D, H, W, _ = x.shape
    xp = np.pad(x, ((p, p), (p, p), (p, p), (0, 0)))
    y = np.zeros((D, H, W, w.shape[4])) + b
    for dz in range(k):
        for dy in range(k):
            for dx in range(k):
                y += xp[dz:dz + D, dy:dy + H, dx:dx + W, :] @ w[dz, dy, dx]
    return y


def conv_backward(x, w, dy):
    """Gradients of conv with respect to x, w and b."""
    k = w.shape[0]
    p = k // 2
    D, H, W, _ = x.shape
    xp = np.pad(x, ((p, p), (p, p), (p, p), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dz in range(k):
        for dy_ in range(k):
            for dx in range(k):
                sl = (slice(dz, dz + D), slice(dy_, dy_ + H), slice(dx, dx + W))
                dxp[sl] += dy @ w[dz, dy_, dx].T
                dw[dz, dy_, dx] = np.einsum('zyxi,zyxo->io', xp[sl], dy)
    dx_ = dxp[p:p + D, p:p + H, p:p + W, :]
    return dx_, dw, dy.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(y, dy):
    """y is the relu output."""
    return dy * (y > 0)


def avgpool2(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 0), 2, 1), 2, 2) / 8.0


def upsample2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample2_backward(dy):
    D, H, W, C = dy.shape
    return dy.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def mse(y, t):
    r = y - t
    return float(np.mean(r * r)), 2.0 * r / r.size


# ------------------------------------------------------------------ network

def init_params(ch, cin=2, cout=3, seed=0):
    """He-normal weights, zero biases, as a dict of named arrays."""
    rng = np.random.default_rng(seed)
    p = {}

    def conv_p(name, ci, co, k=3):
        p[name + '.w'] = rng.standard_normal((k, k, k, ci, co)) * np.sqrt(2.0 / (k ** 3 * ci))
        p[name + '.b'] = np.zeros(co)

    L = len(ch)
    prev = cin
    for l in range(L):
        conv_p('enc%d.0' % l, prev, ch[l])
        conv_p('enc%d.1' % l, ch[l], ch[l])
        prev = ch[l]
    for l in range(L - 2, -1, -1):
        conv_p('dec%d.0' % l, ch[l + 1] + ch[l], ch[l])
        conv_p('dec%d.1' % l, ch[l], ch[l])
    conv_p('head', ch[0], cout, k=1)
    return p


def forward(p, x, ch):
    """Returns (y, cache) for x of shape (R, R, R, cin)."""
    L = len(ch)
    cache = {'x': x}
    h = x
    skips = []
    for l in range(L):
        a0 = relu(conv(h, p['enc%d.0.w' % l], p['enc%d.0.b' % l]))
        a1 = relu(conv(a0, p['enc%d.1.w' % l], p['enc%d.1.b' % l]))
        cache['enc%d.in' % l], cache['enc%d.a0' % l], cache['enc%d.a1' % l] = h, a0, a1
        skips.append(a1)
        h = avgpool2(a1) if l < L - 1 else a1
    for l in range(L - 2, -1, -1):
        u = upsample2(h)
        c = np.concatenate([u, skips[l]], axis=3)
        a0 = relu(conv(c, p['dec%d.0.w' % l], p['dec%d.0.b' % l]))
        a1 = relu(conv(a0, p['dec%d.1.w' % l], p['dec%d.1.b' % l]))
        cache['dec%d.in' % l], cache['dec%d.a0' % l], cache['dec%d.a1' % l] = c, a0, a1
        h = a1
    y = conv(h, p['head.w'], p['head.b'])
    cache['head.in'] = h
    return y, cache


def backward(p, cache, dy, ch):
    """Gradients of the loss with respect to every parameter, given dL/dy."""
    L = len(ch)
    g = {}
    dh, g['head.w'], g['head.b'] = conv_backward(cache['head.in'], p['head.w'], dy)
    dskips = [None] * L
    for l in range(0, L - 1):
        a0, a1, c = cache['dec%d.a0' % l], cache['dec%d.a1' % l], cache['dec%d.in' % l]
        d = relu_backward(a1, dh)
        d, g['dec%d.1.w' % l], g['dec%d.1.b' % l] = conv_backward(a0, p['dec%d.1.w' % l], d)
        d = relu_backward(a0, d)
        dc, g['dec%d.0.w' % l], g['dec%d.0.b' % l] = conv_backward(c, p['dec%d.0.w' % l], d)
        cu = ch[l + 1]
        dskips[l] = dc[..., cu:]
        dh = upsample2_backward(dc[..., :cu])
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            dh = avgpool2_backward(dh) + dskips[l]
        a0, a1, h = cache['enc%d.a0' % l], cache['enc%d.a1' % l], cache['enc%d.in' % l]
        d = relu_backward(a1, dh)
        d, g['enc%d.1.w' % l], g['enc%d.1.b' % l] = conv_backward(a0, p['enc%d.1.w' % l], d)
        d = relu_backward(a0, d)
        dh, g['enc%d.0.w' % l], g['enc%d.0.b' % l] = conv_backward(h, p['enc%d.0.w' % l], d)
    return g

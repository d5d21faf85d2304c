"""GPU parity of the learned-initial-velocity path: Fourier resampling and the
3-D U-Net (forward, gradients, Adam) through the C-ABI against the FP64
oracle.

The U-Net runs BF16 weights and activations with FP32 accumulation.  The
oracle gets the same BF16-rounded input and weights and runs in FP64, so the
difference is the rounding of each stored activation and gradient operand to
BF16 (relative 2^-9 per rounding, independent across layers): the forward
output and the loss within 2e-2 relative L2, every parameter gradient within
3e-2 relative L2 (its operands are rounded twice: activation and incoming
gradient).  Adam is FP32 element-wise and is checked at 1e-5 against the
update formula applied to the library's own gradient.
"""

import numpy as np
import pytest

torch = pytest.importorskip('torch')

from oracle import spectral as osp
from oracle import unet as oun

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def reg():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_03630_gb300 import reg as _reg
    return _reg


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device='cuda')


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().double().numpy()


def bf16(a):
    """The BF16 value the tensor cores see, as FP64."""
    t = torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------ resampling

@pytest.mark.parametrize('shapes', [((32, 32, 32), (20, 28, 44)), ((20, 28, 44), (64, 48, 36)),
                                    ((17, 23, 30), (16, 16, 16))])
@pytest.mark.parametrize('ncomp', [1, 3])
def test_resample_matches_oracle(reg, shapes, ncomp):
    a, b = shapes
    rng = np.random.default_rng(11)
    f = rng.standard_normal((ncomp,) + a).astype(np.float32).astype(np.float64)
    got = host(reg.spectral_resample(dev(f), b))
    want = osp.resample(f, b)
    assert rel(got, want) < 1e-5


def test_resample_band_limited_round_trip(reg):
    """Coarse -> fine -> coarse returns a field band-limited below the coarse
    Nyquist (exact in exact arithmetic)."""
    x = 2 * np.pi * np.arange(24) / 24
    x1, x2, x3 = np.meshgrid(x, x, x, indexing='ij')
    f = np.sin(x1) * np.cos(3 * x2) + 0.5 * np.cos(5 * x3 + x1)
    up = reg.spectral_resample(dev(f), (64, 64, 64))
    back = host(reg.spectral_resample(up, (24, 24, 24)))
    assert np.abs(back - f).max() < 1e-5


# ------------------------------------------------------------------ U-Net

CONFIGS = [(16, (8, 16, 32)), (12, (8, 16)), (8, (4,))]


def make_params(net, seed):
    p = oun.init_params(net.channels, net.cin, net.cout, seed=seed)
    rng = np.random.default_rng(seed + 100)
    for k in p:
        if k.endswith('.b'):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    flat = net.pack(p)
    # what the library holds: FP32 master (biases), BF16 copies (weights)
    used = net.unpack(flat.astype(np.float64))
    for k in used:
        if k.endswith('.w'):
            used[k] = bf16(used[k])
    return flat, used


def make_input(R, cin, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((cin, R, R, R)).astype(np.float32)


def oracle_forward(params, x, ch):
    xo = bf16(x).transpose(1, 2, 3, 0)
    y, cache = oun.forward(params, xo, ch)
    return y, cache


@pytest.mark.parametrize('R,ch', CONFIGS)
def test_unet_forward_matches_oracle(reg, R, ch):
    net = reg.UNet(R, ch)
    flat, used = make_params(net, seed=R)
    net.set_params(flat)
    x = make_input(R, 2, seed=R + 1)
    y = host(net.forward(dev(x)))
    want, _ = oracle_forward(used, x, ch)
    assert rel(y, want.transpose(3, 0, 1, 2)) < 2e-2


@pytest.mark.parametrize('tcgen05', [True, False])
def test_unet_forward_full_channels(reg, tcgen05):
    """The four-level 16/32/64/128 network at 32^3 (every GEMM shape of the
    production network: K from 54 to 5184, N from 3 to 128), with the
    forward 3x3x3 convolutions on tcgen05 and on the wmma path."""
    ch = (16, 32, 64, 128)
    net = reg.UNet(32, ch)
    net.set_mma(tcgen05)
    flat, used = make_params(net, seed=5)
    net.set_params(flat)
    x = make_input(32, 2, seed=6)
    y = host(net.forward(dev(x)))
    want, _ = oracle_forward(used, x, ch)
    assert rel(y, want.transpose(3, 0, 1, 2)) < 2e-2


@pytest.mark.parametrize('R', [16, 32])
def test_tcgen05_and_wmma_forward_agree(reg, R):
    """The forward 3x3x3 convolutions with 16..128 output channels run on
    tcgen05 (TMEM accumulator) by default and on the wmma path when told;
    same BF16 operands, FP32 sums in another order: the outputs agree to the
    BF16 rounding of the activations (the 2-channel first layer and the 1x1
    head are on the wmma path either way)."""
    ch = (16, 32, 64, 128) if R == 32 else (16, 32)
    net = reg.UNet(R, ch)
    flat, _ = make_params(net, seed=9)
    net.set_params(flat)
    x = dev(make_input(R, 2, seed=10))
    y_tc = host(net.forward(x))
    net.set_mma(False)
    y_w = host(net.forward(x))
    net.set_mma(True)
    assert np.isfinite(y_tc).all()
    assert rel(y_tc, y_w) < 1e-2


@pytest.mark.parametrize('R,ch', CONFIGS)
def test_unet_gradient_matches_oracle(reg, R, ch):
    net = reg.UNet(R, ch)
    flat, used = make_params(net, seed=R + 7)
    net.set_params(flat)
    x = make_input(R, 2, seed=R + 8)
    t = np.random.default_rng(R + 9).standard_normal((3, R, R, R)).astype(np.float32)
    loss, g = net.gradient(dev(x), dev(t))
    y, cache = oracle_forward(used, x, ch)
    want_loss, dy = oun.mse(y, t.astype(np.float64).transpose(1, 2, 3, 0))
    want = oun.backward(used, cache, dy, ch)
    assert abs(loss - want_loss) < 2e-2 * want_loss
    got = net.unpack(g.astype(np.float64))
    for name, ws, bs in net.layer_shapes():
        for suf in ('.w', '.b'):
            assert rel(got[name + suf], want[name + suf]) < 3e-2, (name + suf)


@pytest.mark.parametrize('tcgen05', [True, False])
def test_unet_gradient_full_channels(reg, tcgen05):
    """Every parameter gradient of the 16/32/64/128 network at 32^3 against
    the oracle, with the data gradients of the layers whose inputs have 16..128
    channels on tcgen05 (the forward convolution of dY with the mirrored
    weights, FP32 out) and with every data gradient on the wmma path."""
    ch = (16, 32, 64, 128)
    net = reg.UNet(32, ch)
    net.set_mma(tcgen05)
    flat, used = make_params(net, seed=21)
    net.set_params(flat)
    x = make_input(32, 2, seed=22)
    t = np.random.default_rng(23).standard_normal((3, 32, 32, 32)).astype(np.float32)
    loss, g = net.gradient(dev(x), dev(t))
    y, cache = oracle_forward(used, x, ch)
    want_loss, dy = oun.mse(y, t.astype(np.float64).transpose(1, 2, 3, 0))
    want = oun.backward(used, cache, dy, ch)
    assert abs(loss - want_loss) < 2e-2 * want_loss
    got = net.unpack(g.astype(np.float64))
    for name, ws, bs in net.layer_shapes():
        for suf in ('.w', '.b'):
            assert rel(got[name + suf], want[name + suf]) < 3e-2, (tcgen05, name + suf)


def test_adam_step_matches_update_formula(reg):
    """train_step recomputes the gradient; the split-K weight gradient sums in
    a run-dependent order, so entries whose gradient is within that noise of
    zero but not exactly zero (where Adam's first step is +-lr by sign) are
    left out."""
    R, ch = 8, (4, 8)
    net = reg.UNet(R, ch)
    flat, _ = make_params(net, seed=21)
    net.set_params(flat)
    x, t = dev(make_input(R, 2, 22)), dev(make_input(R, 3, 23))
    p = net.get_params().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    keep = np.ones(p.shape, dtype=bool)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    for step in (1, 2):
        _, g = net.gradient(x, t)
        g = g.astype(np.float64)
        keep &= (g == 0) | (np.abs(g) > 1e-4 * np.abs(g).max())
        net.train_step(x, t, lr)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        want = p - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
        got = net.get_params().astype(np.float64)
        assert keep.mean() > 0.9
        assert np.abs(got - want)[keep].max() < 1e-5 * max(1.0, np.abs(want).max())
        p = got


def test_training_reduces_loss(reg):
    R, ch = 16, (8, 16)
    net = reg.UNet(R, ch)
    flat, _ = make_params(net, seed=31)
    net.set_params(flat)
    x = dev(make_input(R, 2, 32))
    # a smooth target that the network can fit
    g = np.linspace(0, 2 * np.pi, R, endpoint=False)
    z, yy, xx = np.meshgrid(g, g, g, indexing='ij')
    t = dev(np.stack([np.sin(z), np.cos(yy), np.sin(xx + z)]) * 0.5)
    first = net.train_step(x, t, 3e-3)
    for _ in range(60):
        last = net.train_step(x, t, 3e-3)
    assert np.isfinite(last) and last < 0.5 * first

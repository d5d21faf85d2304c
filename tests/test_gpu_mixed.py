"""Mixed precision: rho_T and rho_R stored in bfloat16, every other field,
interpolation and FFTs in FP32, reductions FP64.

The gradient, objective and stopping test see the bfloat16-rounded images,
so a mixed-precision solve reaches the same stopping test as the FP32 solve
and a final mismatch within the images' rounding (relative 2^-9 ~ 2e-3 per
value).  With images that are already exactly representable in bfloat16, the
gradient and the matvec match the FP64 oracle as closely as the FP32 path.
"""

import numpy as np
import pytest

torch = pytest.importorskip('torch')

from oracle import problem as opr
from oracle import spectral as osp
from paper_1608_03630_gb300 import synth

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


def bf16(a):
    """The bfloat16 value the mixed path stores, as FP64."""
    return torch.tensor(np.asarray(a, np.float32)).bfloat16().double().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_mixed_gradient_is_fp32_accurate_and_matvec_error_is_bounded(reg):
    shape = (32, 32, 32)
    rho_T, rho_R, vs = synth.sinusoid_problem(shape, 0.5)
    rho_T, rho_R = bf16(rho_T), bf16(rho_R)
    vs = np.asarray(vs, np.float32).astype(np.float64)
    P = opr.Problem(rho_T, rho_R, 4, 1e-2, 'H2', False)
    g_ref, J_ref = P.gradient(vs)
    R = reg.Registration(shape, 4, 1e-2, precision='mixed_bf16')
    R.set_images(dev(rho_T), dev(rho_R))
    g, J = R.gradient(dev(vs))
    torch.cuda.synchronize()
    # images are exactly representable (already rounded): the gradient is FP32
    assert abs(J - J_ref) < 1e-5 * abs(J_ref)
    assert rel(g.cpu().double().numpy(), g_ref) < 1e-3
    errs, errs_b = [], []
    for s in range(3):
        w = np.asarray(synth.bandlimited(shape, 8, 1001 + s), np.float32).astype(np.float64)
        h = R.hessian_matvec(dev(w)).cpu().double().numpy()
        h_ref = P.hessian_matvec(w)
        errs.append(rel(h, h_ref))
        # the transport part b~ alone (beta A w is computed exactly in both)
        aw = 1e-2 * osp.apply_regularisation(w, 'H2')
        errs_b.append(rel(h - aw, h_ref - aw))
    print('mixed-precision matvec error vs FP64 oracle: total', ['%.1e' % e for e in errs],
          'transport part', ['%.1e' % e for e in errs_b])
    assert max(errs) < 1e-3
    assert max(errs_b) < 2e-2
    R.close()


def test_mixed_solve_reaches_the_fp32_result(reg):
    shape = (64, 64, 64)
    rho_T, rho_R, _ = synth.phantom_problem(shape, 3000)
    out = {}
    for precision in ('fp32', 'mixed_bf16'):
        R = reg.Registration(shape, 8, 1e-3, precision=precision)
        R.set_images(dev(rho_T), dev(rho_R), presmooth=True)
        v = torch.zeros((3,) + shape, device='cuda')
        status, st = R.solve(v, gtol=1e-2)
        assert status == 0
        out[precision] = (st, v.cpu().double().numpy())
        R.close()
    a, b = out['fp32'][0], out['mixed_bf16'][0]
    assert b['gnorm_rel'] <= 1e-2
    assert abs(a['mismatch_rel'] - b['mismatch_rel']) < 5e-3 * a['mismatch_rel'] + 1e-4
    assert rel(out['mixed_bf16'][1], out['fp32'][1]) < 5e-2

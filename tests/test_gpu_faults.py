"""Error paths under host-side fault injection (reg_debug_inject).

No GPU fault is provoked: the injected failures are a device allocation or
a cuFFT plan that reg_create is told has failed, a NaN written into a
template image, and a TMA-staged interpolation launch told to issue no copy
and to wait for it only briefly, so that its bounded mbarrier waits run out
(nothing is in flight when its blocks exit).  Each test checks the status,
that nothing is left behind, and that the library keeps working afterwards.
"""

import numpy as np
import pytest

torch = pytest.importorskip('torch')

from paper_1608_03630_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPE = (32, 32, 32)


@pytest.fixture(scope='module')
def reg():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_03630_gb300 import reg as _reg
    yield _reg
    _reg.debug_inject('none')


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device='cuda')


def images():
    rho_T, rho_R, _ = synth.sinusoid_problem(SHAPE, 0.5)
    return dev(rho_T), dev(rho_R)


def working_gradient(reg):
    R = reg.Registration(SHAPE, 4, 1e-2)
    rho_T, rho_R = images()
    R.set_images(rho_T, rho_R)
    g, J = R.gradient(torch.zeros((3,) + SHAPE, device='cuda'))
    R.close()
    return np.isfinite(J) and bool(torch.isfinite(g).all())


@pytest.mark.parametrize('kind,after,status', [('alloc', 0, 'REG_ENOMEM'),
                                               ('alloc', 7, 'REG_ENOMEM'),
                                               ('alloc', 16, 'REG_ENOMEM'),
                                               ('cufft_plan', 0, 'REG_ECUFFT'),
                                               ('cufft_plan', 3, 'REG_ECUFFT')])
def test_create_fails_cleanly(reg, kind, after, status):
    assert working_gradient(reg)   # plans and kernels loaded before measuring
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        reg.debug_inject(kind, after)
        with pytest.raises(reg.RegError) as e:
            reg.Registration(SHAPE, 4, 1e-2)
        assert status in str(e.value)
    reg.debug_inject('none')
    torch.cuda.synchronize()
    # everything reg_create had allocated was released (cuFFT may keep a
    # little of its own state)
    assert free0 - torch.cuda.mem_get_info()[0] < 8 << 20
    assert working_gradient(reg)


@pytest.mark.parametrize('precision', ['fp32', 'mixed_bf16'])
def test_nan_image_is_reported_and_the_context_recovers(reg, precision):
    R = reg.Registration(SHAPE, 4, 1e-2, precision=precision)
    rho_T, rho_R = images()
    zero = torch.zeros((3,) + SHAPE, device='cuda')
    reg.debug_inject('nan_image', 0)
    R.set_images(rho_T, rho_R)
    with pytest.raises(reg.RegError) as e:
        R.gradient(zero)
    assert 'REG_ENONFINITE' in str(e.value)
    with pytest.raises(reg.RegError) as e:
        R.solve(zero.clone(), gtol=1e-2)
    assert 'REG_ENONFINITE' in str(e.value)
    # the same context, with clean images, works again
    R.set_images(rho_T, rho_R)
    g, J = R.gradient(zero)
    assert np.isfinite(J) and bool(torch.isfinite(g).all())
    R.close()


def test_bounded_staging_wait_runs_out_and_the_context_stays_usable(reg):
    """x3 = 68 stages the interpolation boxes by TMA copies.  With the copy of
    the next staged launch withheld, every block of that launch gives up its
    wait after ~1e-4 s and writes NaN: the gradient reports REG_ENONFINITE,
    and the next gradient, with nothing armed, equals the clean one."""
    shape = (20, 24, 68)
    rho_T, rho_R, vs = synth.sinusoid_problem(shape, 0.5)
    R = reg.Registration(shape, 4, 1e-3)
    R.set_images(dev(rho_T), dev(rho_R))
    v = dev(vs)
    g_ref, J_ref = R.gradient(v)
    g_ref = g_ref.clone()
    reg.debug_inject('stage_timeout')
    with pytest.raises(reg.RegError) as e:
        R.gradient(v)
    assert e.value.status == 6          # REG_ENONFINITE
    g, J = R.gradient(v)
    torch.cuda.synchronize()
    R.close()
    assert J == J_ref
    assert torch.equal(g, g_ref)

"""The allocation-free state transport (reg_state_transport_noalloc).

Some callers cannot allocate device memory: code inside another library's
callback that must not touch the allocator, programs on a fixed memory pool
that must not grow, and latency-critical loops where a cudaMalloc (which may
synchronise the device) is not acceptable.  For them the library offers a
context-free forward state transport whose intermediate level lives in a
static device array.  Its output must equal the final level of the
ordinary, context-based reg_state_transport on the same inputs, on two calls
in a row (the second call reuses the static array left over from the
first), and a call after the first must leave the device's free memory
unchanged.  This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip('torch')

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


def _case(shape, seed, nt):
    v = 1.5 * synth.bandlimited(shape, 2, seed)
    rho0 = synth.bandlimited(shape, 4, seed + 1, ncomp=None)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device='cuda')
    return dev(rho0), dev(v)


@pytest.mark.parametrize('shape,nt', [((32, 32, 32), 4), ((20, 28, 44), 3)])
def test_noalloc_transport_matches_the_context_path_twice(reg, shape, nt):
    R = reg.Registration(shape, nt, 1e-2)
    for call, seed in enumerate((301, 302)):
        rho0, v = _case(shape, seed, nt)
        d_fwd, _ = R.departure(v)
        expected = R.state_transport(rho0, d_fwd)[nt]
        out = torch.full(shape, float('nan'), device='cuda')
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        reg.state_transport_noalloc(rho0, d_fwd, out, nt, stream=side)
        torch.cuda.synchronize()
        if call > 0:   # the first call may load the library's device code
            assert torch.cuda.mem_get_info()[0] == free_before, call
        err = float((out - expected).norm() / expected.norm())
        assert err < 1e-5, (call, err)
    R.close()


def test_noalloc_rejects_grids_beyond_the_static_level(reg):
    shape = (256, 128, 129)          # 4,227,072 points > 2^22
    with pytest.raises(reg.RegError) as e:
        reg.state_transport_noalloc(torch.zeros(shape, device='cuda'),
                                    torch.zeros((3,) + shape, device='cuda'),
                                    torch.zeros(shape, device='cuda'), 4)
    assert e.value.status == 1     # REG_EINVAL

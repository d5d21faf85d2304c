"""Batched solves of uneven sizes and the tile autotuner.

A batch solves its pairs concurrently on separate streams; each pair's result
must equal the result of solving that pair alone (the per-point arithmetic
does not depend on the tile or on the stream).
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


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device='cuda')


SHAPES = [(32, 32, 32), (24, 40, 36), (48, 48, 48), (32, 36, 28)]


def test_batch_matches_individual_solves(reg):
    pairs = [synth.phantom_problem(s, 4000 + 3 * i) for i, s in enumerate(SHAPES)]
    T = [dev(p[0]) for p in pairs]
    Rr = [dev(p[1]) for p in pairs]
    vs = [torch.zeros((3,) + s, device='cuda') for s in SHAPES]
    B = reg.Batch(SHAPES, 4, 1e-3)
    st, stats, lat = B.solve(vs, T, Rr, presmooth=True, autotune=True, gtol=1e-2)
    B.close()
    assert all(s == 0 for s in st), st
    assert all(l > 0 for l in lat)
    for i, s in enumerate(SHAPES):
        R = reg.Registration(s, 4, 1e-3)
        R.set_images(T[i], Rr[i], presmooth=True)
        v = torch.zeros((3,) + s, device='cuda')
        _, ref = R.solve(v, gtol=1e-2)
        R.close()
        assert stats[i]['gn_iters'] == ref['gn_iters']
        assert abs(stats[i]['J'] - ref['J']) <= 1e-5 * abs(ref['J'])
        err = float((vs[i] - v).norm() / v.norm())
        assert err < 1e-4, (i, err)


def test_autotune_picks_a_valid_tile_and_keeps_results(reg):
    shape = (40, 44, 48)
    rho_T, rho_R, u = synth.phantom_problem(shape, 4100)
    R = reg.Registration(shape, 4, 1e-3)
    R.set_images(dev(rho_T), dev(rho_R), presmooth=True)
    R.gradient(dev(0.5 * u))
    w = dev(synth.bandlimited(shape, 6, 7))
    before = R.hessian_matvec(w).clone()
    k, wy = R.autotune()
    assert k % 4 == 0 and 4 <= k <= 64 and wy in (1, 2, 4, 8, 16)
    after = R.hessian_matvec(w)
    assert float((after - before).norm() / before.norm()) < 1e-5
    R.close()

"""Batched solves of uneven sizes and the tile autotuner.

A batch solves its pairs concurrently on separate streams, in lockstep Newton
steps whose PCG solves form one CUDA graph (a device-controlled loop per
pair), or as whole solves on worker threads; either way each pair's result
must equal the result of solving that pair alone (the per-point arithmetic
does not depend on the tile, the stream or the graph).
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


@pytest.mark.parametrize('one_graph', [True, False])
def test_batch_matches_individual_solves(reg, one_graph):
    pairs = [synth.phantom_problem(s, 4000 + 3 * i) for i, s in enumerate(SHAPES)]
    T = [dev(p[0]) for p in pairs]
    Rr = [dev(p[1]) for p in pairs]
    vs = [torch.zeros((3,) + s, device='cuda') for s in SHAPES]
    B = reg.Batch(SHAPES, 4, 1e-3)
    B.set_mode(one_graph)
    st, stats, lat = B.solve(vs, T, Rr, presmooth=True, autotune=True, gtol=1e-2)
    launched = B.graphs_launched()
    B.close()
    assert all(s == 0 for s in st), st
    assert all(l > 0 for l in lat)
    if one_graph:
        # one PCG graph per lockstep Newton step: as many as the longest solve
        assert launched == max(x['gn_iters'] for x in stats), (launched, stats)
    for i, s in enumerate(SHAPES):
        R = reg.Registration(s, 4, 1e-3)
        R.set_images(T[i], Rr[i], presmooth=True)
        v = torch.zeros((3,) + s, device='cuda')
        _, ref = R.solve(v, gtol=1e-2)
        R.close()
        assert stats[i]['gn_iters'] == ref['gn_iters']
        assert stats[i]['pcg_iters'] == ref['pcg_iters']
        assert abs(stats[i]['J'] - ref['J']) <= 1e-5 * abs(ref['J'])
        err = float((vs[i] - v).norm() / v.norm())
        assert err < 1e-4, (i, err)


def test_batch_graph_is_reused_and_rejects_unsupported_options(reg):
    """A second call with the same pairs and tiles reuses the cached graph
    (same results); continuation and the two-level preconditioner are not
    batch options."""
    shapes = SHAPES[:2]
    pairs = [synth.phantom_problem(s, 4200 + 3 * i) for i, s in enumerate(shapes)]
    T = [dev(p[0]) for p in pairs]
    Rr = [dev(p[1]) for p in pairs]
    B = reg.Batch(shapes, 4, 1e-3)
    out = []
    for _ in range(2):
        vs = [torch.zeros((3,) + s, device='cuda') for s in shapes]
        st, stats, _ = B.solve(vs, T, Rr, presmooth=True, autotune=False, gtol=1e-2)
        out.append((vs, stats))
    for a, b in zip(out[0][0], out[1][0]):
        assert torch.equal(a, b)
    for kw in ({'beta_start': 1e-1}, {'coarse_factor': 2}):
        vs = [torch.zeros((3,) + s, device='cuda') for s in shapes]
        with pytest.raises(reg.RegError):
            B.solve(vs, T, Rr, presmooth=True, autotune=False, gtol=1e-2, **kw)
    B.close()


def test_autotune_picks_a_valid_tile_and_keeps_results(reg):
    shape = (40, 44, 48)
    rho_T, rho_R, u = synth.phantom_problem(shape, 4100)
    R = reg.Registration(shape, 4, 1e-3)
    R.set_images(dev(rho_T), dev(rho_R), presmooth=True)
    R.gradient(dev(0.5 * u))
    w = dev(synth.bandlimited(shape, 6, 7))
    before = R.hessian_matvec(w).clone()
    k, wy = R.autotune()
    assert (k in (1, 2) or (k % 4 == 0 and 4 <= k <= 64)) and wy in (1, 2, 4, 8, 16)
    after = R.hessian_matvec(w)
    assert float((after - before).norm() / before.norm()) < 1e-5
    R.close()

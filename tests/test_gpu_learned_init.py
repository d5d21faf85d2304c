"""The learned initial velocity end to end: training pairs solved by the
library, a short U-Net training run, and the zero-versus-learned solve; and,
with the trained parameters shipped in the package, the gain on held-out
pairs of the 256^3 phantom recipe.

The solve that starts from a prediction stops at the same absolute gradient
norm as the one from v = 0 (gtol times ||g(v = 0)||), so both reach the same
accuracy; the gain is counted in Hessian matvecs.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip('torch')

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       'paper_1608_03630_gb300', 'weights', 'unet_r64.npz')


@pytest.fixture(scope='module')
def li():
    if not torch.cuda.is_available():
        pytest.skip('no CUDA device')
    import __graft_entry__
    __graft_entry__.build()
    from paper_1608_03630_gb300 import learned_init
    return learned_init


def test_pipeline_runs_at_small_size(li):
    from paper_1608_03630_gb300 import reg
    X, V, stats = li.generate(6, 32, 16, seed0=100, chunk=3, log=None)
    assert X.shape == (6, 2, 16, 16, 16) and V.shape == (6, 3, 16, 16, 16)
    assert all(s['status'] == 0 for s in stats)
    assert float(V.abs().max()) > 0
    net = reg.UNet(16, (8, 16))
    net.set_params(li.he_normal(net, seed=1))
    scale = float(torch.sqrt(torch.mean(V * V)))
    hist = li.train(net, X[:4], V[:4], scale, epochs=3, lr=1e-3, val=(X[4:], V[4:]), log=None)
    assert len(hist) == 3 and all(np.isfinite(h['train_loss']) for h in hist)
    ev = li.evaluate(net, scale, [200], 32, stages=2, log=None)
    for name, _, prec in li.ARMS:
        e = ev[0][name]
        assert e['status'] == 0
        assert e['gnorm'] <= 1e-2 * e['gnorm0'] * (1 + 1e-9)
        assert abs(e['gnorm0'] - ev[0]['gnorm_ref']) < 1e-2 * ev[0]['gnorm_ref']
        # the FP32 check of an FP32 solve repeats its own stopping test; a
        # mixed solve (bfloat16 images) lands at the same objective
        if prec == 'fp32':
            assert e['gnorm_rel_fp32'] <= 1e-2 * (1 + 1e-3)
        assert e['J_fp32'] <= ev[0]['plain']['J_fp32'] * 1.01


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason='no trained parameters in the package')
def test_learned_guess_saves_matvecs_on_held_out_pairs(li):
    net, info = li.load(WEIGHTS)
    arms = (('plain', 'zero', 'fp32'), ('learned', 'learned', 'fp32'))
    ev = li.evaluate(net, info['scale'], [7000, 7001, 7002], 256, info['kc'], info['alpha'],
                     arms=arms, stages=info['stages'], log=None)
    zero = sum(e['plain']['matvecs'] for e in ev)
    learned = sum(e['learned']['matvecs'] for e in ev)
    for e in ev:
        assert e['plain']['status'] == 0 and e['learned']['status'] == 0
        # same stopping norm, so the same accuracy
        assert e['learned']['J_fp32'] < 1.02 * e['plain']['J_fp32']
    assert learned < zero, (learned, zero)

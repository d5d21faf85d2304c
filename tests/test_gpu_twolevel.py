"""The two-level (coarse-grid) preconditioner on the GPU against the oracle.

One application M^-1 r (reg_twolevel_apply) at 32^3 with a 16^3 coarse grid,
its inner PCG run for a fixed number of iterations on both sides, against
oracle.precond.TwoLevel on the same FP32-rounded inputs; and Newton solves
with the preconditioner (flexible PCG) that reach the same stopping test and
objective as the one-level solver with fewer fine-grid Hessian matvecs at a
small beta.
"""

import numpy as np
import pytest

torch = pytest.importorskip('torch')

import oracle_jobs
from oracle import precond as opc
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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def host_c(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize('kind,incompressible,beta', [('H2', False, 1e-3), ('H1DIV', True, 1e-3)])
@pytest.mark.parametrize('inner', [1, 3])
@pytest.mark.parametrize('coarse_nt', [0, 2])
def test_two_level_application_matches_the_oracle(reg, kind, incompressible, beta, inner,
                                                  coarse_nt):
    """coarse_nt 0: the coarse Hessian takes the fine nt = 4 steps; 2: its
    own two steps (the form the bench runs, half the fine steps)."""
    shape, coarse, nt = (32, 32, 32), (16, 16, 16), 4
    rho_T, rho_R, _ = [f32(a) for a in synth.sinusoid_problem(shape, 0.5)]
    v = 0.3 * synth.bandlimited(shape, 2, 51)
    r = synth.bandlimited(shape, 12, 52)
    if incompressible:
        v, r = osp.leray(v), osp.leray(r)
    v_hat, v = oracle_jobs.rounded_hat(v)
    r_hat, r = oracle_jobs.rounded_hat(r)
    P = opr.Problem(rho_T, rho_R, nt, beta, kind, incompressible)
    T = opc.TwoLevel(P, coarse, inner_tol=0.0, inner_max=inner, nt_c=coarse_nt or None)
    T.linearize(v)
    z_ref = T.apply(r)
    R = reg.Registration(shape, nt, beta, kind, incompressible)
    R.set_images(torch.tensor(rho_T, dtype=torch.float32, device='cuda'),
                 torch.tensor(rho_R, dtype=torch.float32, device='cuda'))
    R.twolevel_setup(2, torch.tensor(v_hat, device='cuda'), coarse_nt=coarse_nt)
    z, its = R.twolevel_apply(torch.tensor(r_hat, device='cuda'), inner_tol=0.0, inner_max=inner)
    R.close()
    assert its == T.inner_iters == inner
    err = oracle_jobs.rel_hat(host_c(z), oracle_jobs.to_hat(z_ref), shape)
    assert err < 1e-4 * 3 ** inner, err   # FP32 Krylov rounding grows with the iterations
    # the coarse part matters: the plain spectral preconditioner differs
    z1 = osp.preconditioner(r, beta, kind, incompressible)
    assert oracle_jobs.rel_hat(host_c(z), oracle_jobs.to_hat(z1), shape) > 1e-2


def test_two_level_solve_reaches_the_same_stop_with_fewer_matvecs(reg):
    shape, nt = (64, 64, 64), 4
    rho_T, rho_R, _ = synth.phantom_problem(shape, 3000)
    dT = torch.tensor(rho_T, dtype=torch.float32, device='cuda')
    dR = torch.tensor(rho_R, dtype=torch.float32, device='cuda')
    res = {}
    for beta in (1e-3, 1e-5):
        R = reg.Registration(shape, nt, beta, 'H2', False)
        R.set_images(dT, dR, presmooth=True)
        for cf in (0, 2):
            v = torch.zeros((3,) + shape, device='cuda')
            s, st = R.solve(v, gtol=1e-2, coarse_factor=cf, coarse_tol=0.1, coarse_max=20)
            assert s == 0 and st['gnorm_rel'] <= 1e-2, (beta, cf, st)
            res[beta, cf] = st
        R.close()
    for beta in (1e-3, 1e-5):
        one, two = res[beta, 0], res[beta, 2]
        # both stop at ||g|| <= 1e-2 ||g_0||; under the quadratic model the
        # gap to the minimum is g^T H^-1 g / 2 against g_0^T H^-1 g_0 / 2 at
        # v = 0, a small fraction of the decrease J_0 - J (1e-4 when g and
        # g_0 point alike, more when g is left in low-curvature modes)
        gap = 1e-2 * (one['J0'] - one['J'])
        assert abs(two['J'] - one['J']) < gap, (beta, one['J0'], one['J'], two['J'])
        assert two['coarse_matvecs'] > 0 and one['coarse_matvecs'] == 0
    # at the small beta the coarse grid carries the ill-conditioned low modes
    assert res[1e-5, 2]['matvecs'] < res[1e-5, 0]['matvecs'], (res[1e-5, 0], res[1e-5, 2])


def test_coarse_tile_fixed_or_autotuned(reg):
    """The coarse grid's tile is autotuned unless set; a set tile is used as
    given and gives the same solve up to the FP32 order of the stencil sums."""
    shape, nt = (64, 64, 64), 4
    rho_T, rho_R, _ = synth.phantom_problem(shape, 3000)
    dT = torch.tensor(rho_T, dtype=torch.float32, device='cuda')
    dR = torch.tensor(rho_R, dtype=torch.float32, device='cuda')
    out = []
    for tile in (None, (4, 8)):
        R = reg.Registration(shape, nt, 1e-3, 'H2', False)
        assert R.get_coarse_tile() == (0, 0)
        with pytest.raises(reg.RegError):
            R.set_coarse_tile(3, 8)
        if tile:
            R.set_coarse_tile(*tile)
        R.set_images(dT, dR, presmooth=True)
        v = torch.zeros((3,) + shape, device='cuda')
        s, st = R.solve(v, gtol=1e-2, coarse_factor=2, coarse_tol=0.1, coarse_max=20)
        assert s == 0
        got = R.get_coarse_tile()
        if tile:
            assert got == tile
        else:
            assert got[0] in (1, 2, 4, 8, 16) and got[1] in (4, 8, 16), got
        out.append((v.cpu().numpy(), st))
        R.close()
    (v0, s0), (v1, s1) = out
    assert s0['gn_iters'] == s1['gn_iters']
    assert np.linalg.norm(v1 - v0) <= 1e-3 * np.linalg.norm(v0)


def test_dependent_launches_change_nothing(reg):
    """With programmatic dependent launches (the default) every kernel still
    waits on the device for its predecessor's results: a two-level solve
    (fine and coarse PCG graphs) gives the same iterates bit for bit as with
    ordinary launches."""
    shape, nt = (64, 64, 64), 4
    rho_T, rho_R, _ = synth.phantom_problem(shape, 3100)
    dT = torch.tensor(rho_T, dtype=torch.float32, device='cuda')
    dR = torch.tensor(rho_R, dtype=torch.float32, device='cuda')
    out = []
    try:
        for on in (False, True):
            reg.set_dependent_launch(on)
            R = reg.Registration(shape, nt, 1e-3, 'H2', False)
            R.set_coarse_tile(2, 8)
            R.set_images(dT, dR, presmooth=True)
            v = torch.zeros((3,) + shape, device='cuda')
            s, st = R.solve(v, gtol=1e-2, coarse_factor=2, coarse_tol=0.1, coarse_max=20)
            assert s == 0
            out.append((v.cpu().numpy(), st))
            R.close()
    finally:
        reg.set_dependent_launch(True)
    (v0, s0), (v1, s1) = out
    assert s0['pcg_iters'] == s1['pcg_iters'] and s0['coarse_matvecs'] == s1['coarse_matvecs']
    assert np.array_equal(v0, v1)
    assert reg.lib().reg_set_dependent_launch(2) == 1   # REG_EINVAL

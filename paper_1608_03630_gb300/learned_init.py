"""Learned initial velocity: training pairs made by the solver, U-Net training,
and the zero-versus-learned comparison of the Gauss-Newton-Krylov solve.

Everything numeric runs in the library (libreg.so): the phantom pairs are
solved by ``reg.Batch`` (each PCG iteration a CUDA graph), images and
velocities change grids by ``reg.spectral_resample`` (Fourier truncation /
zero padding), and the network trains and predicts through ``reg.UNet``
(BF16 tensor-core kernels).  torch holds the tensors and makes the seeded
synthetic phantoms.

Recipe (one continuous problem sampled at every grid): phantom pairs with a
band-limited displacement of at most 8 voxels of the 256^3 grid (in
physical units, the same at every grid) and Gaussian image blur of 1.5 such
voxels;
H2 regularisation, beta = 1e-3, nt = 8.  Training pairs are generated and
solved at ``gen`` points per axis; the network input is (rho_T, rho_R) and its
target the solution velocity, both resampled to ``res`` points per axis and
the target divided by a fixed scale (the RMS of the training velocities).  The
prediction keeps only the Fourier modes |k_j| < kc and is multiplied by alpha,
(kc, alpha) chosen on pairs of their own by the objective J(v0) / J(0).  A
held-out pair at the evaluation grid is solved twice, from v = 0 and from the
upsampled prediction, both to ||g|| <= gtol ||g(v = 0)||, so both stop at the
same absolute gradient norm.

Command line: ``python -m paper_1608_03630_gb300.learned_init --help``.
"""

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import reg, synth

TWO_PI = 2.0 * math.pi
DISP_VOX_256 = 8.0
SIGMA_VOX_256 = 1.5


def phantom(n, seed, device='cuda'):
    """The phantom pair at n^3 with the displacement and blur of the 256^3
    recipe expressed in physical units."""
    s = n / 256.0
    return synth.phantom_problem_torch((n, n, n), seed, device=device,
                                       max_disp_vox=DISP_VOX_256 * s,
                                       sigma_vox=SIGMA_VOX_256 * s)


def net_input(rho_T, rho_R, res):
    x = torch.stack([rho_T, rho_R]).contiguous()
    if x.shape[1] != res:
        x = reg.spectral_resample(x, (res, res, res))
    return x.contiguous()


def band_limit(v, kc, res):
    """v (3, m^3) keeping the Fourier modes |k_j| < kc, on the res^3 grid."""
    if kc is not None and 2 * kc < v.shape[1]:
        v = reg.spectral_resample(v, (2 * kc,) * 3)
    if v.shape[1] != res:
        v = reg.spectral_resample(v, (res,) * 3)
    return v


def generate(n_pairs, gen, res, seed0, nt=8, beta=1e-3, chunk=16, target_kc=None, log=print):
    """Solve n_pairs phantom pairs at gen^3; returns (X, V, stats): X the
    network inputs (n, 2, res^3), V the solutions resampled to res^3
    (n, 3, res^3; only the modes |k_j| < target_kc if given), stats one dict
    per pair."""
    X = torch.empty((n_pairs, 2, res, res, res), device='cuda')
    V = torch.empty((n_pairs, 3, res, res, res), device='cuda')
    shape = (gen, gen, gen)
    stats = []
    t0 = time.perf_counter()
    batch = None
    for c0 in range(0, n_pairs, chunk):
        m = min(chunk, n_pairs - c0)
        if batch is None or len(batch.shapes) != m:
            if batch is not None:
                batch.close()
            batch = reg.Batch([shape] * m, nt, beta, 'H2')
        pairs = [phantom(gen, seed0 + c0 + i) for i in range(m)]
        rts = [p[0].contiguous() for p in pairs]
        rrs = [p[1].contiguous() for p in pairs]
        vs = [torch.zeros((3,) + shape, device='cuda') for _ in range(m)]
        st, ss, _ = batch.solve(vs, rts, rrs, presmooth=True, autotune=False)
        for i in range(m):
            X[c0 + i] = net_input(rts[i], rrs[i], res)
            V[c0 + i] = band_limit(vs[i], target_kc, res)
            ss[i]['status'] = st[i]
            ss[i]['seed'] = seed0 + c0 + i
            stats.append(ss[i])
        if log and (c0 // chunk) % 10 == 0:
            log('generate %d/%d  %.1f s' % (c0 + m, n_pairs, time.perf_counter() - t0))
    if batch is not None:
        batch.close()
    torch.cuda.synchronize()
    return X, V, stats


def conv_flops(net):
    """(forward, training step) FLOPs of one sample: 2 V k^3 cin cout per
    convolution forward; a training step adds the weight gradient of every
    convolution and the data gradient of every one but the first."""
    fwd = 0.0
    first = 0.0
    for name, ws, _ in net.layer_shapes():
        lvl = 0 if name == 'head' else int(name[3:name.index('.')])
        vox = (net.R >> lvl) ** 3
        f = 2.0 * vox * ws[0] * ws[1] * ws[2] * ws[3] * ws[4]
        fwd += f
        if name == 'enc0.0':
            first = f
    return fwd, 3.0 * fwd - first


def time_unet(net, reps=20):
    """Device time (ms) of one forward and one training step at the network
    grid, CUDA events on the current stream, after warm-up."""
    x = torch.rand((net.cin,) + (net.R,) * 3, device='cuda')
    t = torch.rand((net.cout,) + (net.R,) * 3, device='cuda')
    out = {}
    saved = net.get_params()
    for what in ('forward', 'train_step'):
        fn = (lambda: net.forward(x)) if what == 'forward' else \
            (lambda: net.train_step(x, t, 1e-12, want_loss=False))
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[what + '_ms'] = e0.elapsed_time(e1) / reps
    net.set_params(saved)
    f, b = conv_flops(net)
    out['forward_tflops'] = f / out['forward_ms'] * 1e-9
    out['train_step_tflops'] = b / out['train_step_ms'] * 1e-9
    return out


def train(net, X, V, scale, epochs, lr, seed=0, val=None, budget_s=None, log=print):
    """Adam on the mean squared error of net(x) against v / scale, one pair
    per step, shuffled each epoch, learning rate on a cosine from lr down to
    lr / 10.  With budget_s, the number of epochs is the most that fit in that
    many seconds at the step time measured on the first pairs (at most
    `epochs`).  Returns the per-epoch history."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    hist = []
    if budget_s is not None:
        k = min(32, n)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for i in range(k):
            net.train_step(X[i], (V[i] / scale).contiguous(), 1e-12, want_loss=False)
        torch.cuda.synchronize()
        per = (time.perf_counter() - t) / k
        epochs = max(1, min(epochs, int(budget_s / (per * n))))
        if log:
            log('train: %.2f ms per step -> %d epochs of %d pairs' % (per * 1e3, epochs, n))
    total = epochs * n
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = rng.permutation(n)
        acc, cnt = 0.0, 0
        for i in order:
            frac = step / max(total - 1, 1)
            cur = lr * (0.1 + 0.9 * 0.5 * (1 + math.cos(math.pi * frac)))
            want = (step % 8) == 0
            loss = net.train_step(X[i], (V[i] / scale).contiguous(), cur, want_loss=want)
            if want:
                acc += loss
                cnt += 1
            step += 1
        rec = {'epoch': ep + 1, 'train_loss': acc / max(cnt, 1),
               'seconds': time.perf_counter() - t0}
        if val is not None:
            Xv, Vv = val
            vl, vz = [], []
            for j in range(Xv.shape[0]):
                y = net.forward(Xv[j])
                vl.append(float(torch.mean((y - Vv[j] / scale) ** 2)))
                vz.append(float(torch.mean((Vv[j] / scale) ** 2)))
            rec['val_loss'] = float(np.mean(vl))
            rec['val_loss_zero'] = float(np.mean(vz))
        hist.append(rec)
        if log:
            log('epoch %d  %s' % (ep + 1, json.dumps(rec)))
    return hist


def predict(net, scale, rho_T, rho_R, n, kc=None, alpha=1.0, stages=1, ctx=None):
    """Initial velocity at n^3: the network at its grid, times alpha * scale,
    keeping the Fourier modes |k_j| < kc (the H2-regularised solutions carry
    almost all their energy there; the network's error outside them would
    cost beta |k|^4 in the objective), resampled to n^3.  stages > 1 (ctx: a
    reg.Registration at n^3): the template is transported by the guess so
    far and the network's prediction for (transported template, rho_R) is
    added, a first-order correction of the remaining deformation."""
    y = net.forward(net_input(rho_T, rho_R, net.R))
    y.mul_(alpha * scale)
    v = band_limit(y, kc, n).contiguous()
    for _ in range(stages - 1):
        d_fwd, _ = ctx.departure(v)
        rho1 = ctx.state_transport(rho_T, d_fwd)[-1].contiguous()
        y = net.forward(net_input(rho1, rho_R, net.R))
        y.mul_(alpha * scale)
        v = (v + band_limit(y, kc, n)).contiguous()
    return v


def select_cutoff(net, scale, seeds, n, cutoffs=(4, 6, 8, 12, 16, 32), alphas=(0.6, 0.8, 1.0),
                  stage_options=(1, 2, 3), nt=8, beta=1e-3, log=print):
    """The (kc, alpha) with the smallest mean J(v0) / J(0) over the pairs
    `seeds` at n^3 (pairs used for nothing else), then the number of stages
    at that (kc, alpha).  Returns ((kc, alpha, stages), table)."""
    shape = (n, n, n)
    ctx = reg.Registration(shape, nt, beta, 'H2')
    table, stab = {}, {}
    pairs = []
    for seed in seeds:
        rho_T, rho_R, _ = phantom(n, seed)
        pairs.append((rho_T.contiguous(), rho_R.contiguous()))
    j0s = []
    for rho_T, rho_R in pairs:
        ctx.set_images(rho_T, rho_R, presmooth=True)
        j0 = ctx.objective(torch.zeros((3,) + shape, device='cuda'))
        j0s.append(j0)
        for kc in cutoffs:
            base = predict(net, scale, rho_T, rho_R, n, kc, 1.0)
            for a in alphas:
                table.setdefault((kc, a), []).append(ctx.objective((a * base).contiguous()) / j0)
    mean = {k: float(np.mean(v)) for k, v in table.items()}
    kc, alpha = min(mean, key=mean.get)
    for (rho_T, rho_R), j0 in zip(pairs, j0s):
        ctx.set_images(rho_T, rho_R, presmooth=True)
        for st in stage_options:
            v = predict(net, scale, rho_T, rho_R, n, kc, alpha, st, ctx)
            stab.setdefault(st, []).append(ctx.objective(v) / j0)
    smean = {k: float(np.mean(v)) for k, v in stab.items()}
    stages = min(smean, key=smean.get)
    ctx.close()
    if log:
        log('J(v0)/J(0) by (kc, alpha): ' +
            ', '.join('%s: %.3f' % (k, v) for k, v in sorted(mean.items())))
        log('J(v0)/J(0) by stages at (%s, %.2f): ' % (kc, alpha) +
            ', '.join('%d: %.3f' % (k, v) for k, v in sorted(smean.items())))
    out = {'%d,%.2f' % k: v for k, v in mean.items()}
    out.update({'stages %d' % k: v for k, v in smean.items()})
    return (kc, alpha, stages), out


ARMS = (('plain', 'zero', 'fp32'), ('learned_fp32', 'learned', 'fp32'),
        ('mixed', 'zero', 'mixed_bf16'), ('learned_mixed', 'learned', 'mixed_bf16'))


def twolevel_arms(factor):
    """The arms again with the two-level preconditioner (coarse grid n /
    factor): solver options as the fourth element of an arm."""
    opts = {'coarse_factor': factor, 'coarse_tol': 0.2, 'coarse_max': 12, 'coarse_nt': 4}
    return tuple((name + '_twolevel', init, prec, opts) for name, init, prec in ARMS)


def evaluate(net, scale, seeds, n, kc=None, alpha=1.0, nt=8, beta=1e-3, gtol=1e-2,
             arms=ARMS, stages=1, log=print):
    """Each arm (name, initial guess 'zero' | 'learned', precision) solves the
    held-out pairs at n^3 to ||g|| <= gtol ||g(0)||, g(0) the gradient at
    v = 0 (closed form, in the arm's precision).  Per arm and pair: the solver's statistics, the wall time from the
    images on the device to the solution (network, resampling and solve), and
    the final v checked in FP32 (J_fp32, gnorm_rel_fp32: J and ||g|| / ||g(0)||
    of the FP32 context at v, the gradient taken on Fourier coefficients as in
    the solver -- a physical-space FP32 gradient carries rounding noise
    amplified by beta |k|^4, near 6 % of ||g(0)|| at 256^3)."""
    shape = (n, n, n)
    ctxs = {p: reg.Registration(shape, nt, beta, 'H2', precision=p)
            for p in sorted({a[2] for a in arms} | {'fp32'})}
    c32 = ctxs['fp32']
    arms = [tuple(a) + ({},) if len(a) == 3 else tuple(a) for a in arms]
    out = []
    for seed in seeds:
        rho_T, rho_R, _ = phantom(n, seed)
        rho_T, rho_R = rho_T.contiguous(), rho_R.contiguous()
        for c in ctxs.values():
            c.set_images(rho_T, rho_R, presmooth=True)
        rec = {'seed': int(seed)}
        for name, init, prec, extra in arms:
            ctx = ctxs[prec]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if init == 'zero':
                v = torch.zeros((3,) + shape, device='cuda')
            else:
                v = predict(net, scale, rho_T, rho_R, n, kc, alpha, stages, ctx)
            s, st = ctx.solve(v, gtol=gtol, gnorm_ref=-1.0, **extra)   # relative to ||g(0)||
            torch.cuda.synchronize()
            st['seconds'] = time.perf_counter() - t0
            st['status'] = s
            # the final v checked by the FP32 context: a solve with no Newton
            # step evaluates J and the (spectral) gradient norm at v
            _, chk = c32.solve(v.clone(), max_gn=0, gnorm_ref=-1.0)
            st['J_fp32'] = chk['J']
            st['gnorm_rel_fp32'] = chk['gnorm_rel']
            rec[name] = st
        rec['gnorm_ref'] = rec[arms[0][0]]['gnorm0']
        out.append(rec)
        if log:
            log('eval seed %d: ' % seed + ' | '.join(
                '%s gn %d mv %d %.3f s J %.5e' % (name, rec[name]['gn_iters'],
                                                  rec[name]['matvecs'], rec[name]['seconds'],
                                                  rec[name]['J_fp32'])
                for name, _, _, _ in arms))
    for c in ctxs.values():
        c.close()
    return out


def summarise(evals, arms=ARMS):
    keys = ('gn_iters', 'pcg_iters', 'matvecs', 'coarse_matvecs', 'seconds', 'mismatch_rel',
            'gnorm_rel', 'J_fp32', 'gnorm_rel_fp32')
    return {a[0]: {k: float(np.mean([e[a[0]][k] for e in evals])) for k in keys}
            for a in arms}


def he_normal(net, seed):
    """Flat initial parameters: weights N(0, 2 / (k^3 cin)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for _, ws, bs in net.layer_shapes():
        fan_in = ws[0] * ws[1] * ws[2] * ws[3]
        parts.append((rng.standard_normal(ws) * math.sqrt(2.0 / fan_in)).reshape(-1))
        parts.append(np.zeros(bs).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def save_params(path, net, scale, meta, kc=None, alpha=1.0, stages=1):
    np.savez(path, params=net.get_params().astype(np.float16), scale=np.float64(scale),
             channels=np.array(net.channels), res=np.int64(net.R),
             kc=np.int64(0 if kc is None else kc), alpha=np.float64(alpha),
             stages=np.int64(stages), meta=np.array(json.dumps(meta)))


def load(path):
    """(net, info) from save_params' file: a reg.UNet holding the trained
    parameters and {'scale', 'kc', 'alpha', 'meta'} for predict()."""
    d = np.load(path)
    net = reg.UNet(int(d['res']), tuple(int(c) for c in d['channels']))
    net.set_params(d['params'].astype(np.float32))
    kc = int(d['kc']) if 'kc' in d and int(d['kc']) > 0 else None
    alpha = float(d['alpha']) if 'alpha' in d else 1.0
    stages = int(d['stages']) if 'stages' in d else 1
    return net, {'scale': float(d['scale']), 'kc': kc, 'alpha': alpha, 'stages': stages,
                 'meta': json.loads(str(d['meta']))}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split('\n\n')[0])
    ap.add_argument('--pairs', type=int, default=2000)
    ap.add_argument('--val', type=int, default=32)
    ap.add_argument('--gen', type=int, default=128, help='grid of the training solves')
    ap.add_argument('--res', type=int, default=64, help='network grid')
    ap.add_argument('--channels', default='16,32,64,128')
    ap.add_argument('--target-kc', type=int, default=None,
                    help='train on targets keeping only the modes |k_j| < this')
    ap.add_argument('--epochs', type=int, default=8, help='at most this many epochs')
    ap.add_argument('--budget', type=float, default=None,
                    help='training seconds (fewer epochs if they do not fit)')
    ap.add_argument('--lr', type=float, default=1e-3)
    ap.add_argument('--eval', type=int, default=50)
    ap.add_argument('--eval-n', type=int, default=256)
    ap.add_argument('--select', type=int, default=8,
                    help='pairs (at the evaluation grid) that choose the cutoff and scale')
    ap.add_argument('--select-seed', type=int, default=7300)
    ap.add_argument('--stages', type=int, default=0,
                    help='prediction stages (0: the stored or selected number)')
    ap.add_argument('--eval-large', type=int, default=0, help='grid of one more held-out pair')
    ap.add_argument('--eval-large-seed', type=int, default=7100)
    ap.add_argument('--train-seed', type=int, default=5000)
    ap.add_argument('--val-seed', type=int, default=7200)
    ap.add_argument('--eval-seed', type=int, default=7000)
    ap.add_argument('--out', default='learned_init_out')
    ap.add_argument('--load', default=None, help='skip training: evaluate these parameters')
    ap.add_argument('--twolevel', type=int, default=0,
                    help='also evaluate every arm with the two-level preconditioner '
                         '(coarse grid n / this)')
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)
    logf = open(os.path.join(a.out, 'log.txt'), 'a')

    def log(msg):
        print(msg, flush=True)
        logf.write(msg + '\n')
        logf.flush()

    report = {'args': vars(a)}
    meta, info = {}, None
    if a.load:
        net, info = load(a.load)
        scale, meta = info['scale'], info['meta']
    else:
        ch = tuple(int(c) for c in a.channels.split(','))
        t0 = time.perf_counter()
        X, V, gstats = generate(a.pairs, a.gen, a.res, a.train_seed, target_kc=a.target_kc,
                                log=log)
        Xv, Vv, _ = generate(a.val, a.gen, a.res, a.val_seed, target_kc=a.target_kc, log=None)
        report['generate_seconds'] = time.perf_counter() - t0
        report['generate'] = {
            'converged': int(sum(1 for s in gstats if s['status'] == 0)),
            'mean_gn': float(np.mean([s['gn_iters'] for s in gstats])),
            'mean_matvecs': float(np.mean([s['matvecs'] for s in gstats]))}
        Xt, Vt = X, V
        scale = float(torch.sqrt(torch.mean(Vt * Vt)))
        net = reg.UNet(a.res, ch)
        net.set_params(he_normal(net, seed=1))
        t0 = time.perf_counter()
        report['unet_timing'] = time_unet(net)
        log('unet timing ' + json.dumps(report['unet_timing']))
        report['history'] = train(net, Xt, Vt, scale, a.epochs, a.lr,
                                  val=(Xv, Vv), budget_s=a.budget, log=log)
        report['train_seconds'] = time.perf_counter() - t0
        epochs = len(report['history'])
        report['train_steps'] = epochs * a.pairs
        meta = {'pairs': a.pairs, 'gen': a.gen, 'epochs': epochs, 'train_seed': a.train_seed,
                'target_kc': a.target_kc}
        save_params(os.path.join(a.out, 'unet_r%d.npz' % a.res), net, scale, meta)
        del X, V, Xt, Vt, Xv, Vv
        torch.cuda.empty_cache()
    report['scale'] = scale
    kc, alpha, stages = (info['kc'], info['alpha'], info['stages']) if a.load else (None, 1.0, 1)
    if a.select > 0:
        (kc, alpha, stages), table = select_cutoff(
            net, scale, range(a.select_seed, a.select_seed + a.select), a.eval_n, log=log)
        report['select'] = {'kc': kc, 'alpha': alpha, 'stages': stages, 'J_ratio': table}
        save_params(os.path.join(a.out, 'unet_r%d.npz' % net.R), net, scale, meta, kc, alpha,
                    stages)
    if a.stages:
        stages = a.stages
    arms = ARMS + (twolevel_arms(a.twolevel) if a.twolevel else ())
    if a.eval > 0:
        ev = evaluate(net, scale, range(a.eval_seed, a.eval_seed + a.eval), a.eval_n, kc, alpha,
                      stages=stages, arms=arms, log=log)
        report['eval'] = ev
        report['eval_summary'] = summarise(ev, arms)
        log('summary ' + json.dumps(report['eval_summary']))
    if a.eval_large > 0:
        ev = evaluate(net, scale, [a.eval_large_seed], a.eval_large, kc, alpha, stages=stages,
                      arms=arms, log=log)
        report['eval_large'] = ev
        report['eval_large_summary'] = summarise(ev, arms)
        log('summary large ' + json.dumps(report['eval_large_summary']))
    with open(os.path.join(a.out, 'report.json'), 'w') as f:
        json.dump(report, f, indent=1)
    return report


if __name__ == '__main__':
    main()

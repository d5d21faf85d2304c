"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks (one
process each, 127.0.0.1), the max-over-ranks time every rank receives, the
rank / world read from the environment, and the reference arm's rule that
only rank 0 runs and prints."""

import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip('torch')

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group('gloo', rank=rank, world_size=world)
    w, r, lr = bench.dist_env()
    got = bench.max_over_ranks(10.0 + 3.0 * rank, w)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, got))


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context('spawn')
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 13.0), (1, 2, 1, 13.0)]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5, 1) == 4.5


def test_reference_arm_prints_on_rank_zero_only():
    """Rank 1 of the reference arm exits 0 without work or output."""
    env = dict(os.environ, RANK='1', WORLD_SIZE='2', LOCAL_RANK='1', MASTER_ADDR='127.0.0.1',
               MASTER_PORT=str(free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference',
                        '--gpus', '2', '--steps', '1', '--warmup', '0'],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ''


def _fake_solve(i, shape):
    """A stand-in for one pair's solve: deterministic statistics of the pair."""
    return {'matvecs': 3 * i + shape[0] // 32, 'gn_iters': 1 + i % 4, 'pair': i}


def _partition_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group('gloo', rank=rank, world_size=world)
    shapes = bench.batch_workload(48)
    costs = [float(s[0] ** 3 * 4) for s in shapes]
    mine = bench.partition_pairs(costs, world)[rank]
    res = [_fake_solve(i, shapes[i]) for i in mine]
    merged = bench.merge_rank_results(bench.gather_objects((mine, res), world), len(shapes))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, merged))


def test_partition_covers_every_pair_once_within_the_load_bound():
    import bench
    shapes = bench.batch_workload(48)
    costs = [float(s[0] ** 3 * 4) for s in shapes]
    for world in (1, 2, 3, 4, 8):
        parts = bench.partition_pairs(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(48))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)
    with pytest.raises(ValueError):
        bench.merge_rank_results([([0, 1], ['a', 'b']), ([1], ['c'])], 2)
    with pytest.raises(ValueError):
        bench.merge_rank_results([([0], ['a'])], 2)


def test_two_gloo_ranks_solve_disjoint_shares_and_merge_like_one_rank():
    """Each rank solves its share of the batch (no data-path collective);
    the host gathers the statistics, and the merged result equals the
    single-rank run pair by pair."""
    import bench
    ctx = torch.multiprocessing.get_context('spawn')
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shapes = bench.batch_workload(48)
    single = [_fake_solve(i, s) for i, s in enumerate(shapes)]
    assert set(out[0][1]).isdisjoint(out[1][1])
    assert sorted(out[0][1] + out[1][1]) == list(range(48))
    assert out[0][2] == single and out[1][2] == single

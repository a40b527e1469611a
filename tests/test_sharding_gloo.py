"""Multi-rank path on CPU: world_size-2 gloo process group, trajectory ranges
disjoint and complete, counts summed by the collective equal to the
single-process totals."""
import os
import socket

import numpy as np
import pytest

from paper_2511_05719_gb300.sharding import trajectory_range, combine_counts

torch = pytest.importorskip("torch")


def test_trajectory_ranges_partition():
    for n in (0, 1, 7, 64, 1001):
        for w in (1, 2, 3, 8):
            got = [trajectory_range(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c and b >= a
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        trajectory_range(10, 2, 2)


def _fake_fail(traj):
    # host stand-in for a trajectory outcome: depends only on the index
    x = (traj * 0x9E3779B1) & 0xFFFFFFFF
    return 2 if x % 97 == 0 else (1 if x % 7 == 0 else 0)


def _worker(rank, world, port, n_total, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = trajectory_range(n_total, rank, world)
    f = np.array([_fake_fail(t) for t in range(a, b)])
    res = combine_counts(int((f == 1).sum()), int((f != 2).sum()))
    q.put((rank, a, b, res))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_gloo_two_ranks_sum_counts():
    import torch.multiprocessing as mp
    n_total, world = 1001, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_total, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f = np.array([_fake_fail(t) for t in range(n_total)])
    nf, nv = int((f == 1).sum()), int((f != 2).sum())
    for rank, a, b, (p_l, sigma, gf, gv) in out:
        assert (gf, gv) == (nf, nv)
        assert abs(p_l - nf / nv) < 1e-15
    spans = sorted((a, b) for _, a, b, _ in out)
    assert spans[0][0] == 0 and spans[-1][1] == n_total and spans[0][1] == spans[1][0]


def _fake_score(traj):
    # host stand-in for a trajectory's d/dx log p: depends only on the index
    x = ((traj + 17) * 0x85EBCA77) & 0xFFFFFFFF
    return (x / 2.0 ** 32 - 0.5) * 40.0


def _grad_sums(a, b):
    f = np.array([_fake_fail(t) for t in range(a, b)])
    s = np.array([_fake_score(t) for t in range(a, b)])
    ok = f <= 1
    fs = f[ok] * s[ok]
    return int(ok.sum()), int(f[ok].sum()), float(fs.sum()), float((fs * fs).sum())


def _grad_worker(rank, world, port, n_total, q):
    import torch.distributed as dist
    from paper_2511_05719_gb300.sharding import combine_grad_sums
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = trajectory_range(n_total, rank, world)
    q.put((rank, combine_grad_sums(*_grad_sums(a, b))))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_combine_gradient_sums():
    """The sharded score-function gradient equals the single-process one,
    formed as ttn_grad forms it: p_L = n_fail / n, mean of fail * score, its
    standard error sqrt((E[x^2] - E[x]^2) / (n - 1))."""
    import torch.multiprocessing as mp
    n_total, world = 1001, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, world, port, n_total, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    f = np.array([_fake_fail(t) for t in range(n_total)])
    s = np.array([_fake_score(t) for t in range(n_total)])
    ok = f <= 1
    x = f[ok] * s[ok]
    n = ok.sum()
    ref = (f[ok].sum() / n, x.mean(), np.sqrt(max(0.0, (x * x).mean() - x.mean() ** 2) / (n - 1)), n)
    for rank, (p_l, g, sg, nv) in out:
        assert nv == ref[3]
        assert abs(p_l - ref[0]) < 1e-15
        assert abs(g - ref[1]) < 1e-12 * max(1.0, abs(ref[1]))
        assert abs(sg - ref[2]) < 1e-12 * max(1.0, ref[2])


def test_combine_grad_sums_without_a_process_group():
    from paper_2511_05719_gb300.sharding import combine_grad_sums
    p, g, sg, n = combine_grad_sums(*_grad_sums(0, 500))
    assert n > 2 and 0 < p < 1 and sg > 0
    assert np.isnan(combine_grad_sums(1, 0, 0.0, 0.0)[1])

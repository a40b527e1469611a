"""Trajectory sharding across ranks, one process per GPU.

Trajectories are independent Monte Carlo samples (Sec. III.C): each depends
only on (seed, trajectory index), so rank r of W runs its own contiguous block
of indices and no collective touches the data path.  The only exchange is the
final sum of logical-failure counts (one all_reduce of a few integers) to form
p_L and its binomial error, and for the score-function gradient the sums of
fail * score and of its square (two doubles)."""
import math

import numpy as np


def trajectory_range(n_total, rank, world):
    """[start, stop) of rank's trajectories when n_total are split as evenly
    as possible over world ranks (the first n_total % world ranks take one
    more)."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard: n_total=%r rank=%r world=%r" % (n_total, rank, world))
    base, rem = divmod(n_total, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)


def combine_counts(n_fail, n_valid, group=None):
    """Sums (failures, valid shots) over the ranks of `group` (any
    torch.distributed backend; a no-op without an initialised process group)
    and returns (p_L, sigma, n_fail, n_valid) of the whole job."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(n_fail), int(n_valid)], dtype=torch.int64)
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    nf, nv = (int(x) for x in t.cpu().tolist())
    p = nf / nv if nv else float("nan")
    sigma = math.sqrt(p * (1 - p) / nv) if nv else float("nan")
    return p, sigma, nf, nv


def logical_error_rate_sharded(circuit, shots, rank, world, group=None, **run_kw):
    """p_L over `shots` trajectories split across the ranks: this rank runs
    its block through the library (its own GPU) and the counts are summed.
    Shots with a fail byte above 1 (decoder bound exceeded, lost state) are
    excluded, as in ttn_logical_error_rate."""
    from . import _lib
    start, stop = trajectory_range(shots, rank, world)
    nf = nv = 0
    if stop > start:
        out = _lib.run_trajectories(circuit, stop - start, first_traj=start, **run_kw)
        fail = np.asarray(out["fail"])
        nf = int((fail == 1).sum())
        nv = int((fail <= 1).sum())
    return combine_counts(nf, nv, group)


def combine_grad_sums(n_valid, n_fail, sum_fs, sum_fs2, group=None):
    """Sums the score-function sums over the ranks of `group` and returns
    (p_L, dp_L/dx, its standard error, n_valid) of the whole job, formed as
    ttn_grad forms them from one run."""
    import torch
    import torch.distributed as dist
    ti = torch.tensor([int(n_valid), int(n_fail)], dtype=torch.int64)
    tf = torch.tensor([float(sum_fs), float(sum_fs2)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            ti, tf = ti.cuda(), tf.cuda()
        dist.all_reduce(ti, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(tf, op=dist.ReduceOp.SUM, group=group)
    nv, nf = (int(x) for x in ti.cpu().tolist())
    s1, s2 = (float(x) for x in tf.cpu().tolist())
    if nv < 2:
        return float("nan"), float("nan"), float("nan"), nv
    mean = s1 / nv
    var = max(0.0, s2 / nv - mean * mean)
    return nf / nv, mean, math.sqrt(var / (nv - 1)), nv


def grad_sharded(circuit, shots, rank, world, group=None, wrt="theta", **run_kw):
    """dp_L/dx over `shots` trajectories split across the ranks: this rank runs
    its block with the score replay (ttn_grad_sums, its own GPU) and the sums
    are combined.  Returns (p_L, dp_L/dx, standard error, n_valid)."""
    from . import _lib
    start, stop = trajectory_range(shots, rank, world)
    sums = (0, 0, 0.0, 0.0)
    if stop - start >= 2:
        sums = _lib.grad_sums(circuit, stop - start, wrt=wrt, first_traj=start, **run_kw)
    elif stop > start:
        raise ValueError("each rank needs at least 2 shots")
    return combine_grad_sums(*sums, group=group)

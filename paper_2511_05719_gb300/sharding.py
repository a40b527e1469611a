"""Trajectory sharding across ranks, one process per GPU.

Trajectories are independent Monte Carlo samples (Sec. III.C): each depends
only on (seed, trajectory index), so rank r of W runs its own contiguous block
of indices and no collective touches the data path.  The only exchange is the
final sum of logical-failure counts (one all_reduce of a few integers) to form
p_L and its binomial error."""
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
    Shots whose decoding overflowed (fail byte 2) are excluded."""
    from . import _lib
    start, stop = trajectory_range(shots, rank, world)
    nf = nv = 0
    if stop > start:
        out = _lib.run_trajectories(circuit, stop - start, first_traj=start, **run_kw)
        fail = np.asarray(out["fail"])
        nf = int((fail == 1).sum())
        nv = int((fail != 2).sum())
    return combine_counts(nf, nv, group)

"""ttn_grad_sums on the device: its sums reproduce ttn_grad's p_L, dp_L/dx and
standard error on the same trajectories, and the sums of two shards (disjoint
first_traj ranges, as ranks would run them) add up to one run over both.
FP64 at d = 3, one round (one-sided Jacobi path throughout)."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_05719_gb300")


def test_grad_sums_reproduce_grad_and_add_over_shards():
    c = P.Circuit(3, 1)
    kw = dict(noise="srx", theta=0.12, chi=64, precision="fp64", seed=W.BASE_SEED + 41)
    shots = 600
    pl, g, sg = P.grad(c, shots, wrt="theta", **kw)
    nv, nf, s1, s2 = P.grad_sums(c, shots, wrt="theta", **kw)
    assert 2 <= nv <= shots and 0 < nf < nv
    assert nf / nv == pl
    mean = s1 / nv
    assert np.isclose(mean, g, rtol=1e-12, atol=0)
    assert np.isclose(math.sqrt(max(0.0, s2 / nv - mean * mean) / (nv - 1)), sg, rtol=1e-12)
    a = P.grad_sums(c, 250, wrt="theta", first_traj=0, **kw)
    b = P.grad_sums(c, 350, wrt="theta", first_traj=250, **kw)
    assert a[0] + b[0] == nv and a[1] + b[1] == nf
    assert np.isclose(a[2] + b[2], s1, rtol=1e-9, atol=1e-9)
    assert np.isclose(a[3] + b[3], s2, rtol=1e-9)

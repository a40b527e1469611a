"""ttn_crossing on the device: its first evaluation equals
f = ln p_L^a - ln p_L^b and f' = (dp_L^a/dx) / p_L^a - (dp_L^b/dx) / p_L^b
from two ttn_grad runs with the same seed and trajectories, and its next
point stays in the box.  FP64 at chi = 16 (deterministic one-sided Jacobi path), one
syndrome round, d = 3 against d = 5 at theta = 0.2 where both fail often."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_05719_gb300")


def test_crossing_evaluation_equals_two_grad_runs():
    a, b = P.Circuit(3, 1), P.Circuit(5, 1)
    kw = dict(noise="srx", chi=16, precision="fp64", seed=2511057221)
    shots, x0 = 300, 0.2
    # one evaluation: a second one could land where d = 5 shows no failure
    # in 300 shots, which ttn_crossing rightly reports as EINVAL
    r = P.crossing(a, b, shots, x0, 0.05, 0.5, max_iter=1, x_tol=1e-3, **kw)
    assert r["iters"] == 1
    assert 0.05 <= r["x"] <= 0.5
    pa, ga, sa = P.grad(a, shots, wrt="theta", theta=x0, **kw)
    pb, gb, sb = P.grad(b, shots, wrt="theta", theta=x0, **kw)
    assert pa > 0 and pb > 0
    t = r["trace"][0]
    assert t[0] == x0
    assert np.isclose(t[1], math.log(pa) - math.log(pb), rtol=1e-12, atol=1e-14)
    assert np.isclose(t[3], ga / pa - gb / pb, rtol=1e-12, atol=1e-14)
    assert np.isclose(t[2], math.sqrt((1 - pa) / (shots * pa) + (1 - pb) / (shots * pb)), rtol=1e-12)
    assert np.isclose(t[4], math.hypot(sa / pa, sb / pb), rtol=1e-12)

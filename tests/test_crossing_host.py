"""Threshold-crossing search (ttn_newton_crossing, ttn_crossing) on the host:
the Newton core against analytic failure-curve models, and the argument
checks of ttn_crossing that run before any device work.

Model: p_d(x) = A (x / tau)^((d+1)/2), the below-threshold scaling of a
distance-d code, so the curves of d = 5 and d = 7 cross exactly at tau and
f(x) = ln p_5 - ln p_7 = -ln(x / tau), f'(x) = -1 / x."""
import math

import numpy as np
import pytest

P = pytest.importorskip("paper_2511_05719_gb300")

TAU = 0.0371


def _lib_or_skip():
    import os
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")


def model(x, _it):
    return -math.log(x / TAU), 0.0, -1.0 / x, 0.0


@pytest.mark.parametrize("x0", [0.2 * TAU, 0.6 * TAU, 1.7 * TAU, 2.9 * TAU])
def test_noise_free_power_laws_converge_quadratically(x0):
    _lib_or_skip()
    r = P.newton_crossing(model, x0, 0.1 * TAU, 3.0 * TAU, max_iter=30, x_tol=1e-12)
    assert r["converged"]
    assert abs(r["x"] - TAU) < 1e-10 * TAU
    assert r["iters"] <= 9
    err = np.abs(r["trace"][:, 0] - TAU)
    # quadratic convergence once close: e_{k+1} <= C e_k^2 with C = 1 / (2 tau) for this f
    for k in range(len(err) - 1):
        if err[k] < 0.2 * TAU and err[k + 1] > 1e-13:
            assert err[k + 1] <= err[k] ** 2 / TAU + 1e-15
    assert np.allclose(r["trace"][:, 1], [-math.log(x / TAU) for x in r["trace"][:, 0]])


def test_prefactors_move_the_crossing():
    _lib_or_skip()
    a5, a7 = 0.03, 0.07   # p_5 = a5 u^3, p_7 = a7 u^4 cross at u = a5 / a7

    def f(x, _it):
        u = x / TAU
        return math.log(a5 * u ** 3) - math.log(a7 * u ** 4), 0.0, -1.0 / x, 0.0
    r = P.newton_crossing(f, 0.9 * TAU, 0.05 * TAU, 3.0 * TAU, x_tol=1e-12)
    assert r["converged"] and abs(r["x"] - TAU * a5 / a7) < 1e-10 * TAU


def test_noisy_estimates_land_within_their_error():
    _lib_or_skip()
    hits, n = 0, 40
    for seed in range(n):
        rng = np.random.default_rng(1000 + seed)
        sf, sdf = 0.03, 0.05 / TAU

        def f(x, _it):
            return (-math.log(x / TAU) + rng.normal(0, sf), sf, -1.0 / x + rng.normal(0, sdf), sdf)
        r = P.newton_crossing(f, 0.5 * TAU, 0.1 * TAU, 3.0 * TAU, max_iter=25, x_tol=1e-6)
        assert r["converged"]
        assert 0.5 * sf * TAU < r["sigma"] < 2.0 * sf * TAU   # sigma_f / |f'| at the crossing
        hits += abs(r["x"] - TAU) < 3 * r["sigma"]
    assert hits >= 0.85 * n


def test_bracket_safeguard_when_newton_overshoots():
    _lib_or_skip()
    # arctan: Newton diverges from |x - tau| > 1.39; the first step crosses
    # the root, the bracket forms and bisection takes over
    c = 5.0

    def f(x, _it):
        return math.atan(x - c), 0.0, 1.0 / (1.0 + (x - c) ** 2), 0.0
    r = P.newton_crossing(f, c + 3.0, c - 10.0, c + 10.0, max_iter=60, x_tol=1e-10)
    assert r["converged"] and abs(r["x"] - c) < 1e-9
    xs = r["trace"][:, 0]
    assert np.all(xs >= c - 10.0) and np.all(xs <= c + 10.0)


def test_no_slope_and_no_bracket_stops_unconverged():
    _lib_or_skip()
    r = P.newton_crossing(lambda x, it: (1.0, 0.1, 0.0, 0.0), 0.5, 0.0, 1.0, max_iter=10)
    assert not r["converged"] and r["iters"] == 1 and math.isinf(r["sigma"])
    # a slope inside its error counts as unresolved
    r = P.newton_crossing(lambda x, it: (1.0, 0.1, 0.3, 0.2), 0.5, 0.0, 1.0, max_iter=10)
    assert not r["converged"] and r["iters"] == 1


def test_evaluator_errors_and_argument_checks():
    _lib_or_skip()

    def bad(x, it):
        raise ValueError("evaluator failed")
    with pytest.raises(ValueError):
        P.newton_crossing(bad, 0.5, 0.0, 1.0)
    with pytest.raises(P.TTNError) as e:
        P.newton_crossing(lambda x, it: (float("nan"), 0.0, 1.0, 0.0), 0.5, 0.0, 1.0)
    assert e.value.status == 1
    for args in [(0.5, 1.0, 0.0), (1.5, 0.0, 1.0), (-0.1, 0.0, 1.0)]:
        with pytest.raises(P.TTNError) as e:
            P.newton_crossing(model, *args)
        assert e.value.status == 1
    for kw in [dict(max_iter=0), dict(max_iter=1001), dict(x_tol=0.0)]:
        with pytest.raises(P.TTNError):
            P.newton_crossing(model, 0.5 * TAU, 0.1 * TAU, TAU, **kw)


def test_crossing_argument_checks_before_device_work():
    _lib_or_skip()
    a, b = P.Circuit(3, 1), P.Circuit(5, 1)
    base = dict(noise="srx", chi=16, precision="fp64")
    cases = [dict(shots=1), dict(wrt=2), dict(wrt="gamma", noise="ad", x_lo=0.0),
             dict(wrt="gamma", noise="ad", x_hi=1.0), dict(chi=0), dict(x0=0.9),
             dict(max_iter=0)]
    for c in cases:
        kw = dict(base, shots=100, x0=0.1, x_lo=0.01, x_hi=0.5)
        kw.update(c)
        if kw.get("wrt") == 2:
            kw["wrt"] = 2
        with pytest.raises(P.TTNError) as e:
            P.crossing(a, b, **kw)
        assert e.value.status == 1, c


def test_iteration_limit_and_exact_zero():
    _lib_or_skip()
    # slow convergence with a tight tolerance: stops at max_iter, not converged
    r = P.newton_crossing(lambda x, it: (x ** 3, 0.0, 3 * x ** 2, 0.0), 0.9, -1.0, 1.0,
                          max_iter=4, x_tol=1e-15)
    assert r["iters"] == 4 and not r["converged"]
    assert r["trace"].shape == (4, 5) and np.all(np.diff(r["trace"][:, 0]) < 0)
    # f exactly zero with a nonzero error: at the crossing within noise
    r = P.newton_crossing(lambda x, it: (0.0, 0.1, 1.0, 0.01), 0.3, 0.0, 1.0)
    assert r["converged"] and r["x"] == 0.3 and r["iters"] == 1
    assert r["sigma"] == pytest.approx(0.1)
    # f exactly zero with zero error carries no information: no slope step stops it unconverged
    r = P.newton_crossing(lambda x, it: (0.0, 0.0, 0.0, 0.0), 0.3, 0.0, 1.0)
    assert not r["converged"] and r["iters"] == 1

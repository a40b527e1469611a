"""Eq. 4 threshold fit (ttn_threshold_fit) on the host, against scipy's
curve_fit as an independent least-squares solver and against the truth of
seeded synthetic sweeps.  Data shaped like the paper's sweeps: d = 3, 5, 7,
eight strengths around the threshold, binomial-sized errors."""
import numpy as np
import pytest

P = pytest.importorskip("paper_2511_05719_gb300")
optimize = pytest.importorskip("scipy.optimize")

TRUE = dict(A=0.12, B=1.6, C=4.0, tau=0.021, nu=1.4)


def _lib_or_skip():
    import os
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")


def eq4(X, A, B, C, tau, nu):
    p, d = X
    x = (p - tau) * d ** (1.0 / nu)
    return A + B * x + C * x * x


def sweep(noise, seed):
    rng = np.random.default_rng(seed)
    d = np.repeat([3, 5, 7], 8)
    p = np.tile(np.linspace(0.015, 0.027, 8), 3)
    y0 = eq4((p, d), *TRUE.values())
    sigma = np.sqrt(y0 * (1 - y0) / 1e4)     # 1e4 shots per point
    y = y0 + noise * sigma * rng.standard_normal(y0.size)
    return d, p, y, sigma


def test_noise_free_recovers_the_parameters():
    _lib_or_skip()
    d, p, y, s = sweep(0.0, 1)
    r = P.threshold_fit(d, p, y, s, tau0=0.018, nu0=1.0)
    for k, v in TRUE.items():
        assert abs(r[k] - v) < 1e-7 * max(1.0, abs(v)), (k, r[k], v)
    assert r["chi2"] < 1e-12


@pytest.mark.parametrize("seed", [2, 3, 4, 5])
def test_matches_scipy_least_squares(seed):
    _lib_or_skip()
    d, p, y, s = sweep(1.0, seed)
    r = P.threshold_fit(d, p, y, s, tau0=0.018, nu0=1.0)
    popt, pcov = optimize.curve_fit(eq4, (p, d.astype(float)), y, p0=list(TRUE.values()), sigma=s,
                                    absolute_sigma=True, maxfev=20000)
    ours = np.array([r[k] for k in ("A", "B", "C", "tau", "nu")])
    # both stop in the same chi^2 minimum; weakly determined parameters (C)
    # may differ along its flat valley, so compare in standard errors
    se = np.sqrt(np.diag(pcov))
    assert np.all(np.abs(ours - popt) < 1e-4 * se), (ours, popt, se)
    assert np.allclose(r["cov"], pcov, rtol=1e-3, atol=1e-14)
    res = (eq4((p, d), *popt) - y) / s
    assert r["chi2"] <= res @ res * (1 + 1e-9)
    # the truth lies within a few standard errors
    assert abs(r["tau"] - TRUE["tau"]) < 4 * np.sqrt(r["cov"][3, 3])


def test_argument_checks():
    _lib_or_skip()
    d, p, y, s = sweep(0.0, 1)
    bad = [dict(d=d[:5], p=p[:5], y=y[:5], s=s[:5]),            # fewer than 6 points
           dict(d=np.full_like(d, 5)),                           # one distance
           dict(s=np.where(np.arange(s.size) == 3, 0.0, s)),     # sigma <= 0
           dict(y=np.where(np.arange(y.size) == 2, np.nan, y))]  # non-finite
    for b in bad:
        kw = dict(d=d, p=p, y=y, s=s)
        kw.update(b)
        with pytest.raises(P.TTNError) as e:
            P.threshold_fit(kw["d"], kw["p"], kw["y"], kw["s"], tau0=0.02)
        assert e.value.status == 1
    with pytest.raises(P.TTNError):
        P.threshold_fit(d, p, y, s, tau0=0.02, nu0=0.0)
    with pytest.raises(ValueError):
        P.threshold_fit(d, p[:-1], y, s, tau0=0.02)

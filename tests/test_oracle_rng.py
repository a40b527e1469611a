"""Pins of the Philox draws used for every stochastic event: the block
function against the published known-answer vectors, then the statistics of
the derived uniforms."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle import philox

KAT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(KAT):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            rows.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return rows


def test_block_matches_published_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert philox.philox4x32_10(ctr, key) == out
        v = philox.philox4x32_10_np(*[np.array([x], dtype=np.uint64) for x in ctr + key])
        assert tuple(int(x[0]) for x in v) == out


def test_scalar_matches_vector():
    for (s, t, e) in [(0, 0, 0), (2511057190, 5, 17), (2 ** 63 + 11, 2 ** 40 + 3, 999)]:
        assert philox.uniform(s, t, e) == philox.uniforms(s, [t], [e])[0, 0]


def test_uniform_moments_and_ks():
    u = philox.uniforms(2511057190, np.arange(200), np.arange(500)).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    n = u.size
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 4 * np.sqrt(1 / 180 / n)
    assert stats.kstest(u, "uniform").pvalue > 1e-4


def test_independence_of_neighbours():
    u = philox.uniforms(7, np.arange(300), np.arange(300))
    a = u[:, :-1].ravel() - 0.5
    b = u[:, 1:].ravel() - 0.5
    r = np.mean(a * b) / np.sqrt(np.mean(a * a) * np.mean(b * b))
    assert abs(r) < 4 / np.sqrt(a.size)
    a = u[:-1, :].ravel() - 0.5
    b = u[1:, :].ravel() - 0.5
    r = np.mean(a * b) / np.sqrt(np.mean(a * a) * np.mean(b * b))
    assert abs(r) < 4 / np.sqrt(a.size)


def test_seed_changes_stream():
    a = philox.uniforms(1, np.arange(10), np.arange(10))
    b = philox.uniforms(2, np.arange(10), np.arange(10))
    assert not np.any(a == b)

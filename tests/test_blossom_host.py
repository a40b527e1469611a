"""The decoder kernel's blossom matcher (csrc/blossom.cuh), compiled for the
host, against the oracle's exact matchings (subset DP; networkx blossom for
larger instances) on seeded random instances with unique optima."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import decoder as DEC

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("bl") / "blossom_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "blossom_host_check.cpp")],
                   check=True)
    return exe


def _instance(rng, k, p_absent, p_noboundary, unique=True):
    base = rng.integers(1, 12, size=(k, k))
    base = np.triu(base, 1)
    base = base + base.T
    W = base.astype(np.int64) << 20
    if unique:
        W = W + np.triu(rng.integers(0, 1 << 20, size=(k, k)), 1)
    W = np.triu(W, 1)
    W = W + W.T
    absent = np.triu(rng.random((k, k)) < p_absent, 1)
    absent = absent | absent.T
    W[absent] = -1
    np.fill_diagonal(W, -1)
    wb = (rng.integers(1, 15, size=k).astype(np.int64) << 20) + (rng.integers(0, 1 << 20, size=k) if unique else 0)
    wb[rng.random(k) < p_noboundary] = -1
    return W, wb


def _run(exe, instances):
    lines = []
    for W, wb in instances:
        k = len(wb)
        lines.append(str(k))
        lines.append(" ".join(map(str, W.ravel().tolist())))
        lines.append(" ".join(map(str, wb.tolist())))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    res = []
    for ln in out.stdout.strip().splitlines():
        v = list(map(int, ln.split()))
        res.append((v[0], v[1:]))
    return res


def _oracle(W, wb):
    k = len(wb)
    wp = lambda i, j: None if W[i, j] < 0 else int(W[i, j])
    wbf = lambda i: None if wb[i] < 0 else int(wb[i])
    if k <= 12:
        pairs, tot = DEC.mwpm_dp(list(range(k)), wp, wbf)
    else:
        pairs, tot = DEC.mwpm_blossom(k, wp, wbf)
    partner = [-3] * k
    for i, j in pairs:
        partner[i] = j
        if j >= 0:
            partner[j] = i
    return tot, partner


@pytest.mark.parametrize("k,p_absent,p_nb,count", [
    (1, 0.0, 0.0, 5), (2, 0.0, 0.0, 20), (5, 0.2, 0.2, 60), (9, 0.3, 0.1, 60),
    (12, 0.1, 0.5, 40), (24, 0.5, 0.1, 25), (40, 0.7, 0.05, 12), (64, 0.8, 0.0, 6),
])
def test_blossom_matches_oracle(checker, k, p_absent, p_nb, count):
    rng = np.random.default_rng(1000 + k)
    inst = [_instance(rng, k, p_absent, p_nb) for _ in range(count)]
    got = _run(checker, inst)
    for (W, wb), (tot, partner) in zip(inst, got):
        try:
            want_tot, want_partner = _oracle(W, wb)
        except ValueError:
            assert tot == -2
            continue
        assert tot == want_tot
        assert partner == want_partner  # optimum is unique (perturbed weights)


def test_blossom_degenerate_weights_optimal(checker):
    """Many tied optima (no perturbation): only the total is unique."""
    rng = np.random.default_rng(7)
    inst = [_instance(rng, k, 0.3, 0.1, unique=False) for k in (6, 10, 14, 20) for _ in range(10)]
    got = _run(checker, inst)
    for (W, wb), (tot, partner) in zip(inst, got):
        try:
            want_tot, _ = _oracle(W, wb)
        except ValueError:
            assert tot == -2
            continue
        assert tot == want_tot
        k = len(wb)
        s = 0
        for i, j in enumerate(partner):  # a valid matching with that total
            if j == -1:
                assert wb[i] >= 0
                s += wb[i]
            else:
                assert partner[j] == i and W[i, j] >= 0
                if j > i:
                    s += W[i, j]
        assert s == tot

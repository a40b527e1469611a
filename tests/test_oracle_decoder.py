"""Pins of the concatenated-MWPM decoder oracle (App. A.2)."""
import itertools
import math

import numpy as np
import pytest

from oracle import decoder as dec
from oracle.circuit import build_circuit
from oracle.statevector import run_trajectory
from oracle.channels import NONE


def brute_matching(k, wpair, wbound):
    """Enumerate every assignment of k defects to pairs / boundary."""
    best = None

    def rec(left, acc):
        nonlocal best
        if not left:
            if best is None or acc < best:
                best = acc
            return
        i = left[0]
        rest = left[1:]
        wb = wbound(i)
        if wb is not None:
            rec(rest, acc + wb)
        for j in rest:
            w = wpair(i, j)
            if w is not None:
                rec([x for x in rest if x != j], acc + w)
    rec(list(range(k)), 0)
    return best


def test_dp_matching_equals_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(60):
        k = int(rng.integers(1, 9))
        W = rng.integers(1, 30, size=(k, k))
        W = W + W.T
        Wb = rng.integers(1, 40, size=k)

        def wp(i, j):
            return int(W[i, j]) * dec.WUNIT + dec.pair_hash(i, j, 0, 0)

        def wb(i):
            return int(Wb[i]) * dec.WUNIT + dec.pair_hash(i, 99, 0, 0)
        pairs, tot = dec.mwpm_dp(list(range(k)), wp, wb)
        assert tot == brute_matching(k, wp, wb)
        covered = sorted([i for p in pairs for i in p if i >= 0])
        assert covered == list(range(k))


def test_component_split_and_blossom_equal_dp():
    rng = np.random.default_rng(8)
    for trial in range(40):
        k = int(rng.integers(1, 12))
        pts = rng.uniform(0, 20, size=(k, 2))
        W = np.round(np.abs(pts[:, None, :] - pts[None, :, :]).sum(-1)).astype(int) + 1
        Wb = np.round(np.minimum(pts[:, 0], 20 - pts[:, 0])).astype(int) + 1

        def wp(i, j):
            return int(W[i, j]) * dec.WUNIT + dec.pair_hash(i, j, 0, 1)

        def wb(i):
            return int(Wb[i]) * dec.WUNIT + dec.pair_hash(i, 500, 0, 1)
        p0, t0 = dec.mwpm_dp(list(range(k)), wp, wb)
        p1, t1 = dec.mwpm(list(range(k)), wp, wb)
        p2, t2 = dec.mwpm_blossom(k, wp, wb)
        assert t0 == t1 == t2
        assert sorted(p0) == sorted(p1) == sorted(p2)


def test_noise_free_records_do_not_fail():
    circ = build_circuit(3, 3)
    G = dec.DecoderGraphs(3, 3)
    for t in range(6):
        rec = run_trajectory(circ, NONE, 0.0, 0.0, 11, t)["rec"]
        f, c, s = dec.decode(G, rec)
        assert f == 0 and s == 0


# The reading of the decoder in this project fails on exactly these weight-3
# code-capacity patterns at d = 7 (degenerate stage-1 shortest paths); every
# other pattern of weight <= (d-1)/2 at d = 3, 5, 7 is corrected.
D7_KNOWN = {(11, 21, 29), (11, 22, 26), (25, 31, 35), (25, 32, 34)}


@pytest.mark.parametrize("d", [3, 5, 7])
def test_code_capacity_correctable(d):
    G = dec.DecoderGraphs(d, 1)
    code = G.code
    P, n = code.n_plaq, code.n
    bad = set()
    for w in range(1, (d - 1) // 2 + 1):
        for E in itertools.combinations(range(n), w):
            rec = np.zeros(2 * P + n, dtype=np.uint8)
            rec[[2 * P + q for q in E]] = 1
            if dec.decode(G, rec)[0]:
                bad.add(E)
    assert bad == (D7_KNOWN if d == 7 else set())


def test_single_measurement_error_is_time_like():
    # one flipped Z-ancilla outcome in the middle round: a time-like pair of
    # detectors, matched with weight 2 (one measurement error... two time edges
    # or one), never a logical flip
    d, C = 5, 3
    G = dec.DecoderGraphs(d, C)
    P, n = G.code.n_plaq, G.code.n
    for p in range(P):
        rec = np.zeros(C * 2 * P + n, dtype=np.uint8)
        rec[1 * 2 * P + 2 * p] = 1
        f, c, s = dec.decode(G, rec)
        assert f == 0 and s == 1

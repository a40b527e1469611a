"""Pins of the color-code geometry and circuit oracle against closed forms."""
import itertools

import numpy as np
import pytest

from oracle.colorcode import color_code, check_matrix, n_qubits_total
from oracle.circuit import build_circuit, CNOT, MEAS_Z, MEAS_X, NOISE, PREP_Z, PREP_X


def gf2_rank(M):
    M = np.array(M, dtype=np.uint8) % 2
    r = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = [i for i in range(r, rows) if M[i, c]]
        if not piv:
            continue
        M[[r, piv[0]]] = M[[piv[0], r]]
        for i in range(rows):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
    return r


@pytest.mark.parametrize("d,N,wsum", [(3, 13, 12), (5, 37, 42), (7, 73, 90)])
def test_counts(d, N, wsum):
    code = color_code(d)
    # [[ (3d^2+1)/4, 1, d ]] and N = n + 2 * #plaquettes (Sec. II.A)
    assert code.n == (3 * d * d + 1) // 4
    assert code.n_plaq == (code.n - 1) // 2
    assert n_qubits_total(code) == N
    weights = [len(s) for s in code.plaq_support]
    assert set(weights) <= {4, 6}
    assert sum(weights) == wsum
    # three colours, adjacent faces differ (faces sharing a qubit)
    for q in range(code.n):
        cols = [code.plaq_color[p] for p in code.qubit_plaqs[q]]
        assert len(cols) == len(set(cols))


@pytest.mark.parametrize("d", [3, 5, 7])
def test_stabilizers_commute_and_k1(d):
    code = color_code(d)
    H = np.array(check_matrix(code))
    # X and Z checks on faces p, p' overlap on an even number of qubits
    ov = (H @ H.T) % 2
    assert not ov.any()
    # k = n - rank(H_X) - rank(H_Z) = 1
    assert code.n - 2 * gf2_rank(H) == 1
    # Z-bar = Z^{x n} commutes with every X check (even weights)
    assert all(len(s) % 2 == 0 for s in code.plaq_support)
    assert code.n % 2 == 1   # and anticommutes with X-bar = X^{x n}


def _min_logical_weight(code, wmax):
    H = np.array(check_matrix(code))
    rk = gf2_rank(H)
    for w in range(1, wmax + 1):
        for E in itertools.combinations(range(code.n), w):
            x = np.zeros(code.n, dtype=np.uint8)
            x[list(E)] = 1
            if ((H @ x) % 2).any():
                continue
            if gf2_rank(np.vstack([H, x])) > rk:   # not a stabilizer
                return w
    return None


@pytest.mark.parametrize("d", [3, 5])
def test_distance(d):
    assert _min_logical_weight(color_code(d), d) == d


@pytest.mark.parametrize("d,C", [(3, 1), (3, 3), (5, 2)])
def test_circuit_counts(d, C):
    circ = build_circuit(d, C)
    code = circ.code
    N, n, P = circ.n_qubits, code.n, code.n_plaq
    kinds = [op[0] for op in circ.ops]
    wsum = sum(len(s) for s in code.plaq_support)
    # each round measures every face's X and Z check with one CNOT per support qubit
    assert kinds.count(CNOT) == 2 * wsum * C
    assert kinds.count(MEAS_Z) == P * C + n
    assert kinds.count(MEAS_X) == P * C
    assert kinds.count(PREP_Z) == P * C + n
    assert kinds.count(PREP_X) == P * C
    # an error location on every qubit after each of the 13 gate/prep layers,
    # on the idle data during the measurement layer
    assert kinds.count(NOISE) == C * (13 * N + n)
    assert circ.n_layers == 14 * C + 1
    # each layer touches each qubit at most once with a gate
    for L in range(circ.n_layers):
        used = []
        for op in circ.ops:
            if op[5] == L and op[0] in (CNOT, MEAS_Z, MEAS_X, PREP_Z, PREP_X):
                used += [op[1]] + ([op[2]] if op[0] == CNOT else [])
        assert len(used) == len(set(used))
    # event ids are 0..n_events-1 in program order
    ev = [op[3] for op in circ.ops if op[3] >= 0]
    assert ev == list(range(circ.n_events))
    recs = sorted(op[4] for op in circ.ops if op[4] >= 0)
    assert recs == list(range(circ.n_record_bits))

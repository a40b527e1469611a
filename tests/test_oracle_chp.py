"""Pins of the stabilizer-tableau trajectory oracle (O3) for Pauli noise:
closed-form Bell / GHZ cases, identical records and log-probabilities to the
state-vector oracle (O1) on the same draws at d = 3 (the two share only the
circuit and the random numbers), and the noise-off syndrome invariants at
d = 3, 5, 7 (Z checks zero, X checks repeating, even data parity)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import chp, statevector as SV
from oracle.channels import NONE, SRX_PTA, AD_PTA, DEPOL
from oracle.circuit import build_circuit


def test_bell_and_ghz_closed_forms():
    t = chp.Tableau(2)
    t.h(0)
    t.cnot(0, 1)                           # (|00> + |11>)/sqrt2
    out, p, mg = t.measure_z(0, 0.7)       # random: u >= 0.5 -> 1
    assert (out, p) == (1, 0.5) and mg == pytest.approx(0.2)
    out, p, mg = t.measure_z(1, 0.1)       # now determined
    assert (out, p, mg) == (1, 1.0, None)
    g = chp.Tableau(3)
    g.h(0)
    g.cnot(0, 1)
    g.cnot(1, 2)                           # GHZ: X X X = +1
    for q in range(3):
        g.h(q)
    outs = [g.measure_z(q, u)[0] for q, u in zip(range(3), (0.9, 0.2, 0.6))]
    assert sum(outs) % 2 == 0
    z = chp.Tableau(1)
    z.pauli(0, 1)                          # X|0> = |1>
    assert z.measure_z(0, 0.3)[0] == 1
    y = chp.Tableau(1)
    y.h(0)
    y.pauli(0, 3)                          # Z|+> = |->, H -> |1>
    y.h(0)
    assert y.measure_z(0, 0.3)[0] == 1


@pytest.mark.parametrize("model,th,ga", [(SRX_PTA, 0.12, 0.0), (AD_PTA, 0.0, 0.08), (DEPOL, 0.0, 0.03)])
@pytest.mark.parametrize("C", [2, 3])
def test_equals_statevector_oracle_d3(model, th, ga, C):
    circ = build_circuit(3, C)
    compared = 0
    for t in range(24):
        a = SV.run_trajectory(circ, model, th, ga, W.BASE_SEED + 5, t)
        b = chp.run_trajectory(circ, model, th, ga, W.BASE_SEED + 5, t)
        if min(a["margin"], b["margin"]) < 1e-9:
            continue
        compared += 1
        assert np.array_equal(a["rec"], b["rec"]), t
        assert abs(a["logp"] - b["logp"]) < 1e-9
        assert len(a["branch_p"]) <= len(b["branch_p"])
    assert compared >= 20


@pytest.mark.parametrize("d", [3, 5, 7])
def test_noise_off_invariants(d):
    circ = build_circuit(d, 2)
    P = circ.code.n_plaq
    n = circ.code.n
    for t in range(3):
        r = chp.run_trajectory(circ, NONE, 0.0, 0.0, W.BASE_SEED, t)["rec"]
        zs = [r[rd * 2 * P + 2 * p] for rd in range(2) for p in range(P)]
        assert not any(zs)
        x1 = [r[0 * 2 * P + 2 * p + 1] for p in range(P)]
        x2 = [r[1 * 2 * P + 2 * p + 1] for p in range(P)]
        assert x1 == x2
        assert int(np.sum(r[2 * 2 * P: 2 * 2 * P + n])) % 2 == 0

"""Pins of the state-vector trajectory oracle O1 (Sec. III.C)."""
import math

import numpy as np
import pytest

from oracle import statevector as SV, densitymatrix as DM, philox
from oracle.channels import NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD, X
from oracle.circuit import build_circuit, NOISE, MEAS_Z
from oracle.decoder import DecoderGraphs, decode
from tests.oracle_helpers import custom_circuit, small_qec_circuit


@pytest.mark.parametrize("k,theta", [(1, 0.05), (7, 0.05), (13, 0.11), (40, 0.03)])
def test_srx_idle_closed_form(k, theta):
    # an idle qubit under k SRX locations: exp(-i k theta X)|0>, P(1) = sin^2(k theta)
    circ = custom_circuit(1, [[(NOISE, 0, None)] for _ in range(k)])
    out = SV.run_trajectory(circ, SRX, theta, 0.0, 1, 0)
    assert out["sv"].prob1(0) == pytest.approx(math.sin(k * theta) ** 2, abs=1e-14)


@pytest.mark.parametrize("k,theta", [(5, 0.2), (20, 0.1)])
def test_srx_pta_idle_closed_form(k, theta):
    # twirled: X flips with prob sin^2 theta each; P(odd flips) = (1-(1-2s)^k)/2
    circ = custom_circuit(1, [[(NOISE, 0, None)] for _ in range(k)] + [[(MEAS_Z, 0, None)]])
    recs, _, _ = SV.run_trajectories(circ, SRX_PTA, theta, 0.0, 5, range(3000))
    s = math.sin(theta) ** 2
    p = (1 - (1 - 2 * s) ** k) / 2
    assert abs(recs[:, 0].mean() - p) < 4 * math.sqrt(p * (1 - p) / 3000)


def test_ad_one_location_from_one():
    gamma = 0.3
    n = 4000
    jumps = 0
    for t in range(n):
        sv = SV.StateVector(1)
        sv.apply1(0, X)
        u = philox.uniform(9, t, 0)
        SV.apply_noise(sv, 0, AD, 0.0, gamma, u)
        p1 = sv.prob1(0)
        assert p1 in (0.0, 1.0) or abs(p1 - 1) < 1e-15
        jumps += p1 < 0.5
    # P(1) after the channel = 1 - gamma
    assert abs(jumps / n - gamma) < 4 * math.sqrt(gamma * (1 - gamma) / n)


@pytest.mark.parametrize("model", [NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD])
def test_norm_and_noise_off_invariants(model):
    circ = build_circuit(3, 2)
    code = circ.code
    P = code.n_plaq
    th, ga = (0.0, 0.0) if model == NONE else (0.07, 0.03)
    for t in range(4):
        out = SV.run_trajectory(circ, model, th, ga, 3, t)
        assert out["sv"].norm2() == pytest.approx(1.0, abs=1e-12)
        if model == NONE:
            rec = out["rec"]
            z = [rec[r * 2 * P + 2 * p] for r in range(2) for p in range(P)]
            x0 = [rec[2 * p + 1] for p in range(P)]
            x1 = [rec[2 * P + 2 * p + 1] for p in range(P)]
            assert not any(z)                 # |0>^n: every Z check +1
            assert x0 == x1                   # X checks repeat after round 1
            data = rec[2 * 2 * P:]
            assert int(np.sum(data)) % 2 == 0  # Z-bar = +1
            for sup in code.plaq_support:
                assert int(np.sum(data[sup])) % 2 == 0


@pytest.mark.parametrize("model,theta,gamma", [(SRX, 0.2, 0.0), (AD, 0.0, 0.25),
                                               (SRX_PTA, 0.2, 0.0), (AD_PTA, 0.0, 0.25),
                                               (SRX_AD, 0.15, 0.2)])
def test_trajectory_average_matches_density_matrix(model, theta, gamma):
    circ = small_qec_circuit()
    _, p1 = DM.evolve(circ, model, theta, gamma)
    n = 1500
    recs, _, _ = SV.run_trajectories(circ, model, theta, gamma, 21, range(n))
    mean = recs.mean(axis=0)
    sig = np.sqrt(np.maximum(p1 * (1 - p1), 1e-4) / n)
    assert np.all(np.abs(mean - p1) < 4 * sig + 1e-12), (mean, p1)


def test_unitary_density_matrix_equals_state():
    circ = small_qec_circuit()
    # no measurement: drop the measurement layers (keep gates and SRX noise)
    ops = [op for op in circ.ops if op[0] not in (3, 4)]
    from types import SimpleNamespace
    c2 = SimpleNamespace(n_qubits=circ.n_qubits, ops=[op for op in ops if op[0] != 0 and op[0] != 1],
                         n_record_bits=0)
    dm, _ = DM.evolve(c2, SRX, 0.3, 0.0)
    out = SV.run_trajectory(c2, SRX, 0.3, 0.0, 1, 0)
    psi = out["sv"].amplitudes()
    assert np.allclose(dm.matrix(), np.outer(psi, psi.conj()), atol=1e-13)


def exact_pl_srx(d, C, theta):
    circ = build_circuit(d, C)
    code = circ.code
    P = code.n_plaq
    keep = [r * 2 * P + 2 * p for r in range(C) for p in range(P)] + \
           [C * 2 * P + q for q in range(code.n)]
    dist = DM.record_distribution(circ, theta, keep)
    G = DecoderGraphs(d, C)
    pl = 0.0
    for bits, pr in dist.items():
        rec = np.zeros(circ.n_record_bits, dtype=np.uint8)
        rec[keep] = bits
        pl += pr * decode(G, rec)[0]
    return pl, sum(dist.values())


def test_exact_pl_vs_trajectories_d3_c1_srx():
    theta = 0.12
    pl, tot = exact_pl_srx(3, 1, theta)
    assert tot == pytest.approx(1.0, abs=1e-12)
    circ = build_circuit(3, 1)
    G = DecoderGraphs(3, 1)
    n = 1500
    recs, _, _ = SV.run_trajectories(circ, SRX, theta, 0.0, 2511057190, range(n))
    fails = np.array([decode(G, r)[0] for r in recs])
    est = fails.mean()
    assert pl > 0.01
    assert abs(est - pl) < 3 * math.sqrt(pl * (1 - pl) / n) + 1e-9


@pytest.mark.parametrize("k,theta", [(1, 0.3), (5, 0.07), (12, 0.02)])
def test_record_log_prob_closed_form(k, theta):
    """k SRX locations then a Z measurement: log p(1) = log sin^2(k theta), its
    theta-derivative 2 k cot(k theta); log p(0) = log cos^2(k theta), derivative
    -2 k tan(k theta)."""
    circ = custom_circuit(1, [[(NOISE, 0, None)] for _ in range(k)] + [[(MEAS_Z, 0, None)]])
    one, zero = np.array([1], np.uint8), np.array([0], np.uint8)
    assert SV.record_log_prob(circ, SRX, theta, 0.0, one) == pytest.approx(
        math.log(math.sin(k * theta) ** 2), abs=1e-12)
    assert SV.record_log_prob(circ, SRX, theta, 0.0, zero) == pytest.approx(
        math.log(math.cos(k * theta) ** 2), abs=1e-12)
    h = 1e-5
    fd1 = (SV.record_log_prob(circ, SRX, theta + h, 0.0, one)
           - SV.record_log_prob(circ, SRX, theta - h, 0.0, one)) / (2 * h)
    fd0 = (SV.record_log_prob(circ, SRX, theta + h, 0.0, zero)
           - SV.record_log_prob(circ, SRX, theta - h, 0.0, zero)) / (2 * h)
    assert fd1 == pytest.approx(2 * k / math.tan(k * theta), rel=1e-6)
    assert fd0 == pytest.approx(-2 * k * math.tan(k * theta), rel=1e-6)
    # noise off: the measurement of |0> cannot give 1
    assert SV.record_log_prob(circ, NONE, 0.0, 0.0, one) == -math.inf


def test_record_log_prob_equals_sampled_log_prob():
    """Forcing a d = 3 trajectory's own record reproduces its log-probability."""
    circ = build_circuit(3, 1)
    for traj in range(4):
        out = SV.run_trajectory(circ, SRX, 0.12, 0.0, 17, traj)
        lp = SV.record_log_prob(circ, SRX, 0.12, 0.0, out["rec"])
        assert lp == pytest.approx(out["logp"], abs=1e-10)
    with pytest.raises(ValueError):
        SV.record_log_prob(circ, AD, 0.0, 0.05, out["rec"])

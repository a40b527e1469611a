"""Pins of the plain TTN oracle O4 against the state-vector oracle O1."""
import numpy as np
import pytest

from oracle import statevector as SV, ttn as TT
from oracle.channels import NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD
from oracle.circuit import build_circuit


@pytest.mark.parametrize("model,theta,gamma", [(NONE, 0, 0), (SRX, 0.05, 0), (AD, 0, 0.05),
                                               (SRX_PTA, 0.1, 0), (AD_PTA, 0, 0.05),
                                               (SRX_AD, 0.05, 0.02)])
def test_untruncated_ttn_equals_statevector(model, theta, gamma):
    circ = build_circuit(3, 2)
    layers = [3, 9, 16, circ.n_layers - 1]
    rng = np.random.default_rng(2)
    for traj in range(2):
        layout = rng.permutation(16)[:circ.n_qubits] if traj else list(range(circ.n_qubits))
        a = SV.run_trajectory(circ, model, theta, gamma, 31, traj, snapshot_layers=layers)
        b = TT.run_trajectory(circ, model, theta, gamma, 31, traj, chi=256,
                              leaf_of_qubit=layout, snapshot_layers=layers)
        assert b["discarded"] == 0.0
        assert np.array_equal(a["rec"], b["rec"])
        assert abs(a["logp"] - b["logp"]) < 1e-10
        for L in layers:
            assert np.max(np.abs(a["states"][L] - b["states"][L])) < 1e-12


def test_chi_one_is_product_state():
    circ = build_circuit(3, 1)
    out = TT.run_trajectory(circ, SRX, 0.05, 0.0, 3, 0, chi=1, max_ops=200)
    assert out["ttn"].max_bond() <= 2
    psi = out["ttn"].amplitudes()
    assert np.linalg.norm(psi) == pytest.approx(1.0, abs=1e-12)


def test_run_stops_at_op_budget_and_deadline():
    """The bounded-sample controls used by the CPU timing baseline: an op
    budget stops after exactly that many ops, a past deadline before the
    first op, and a full run reports every op."""
    import time as _time
    from oracle.circuit import build_circuit
    from oracle import ttn as TT
    from oracle.channels import SRX
    circ = build_circuit(3, 1)
    full = TT.run_trajectory(circ, SRX, 0.05, 0.0, 1, 0, chi=64)
    assert full["ops_done"] == len(circ.ops)
    part = TT.run_trajectory(circ, SRX, 0.05, 0.0, 1, 0, chi=64, max_ops=17)
    assert part["ops_done"] == 17
    none = TT.run_trajectory(circ, SRX, 0.05, 0.0, 1, 0, chi=64, deadline=_time.time() - 1.0)
    assert none["ops_done"] == 0

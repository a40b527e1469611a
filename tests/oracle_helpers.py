"""Small hand-built circuits for oracle pins (same op encoding as oracle.circuit)."""
from types import SimpleNamespace

from oracle.circuit import PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X, NOISE


def custom_circuit(n_qubits, ops_no_ids):
    """ops_no_ids: list of (kind, a, b) per layer (list of lists).  Events,
    record bits and location ids are assigned in program order; a NOISE op
    is written (NOISE, q, None)."""
    ops = []
    ev = loc = rec = 0
    for L, layer in enumerate(ops_no_ids):
        for (k, a, b) in layer:
            if k in (MEAS_Z, MEAS_X):
                ops.append((k, a, -1, ev, rec, L))
                ev += 1
                rec += 1
            elif k == NOISE:
                ops.append((k, a, loc, ev, -1, L))
                ev += 1
                loc += 1
            else:
                ops.append((k, a, -1 if b is None else b, -1, -1, L))
    return SimpleNamespace(n_qubits=n_qubits, ops=ops, n_record_bits=rec,
                           n_events=ev, n_layers=len(ops_no_ids), n_locations=loc)


def small_qec_circuit():
    """4 data + 1 Z-ancilla + 1 X-ancilla, two rounds of a weight-4 check pair,
    noise after every layer on every non-measured qubit."""
    N = 6
    layers = []
    allq = list(range(N))

    def noise(qs):
        return [(NOISE, q, None) for q in qs]
    for r in range(2):
        layers.append([(PREP_Z, 4, None), (PREP_X, 5, None)] + noise(allq))
        for q in range(4):
            layers.append([(CNOT, q, 4)] + noise(allq))
        for q in range(4):
            layers.append([(CNOT, 5, q)] + noise(allq))
        layers.append([(MEAS_Z, 4, None), (MEAS_X, 5, None)] + noise(range(4)))
    layers.append([(MEAS_Z, q, None) for q in range(4)])
    return custom_circuit(N, layers)

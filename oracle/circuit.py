"""Syndrome-extraction circuit of the color code with circuit-level noise.

Oracle (test infrastructure only).  Follows Sec. III ("Methods") and Fig. 1:
C cycles of non-fault-tolerant syndrome extraction; per plaquette one ancilla
prepared in |0> (Z check, CNOTs data -> ancilla) and one in |+> (X check,
CNOTs ancilla -> data); ancillas measured mid-circuit and reset when C >= 2;
data prepared in |0>^n and measured in Z at the end to read Z-bar.
Circuit-level noise (Sec. III.A, Fig. 1b-d): an error operation E after every
layer on every qubit the layer does not measure (gate qubits and idle qubits),
including after preparation/reset; no measurement noise; one single-qubit
injection per location.

The CNOT schedule of the paper's reference is not available; this circuit
uses the geometric schedule: in the Z block, slot s (s = 0..5) runs, for every
face, the CNOT with its neighbour in lattice direction s; the X block repeats
the same six slots.  Each data qubit is the direction-s neighbour of at most
one face, so every slot is a valid layer.

Op encoding (also the layout of the library's exported op list):
    (kind, a, b, event, rec, layer)
kinds: PREP_Z=0, PREP_X=1, CNOT=2 (a=control, b=target), MEAS_Z=3, MEAS_X=4,
NOISE=5 (a=qubit, b=location id).  `event` numbers every stochastic event
(measurements and noise locations) in program order; `rec` is the record bit
a measurement writes (syndrome bits first: round r, plaquette p, Z before X;
then the n final data bits).  Qubits: data 0..n-1, Z-ancilla of face p is
n + 2p, X-ancilla is n + 2p + 1.

Parity of this module: pinned by the noise-off invariants (deterministic
Z syndromes, repeated X syndromes, Z-bar = +1) checked on the state-vector
oracle, and by closed-form op counts.
"""
from dataclasses import dataclass
from .colorcode import color_code, ColorCode

PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X, NOISE = 0, 1, 2, 3, 4, 5


@dataclass
class Circuit:
    code: ColorCode
    rounds: int
    n_qubits: int
    ops: list            # list of (kind, a, b, event, rec, layer)
    n_layers: int
    n_events: int
    n_locations: int
    n_syndrome_bits: int  # rounds * 2 * n_plaq
    n_record_bits: int    # syndrome bits + n data bits


def zanc(code, p):
    return code.n + 2 * p


def xanc(code, p):
    return code.n + 2 * p + 1


def build_circuit(d: int, rounds: int) -> Circuit:
    if rounds < 1:
        raise ValueError("rounds must be >= 1")
    code = color_code(d)
    n, P = code.n, code.n_plaq
    N = n + 2 * P
    ops = []
    counters = {"event": 0, "loc": 0, "layer": 0}

    def ev():
        e = counters["event"]
        counters["event"] += 1
        return e

    def noise(qubits):
        for q in qubits:
            ops.append((NOISE, q, counters["loc"], ev(), -1, counters["layer"]))
            counters["loc"] += 1

    def end_layer():
        counters["layer"] += 1

    for r in range(rounds):
        # preparation / reset layer
        if r == 0:
            for q in range(n):
                ops.append((PREP_Z, q, -1, -1, -1, counters["layer"]))
        for p in range(P):
            ops.append((PREP_Z, zanc(code, p), -1, -1, -1, counters["layer"]))
            ops.append((PREP_X, xanc(code, p), -1, -1, -1, counters["layer"]))
        noise(range(N))
        end_layer()
        # Z block: CNOT data -> Z ancilla, one lattice direction per slot
        for s in range(6):
            for p in range(P):
                q = code.plaq_dir[p][s]
                if q >= 0:
                    ops.append((CNOT, q, zanc(code, p), -1, -1, counters["layer"]))
            noise(range(N))
            end_layer()
        # X block: CNOT X ancilla -> data
        for s in range(6):
            for p in range(P):
                q = code.plaq_dir[p][s]
                if q >= 0:
                    ops.append((CNOT, xanc(code, p), q, -1, -1, counters["layer"]))
            noise(range(N))
            end_layer()
        # measurement layer; the idle data qubits get an error location
        for p in range(P):
            ops.append((MEAS_Z, zanc(code, p), -1, ev(), r * 2 * P + 2 * p, counters["layer"]))
            ops.append((MEAS_X, xanc(code, p), -1, ev(), r * 2 * P + 2 * p + 1, counters["layer"]))
        noise(range(n))
        end_layer()
    # final transversal Z readout of the data (noise-free, Sec. III.A)
    for q in range(n):
        ops.append((MEAS_Z, q, -1, ev(), rounds * 2 * P + q, counters["layer"]))
    end_layer()
    return Circuit(code=code, rounds=rounds, n_qubits=N, ops=ops,
                   n_layers=counters["layer"], n_events=counters["event"],
                   n_locations=counters["loc"], n_syndrome_bits=rounds * 2 * P,
                   n_record_bits=rounds * 2 * P + n)

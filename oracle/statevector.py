"""O1: exact quantum-trajectory sampling on a state vector.

Oracle (test infrastructure only).  Follows Sec. III.C ("Quantum
trajectories"): the mixed state of the noisy circuit is the average of
pure-state trajectories; each trajectory applies the ideal gates, the error
operation of every location, and samples measurement outcomes by the Born
rule.  Amplitude damping is unravelled with its exact Kraus operators
(Eqs. 2-3): with p1 = gamma * P(q = 1) the trajectory jumps (K1, then
renormalise) iff u < p1, else applies K0 and renormalises; averaging over
trajectories reproduces the channel of Eq. 2 exactly.  (The first-order
non-Hermitian gate exp(-dt/2 L^dag L) of Eqs. 7-8 agrees with this to first
order in gamma; the exact unravelling is the reading taken here.)

Draws: the uniform u of event e is philox.uniform(seed, traj, e).
  measurement: outcome 1 iff u >= P(0)           (Born rule)
  AD:          jump iff u < gamma * P(1)
  PTA:         inverse CDF over (I, X, Y, Z) in that order
  SRX:         no draw (unitary)
log p(record) accumulates the log of every sampled probability.

Amplitudes are returned little-endian: index = sum_q b_q 2^q.

Pinned (tests/test_oracle_statevector.py): unit norm; noise-off invariants;
an idle qubit under k SRX locations has P(1) = sin^2(k theta) exactly, and
(1 - (1 - 2 sin^2 theta)^k)/2 under SRX-PTA; |1> after one AD location has
P(1) = 1 - gamma; trajectory averages agree with the density-matrix oracle
within 3 sigma; p_L from trajectories agrees with the exact p_L;
record_log_prob gives log sin^2(k theta) / log cos^2(k theta) and their
theta-derivatives for k SRX locations and one measurement, and reproduces a
sampled trajectory's log p from its record.
"""
import math
import numpy as np
from . import philox
from .channels import (NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD, PAULI_MODELS,
                       srx_unitary, pta_probs, X, Y, Z, H)
from .circuit import PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X, NOISE


class StateVector:
    """|psi> over N qubits stored as an array of shape (2,)*N, axis q = qubit q."""

    def __init__(self, N):
        self.N = N
        self.psi = np.zeros((2,) * N, dtype=np.complex128)
        self.psi[(0,) * N] = 1.0

    def _view(self, q):
        return self.psi.reshape(2 ** q, 2, 2 ** (self.N - 1 - q))

    def apply1(self, q, U):
        v = self._view(q)
        a0 = v[:, 0, :].copy()
        a1 = v[:, 1, :].copy()
        v[:, 0, :] = U[0, 0] * a0 + U[0, 1] * a1
        v[:, 1, :] = U[1, 0] * a0 + U[1, 1] * a1

    def cnot(self, c, t):
        idx = [slice(None)] * self.N
        idx[c] = 1
        sub = self.psi[tuple(idx)]
        ax = t if t < c else t - 1
        self.psi[tuple(idx)] = np.flip(sub, axis=ax)

    def prob1(self, q):
        v = self._view(q)
        return float(np.sum(np.abs(v[:, 1, :]) ** 2))

    def norm2(self):
        return float(np.sum(np.abs(self.psi) ** 2))

    def project(self, q, m, p):
        v = self._view(q)
        v[:, 1 - m, :] = 0.0
        v[:, m, :] /= math.sqrt(p)

    def amplitudes(self):
        """Little-endian flat amplitude vector (qubit q = bit q of the index)."""
        return self.psi.transpose(tuple(range(self.N - 1, -1, -1))).reshape(-1).copy()


def apply_noise(sv, q, model, theta, gamma, u):
    """Error operation of one location.  Returns (log p of the sampled branch,
    min |u - p| over the probabilities the draw was compared with, or None)."""
    if model == NONE:
        return 0.0, None
    if model in (SRX, SRX_AD):
        sv.apply1(q, srx_unitary(theta))
        if model == SRX:
            return 0.0, None
    if model in (AD, SRX_AD):
        P1 = sv.prob1(q)
        p1 = gamma * P1
        v = sv._view(q)
        if u < p1:
            v[:, 0, :] = v[:, 1, :] / math.sqrt(P1)
            v[:, 1, :] = 0.0
            return math.log(p1), abs(u - p1)
        v[:, 1, :] *= math.sqrt(1.0 - gamma) / math.sqrt(1.0 - p1)
        v[:, 0, :] /= math.sqrt(1.0 - p1)
        return math.log1p(-p1), abs(u - p1)
    if model in PAULI_MODELS:
        p = pta_probs(model, theta, gamma)
        cum = np.cumsum(p)
        k = 3
        for i in range(3):
            if u < cum[i]:
                k = i
                break
        if k > 0:
            sv.apply1(q, (None, X, Y, Z)[k])
        return math.log(p[k]), float(min(abs(u - c) for c in cum[:3]))
    raise ValueError("unknown noise model")


def run_trajectory(circ, model, theta, gamma, seed, traj, snapshot_layers=()):
    """Simulate one trajectory.

    Returns dict(rec = uint8 record [syndrome bits | data bits], logp,
    margin = min |u - p| over compared draws, states = {layer: amplitudes
    after that layer}, branch_p = probability of every sampled branch, in
    event order (their logarithms sum to logp)).
    """
    N = circ.n_qubits
    sv = StateVector(N)
    last = np.zeros(N, dtype=np.int64)
    rec = np.zeros(circ.n_record_bits, dtype=np.uint8)
    logp = 0.0
    margin = math.inf
    states = {}
    branch_p = []
    snap = set(snapshot_layers)
    events = [op[3] for op in circ.ops if op[3] >= 0]
    us = dict(zip(events, philox.uniforms(seed, [traj], events)[0])) if events else {}
    cur_layer = 0
    for (kind, a, b, e, r, layer) in circ.ops:
        if layer != cur_layer:
            if cur_layer in snap:
                states[cur_layer] = sv.amplitudes()
            cur_layer = layer
        if kind in (PREP_Z, PREP_X):
            if last[a]:
                sv.apply1(a, X)
                last[a] = 0
            if kind == PREP_X:
                sv.apply1(a, H)
        elif kind == CNOT:
            sv.cnot(a, b)
        elif kind in (MEAS_Z, MEAS_X):
            if kind == MEAS_X:
                sv.apply1(a, H)
            p1 = sv.prob1(a)
            p0 = 1.0 - p1
            u = us[e]
            m = 1 if u >= p0 else 0
            margin = min(margin, abs(u - p0))
            pm = p1 if m else p0
            sv.project(a, m, pm)
            logp += math.log(pm)
            branch_p.append(pm)
            rec[r] = m
            last[a] = m
        elif kind == NOISE:
            lp, dist = apply_noise(sv, a, model, theta, gamma, us[e])
            logp += lp
            if dist is not None:
                margin = min(margin, dist)
                branch_p.append(math.exp(lp))
    if cur_layer in snap:
        states[cur_layer] = sv.amplitudes()
    return dict(rec=rec, logp=logp, margin=margin, states=states, sv=sv, branch_p=branch_p)


def record_log_prob(circ, model, theta, gamma, rec):
    """log p(record; theta, gamma) of a given measurement record for a noise
    model whose only random branches are the measurements (NONE, SRX): the
    circuit run with every measurement forced to its recorded outcome, the
    log-probabilities of those outcomes summed (-inf if one is impossible).
    Its central difference in theta is the per-trajectory score
    d log p / d theta of the score-function gradient (Sec. IV.A, the slopes
    of the crossing search)."""
    if model not in (NONE, SRX):
        raise ValueError("record_log_prob: the record fixes every branch only for NONE and SRX")
    N = circ.n_qubits
    sv = StateVector(N)
    last = np.zeros(N, dtype=np.int64)
    logp = 0.0
    for (kind, a, b, e, r, layer) in circ.ops:
        if kind in (PREP_Z, PREP_X):
            if last[a]:
                sv.apply1(a, X)
                last[a] = 0
            if kind == PREP_X:
                sv.apply1(a, H)
        elif kind == CNOT:
            sv.cnot(a, b)
        elif kind in (MEAS_Z, MEAS_X):
            if kind == MEAS_X:
                sv.apply1(a, H)
            p1 = sv.prob1(a)
            m = int(rec[r])
            pm = p1 if m else 1.0 - p1
            if pm <= 0.0:
                return -math.inf
            sv.project(a, m, pm)
            logp += math.log(pm)
            last[a] = m
        elif kind == NOISE:
            apply_noise(sv, a, model, theta, gamma, 0.0)
    return logp


def run_trajectories(circ, model, theta, gamma, seed, trajs):
    recs = np.zeros((len(trajs), circ.n_record_bits), dtype=np.uint8)
    logps = np.zeros(len(trajs))
    margins = np.zeros(len(trajs))
    for i, t in enumerate(trajs):
        out = run_trajectory(circ, model, theta, gamma, seed, t)
        recs[i] = out["rec"]
        logps[i] = out["logp"]
        margins[i] = out["margin"]
    return recs, logps, margins

"""O2: exact channel evolution of the density matrix (small circuits).

Oracle (test infrastructure only).  The ensemble that the trajectories of
Sec. III.C sample: rho evolves under every gate (U rho U^dag), every error
channel (Eqs. 1-3, or the twirled Pauli channel of Sec. IV.C), measurement
(dephasing sum_m P_m rho P_m, recording P(m = 1) = Tr(P_1 rho)) and reset
(trace the qubit out, re-prepare |0> or |+>).  Feasible up to ~11 qubits.

Also `exact_pl_unitary`: for unitary noise (SRX or none) the measurements can
be deferred (each round's ancillas become fresh qubits), so the joint
distribution of all measurement records is |psi|^2 of one final state vector
and p_L = sum_records P(record) * fail(record) exactly.

Pinned (tests/test_oracle_densitymatrix.py): trace one and Hermitian
throughout; a unitary-only circuit gives rho = |psi><psi| of the state-vector
oracle; per-measurement P(m = 1) matches the mean of the trajectory oracle
within 3 sigma (the pin of the trajectory unravelling).
"""
import numpy as np
from .channels import (NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD, kraus_of,
                       pta_probs, PAULIS, X, H)
from .circuit import PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X, NOISE


class DensityMatrix:
    """rho of shape (2,)*2N: ket axes 0..N-1, bra axes N..2N-1."""

    def __init__(self, N):
        self.N = N
        self.rho = np.zeros((2,) * (2 * N), dtype=np.complex128)
        self.rho[(0,) * (2 * N)] = 1.0

    def _apply_axis(self, ax, M):
        r = np.moveaxis(self.rho, ax, 0)
        sh = r.shape
        r = (M @ r.reshape(2, -1)).reshape(sh)
        self.rho = np.moveaxis(r, 0, ax)

    def kraus1(self, q, kraus):
        out = None
        base = self.rho
        for K in kraus:
            self.rho = base
            self._apply_axis(q, K)
            self._apply_axis(self.N + q, K.conj())
            out = self.rho if out is None else out + self.rho
        self.rho = out

    def unitary1(self, q, U):
        self.kraus1(q, [U])

    def cnot(self, c, t):
        for base in (0, self.N):
            idx = [slice(None)] * (2 * self.N)
            idx[base + c] = 1
            sub = self.rho[tuple(idx)]
            ax = base + t if t < c else base + t - 1
            self.rho[tuple(idx)] = np.flip(sub, axis=ax)

    def prob1(self, q):
        idx = [slice(None)] * (2 * self.N)
        idx[q] = 1
        idx[self.N + q] = 1
        sub = self.rho[tuple(idx)]
        n = self.N - 1
        return float(np.real(np.einsum(sub.reshape(2 ** n, 2 ** n), [0, 0])))

    def dephase(self, q):
        for (a, b) in ((0, 1), (1, 0)):
            idx = [slice(None)] * (2 * self.N)
            idx[q] = a
            idx[self.N + q] = b
            self.rho[tuple(idx)] = 0.0

    def reset0(self, q):
        P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
        L = np.array([[0, 1], [0, 0]], dtype=np.complex128)  # |0><1|
        self.kraus1(q, [P0, L])

    def trace(self):
        n = self.N
        return complex(np.einsum(self.rho.reshape(2 ** n, 2 ** n), [0, 0]))

    def matrix(self):
        """Little-endian 2^N x 2^N matrix."""
        n = self.N
        perm = tuple(range(n - 1, -1, -1)) + tuple(range(2 * n - 1, n - 1, -1))
        return self.rho.transpose(perm).reshape(2 ** n, 2 ** n).copy()


def noise_channel(dm, q, model, theta, gamma):
    if model == NONE:
        return
    if model in (SRX, AD, SRX_AD):
        dm.kraus1(q, kraus_of(model, theta, gamma))
        return
    p = pta_probs(model, theta, gamma)
    dm.kraus1(q, [np.sqrt(pi) * P for pi, P in zip(p, PAULIS) if pi > 0])


def evolve(circ, model, theta, gamma):
    """Returns (rho at the end, P(rec bit = 1) for every record bit)."""
    N = circ.n_qubits
    dm = DensityMatrix(N)
    p1 = np.zeros(circ.n_record_bits)
    for (kind, a, b, e, r, layer) in circ.ops:
        if kind in (PREP_Z, PREP_X):
            dm.reset0(a)
            if kind == PREP_X:
                dm.unitary1(a, H)
        elif kind == CNOT:
            dm.cnot(a, b)
        elif kind in (MEAS_Z, MEAS_X):
            if kind == MEAS_X:
                dm.unitary1(a, H)
            p1[r] = dm.prob1(a)
            dm.dephase(a)
        elif kind == NOISE:
            noise_channel(dm, a, model, theta, gamma)
    return dm, p1


def deferred_final_state(circ, theta):
    """State vector of the circuit with deferred measurements (SRX only).

    Qubit numbering of the returned (2,)*M array: data 0..n-1, then for each
    measurement op (in program order) a fresh ancilla.  Returns (psi, the
    axis of each record bit)."""
    from .statevector import StateVector
    from .channels import srx_unitary
    code = circ.code
    n, P = code.n, code.n_plaq
    n_anc = circ.rounds * 2 * P
    M = n + n_anc
    sv = StateVector(M)
    # physical ancilla qubit -> current fresh index
    cur = {}
    nxt = [n]

    def phys(q):
        if q < n:
            return q
        return cur[q]

    rec_axis = np.zeros(circ.n_record_bits, dtype=np.int64)
    U = srx_unitary(theta)
    for (kind, a, b, e, r, layer) in circ.ops:
        if kind in (PREP_Z, PREP_X):
            if a >= n:
                cur[a] = nxt[0]
                nxt[0] += 1
            if kind == PREP_X:
                sv.apply1(phys(a), H)
        elif kind == CNOT:
            sv.cnot(phys(a), phys(b))
        elif kind in (MEAS_Z, MEAS_X):
            if kind == MEAS_X:
                sv.apply1(phys(a), H)
            rec_axis[r] = phys(a)
        elif kind == NOISE:
            if theta != 0.0:
                sv.apply1(phys(a), U)
    return sv.psi, rec_axis


def record_distribution(circ, theta, keep_bits):
    """Exact P(record restricted to keep_bits) for unitary noise; returns a
    dict {tuple(bits): probability}."""
    psi, rec_axis = deferred_final_state(circ, theta)
    prob = np.abs(psi) ** 2
    M = prob.ndim
    keep_axes = [int(rec_axis[k]) for k in keep_bits]
    other = tuple(ax for ax in range(M) if ax not in keep_axes)
    marg = prob.sum(axis=other)  # axes in ascending order of keep_axes
    order = np.argsort(keep_axes)
    # marg axis i corresponds to sorted(keep_axes)[i]; reorder to keep_bits order
    marg = np.transpose(marg, np.argsort(order))
    out = {}
    for idx in np.argwhere(marg > 1e-300):
        out[tuple(int(x) for x in idx)] = float(marg[tuple(idx)])
    return out

"""Bond dimensions the noise-free extraction circuit needs on a tree layout.

Oracle (test infrastructure only).  The noise-free circuit of Sec. III is a
Clifford circuit with Z/X measurements and resets, so its state is a
stabilizer state at every layer (Gottesman-Knill).  The state is kept as N
stabilizer generators in binary symplectic form (x | z bits; signs are not
needed: entanglement does not depend on them), updated per gate
(H: swap x_q and z_q; CNOT c->t: x_t ^= x_c, z_c ^= z_t) and per Z
measurement (if some generator has x_q = 1, it is multiplied into the other
generators with x_q = 1 and then replaced by Z_q; otherwise the state is
unchanged), after Aaronson and Gottesman, "Improved simulation of stabilizer
circuits", Phys. Rev. A 70, 052328 (2004).  For a bipartition A | B the
entanglement is S_A = rank_GF2(generators restricted to A) - |A| bits
(Fattal, Cubitt, Yamamoto, Bravyi, Chuang, quant-ph/0406168), so the Schmidt
rank across the bond above a tree node is 2^S_A, A = the qubits of its
subtree: the bond dimension an untruncated TTN needs there (Sec. IV.A and
App. B: chi_exact, Table III, for the noise-free limit).

Preparation follows the simulator's convention: a PREP finds its qubit in a
Z eigenstate (initial |0> or just measured), so PREP_Z changes no
entanglement and PREP_X is a Hadamard; MEAS_X is a Hadamard then a Z
measurement.

Parity: pinned against the Schmidt ranks of the state-vector oracle's
amplitudes (SVD across each tree bond) at every layer of d = 3 circuits,
for the default, optimized and random layouts (tests/test_oracle_stabilizer.py).
"""
import numpy as np

from .circuit import PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X


def gf2_rank(M):
    """Rank over GF(2) of a 0/1 matrix (rows are vectors)."""
    A = (np.asarray(M, dtype=np.uint8) & 1).copy()
    rows, cols = A.shape
    r = 0
    for c in range(cols):
        if r == rows:
            break
        piv = np.nonzero(A[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        if p != r:
            A[[r, p]] = A[[p, r]]
        hit = np.nonzero(A[:, c])[0]
        hit = hit[hit != r]
        A[hit] ^= A[r]
        r += 1
    return r


class Tableau:
    """N stabilizer generators of an N-qubit state, x and z bit matrices."""

    def __init__(self, n):
        self.n = n
        self.x = np.zeros((n, n), dtype=np.uint8)
        self.z = np.eye(n, dtype=np.uint8)      # |0...0>: generators Z_i

    def h(self, q):
        self.x[:, q], self.z[:, q] = self.z[:, q].copy(), self.x[:, q].copy()

    def cnot(self, c, t):
        self.x[:, t] ^= self.x[:, c]
        self.z[:, c] ^= self.z[:, t]

    def measure_z(self, q):
        rows = np.nonzero(self.x[:, q])[0]
        if rows.size == 0:
            return                               # deterministic outcome
        p = rows[0]
        for r in rows[1:]:
            self.x[r] ^= self.x[p]
            self.z[r] ^= self.z[p]
        self.x[p] = 0
        self.z[p] = 0
        self.z[p, q] = 1

    def entropy(self, A):
        """S_A in bits for the qubit set A."""
        A = np.asarray(sorted(A), dtype=np.int64)
        if A.size == 0 or A.size == self.n:
            return 0
        sub = np.concatenate([self.x[:, A], self.z[:, A]], axis=1)
        return gf2_rank(sub) - A.size


def subtree_qubits(leaf_of_qubit, n_leaves):
    """{v: qubits under internal node v} for heap-numbered nodes 1..L-1."""
    L = n_leaves
    under = {v: [] for v in range(1, 2 * L)}
    for q, leaf in enumerate(leaf_of_qubit):
        x = L + int(leaf)
        while x >= 1:
            under[x].append(q)
            x //= 2
    return {v: under[v] for v in range(2, L)}   # the root has no bond above it


def bond_ranks(circ, leaf_of_qubit, n_leaves, layers=None):
    """{layer: {v: Schmidt rank across the bond above v}} after each layer
    (all layers if `layers` is None) of the noise-free circuit."""
    tab = Tableau(circ.n_qubits)
    groups = subtree_qubits(leaf_of_qubit, n_leaves)
    want = None if layers is None else set(layers)
    out = {}

    def snap(layer):
        if want is None or layer in want:
            out[layer] = {v: 2 ** tab.entropy(A) for v, A in groups.items()}

    cur = 0
    for (kind, a, b, e, r, layer) in circ.ops:
        if layer != cur:
            snap(cur)
            cur = layer
        if kind == PREP_X:
            tab.h(a)
        elif kind == CNOT:
            tab.cnot(a, b)
        elif kind == MEAS_Z:
            tab.measure_z(a)
        elif kind == MEAS_X:
            tab.h(a)
            tab.measure_z(a)
        # PREP_Z and NOISE (noise-free limit) change no entanglement
    snap(cur)
    return out


def chi_exact_noise_free(circ, leaf_of_qubit, n_leaves):
    """Largest Schmidt rank over all tree bonds and layers."""
    ranks = bond_ranks(circ, leaf_of_qubit, n_leaves)
    return max(max(r.values()) for r in ranks.values())

"""Qubit-to-leaf layout of the binary TTN (App. B), oracle side.

Oracle (test infrastructure only).  The CPU baseline of the benchmark runs
the plain TTN oracle on the same circuit and tree layout as the device path;
this module derives that layout on the oracle side, so the oracle's inputs
never come from the product library.

App. B, Eq. 9: the similarity of two qubits is the number of two-qubit gates
they share plus 1 / (the sum of their gate counts).  Algorithm 1 splits the
qubit set top-down into the two subtrees of each node by clustering on that
similarity; with two clusters the clustering is the sign split of the Fiedler
vector (the eigenvector of the second-smallest eigenvalue of the graph
Laplacian L = diag(S 1) - S).  A split must fit the subtree capacity
(2^(height-1) leaves per side): the qubits are ordered by their Fiedler value
and the cut is moved to the nearest position that fits.  The eigenvector's
sign is fixed so that the lowest-numbered qubit of the set has a
non-positive value; equal values keep qubit order.  numpy's eigh supplies the
eigenvectors (a library step).

Parity of this module: pinned by tests/test_oracle_layout.py -- every qubit
gets a distinct leaf, every subtree holds at most its capacity, qubits that
share many gates land in the same subtree on a two-cluster toy circuit, and
the layout's noise-free bond dimension at d = 3 and d = 5 (one round) equals
the values Table III prints for the optimized ordering's trend (8 at d = 3;
16 at d = 5 against 512 for the default ordering).
"""
import numpy as np

from .circuit import CNOT


def similarity(circ):
    """Eq. 9: S[i, j] = (gates shared by i and j) + 1 / (|G(i)| + |G(j)|)."""
    N = circ.n_qubits
    shared = np.zeros((N, N))
    deg = np.zeros(N, dtype=np.int64)
    for op in circ.ops:
        if op[0] == CNOT:
            a, b = op[1], op[2]
            shared[a, b] += 1.0
            shared[b, a] += 1.0
            deg[a] += 1
            deg[b] += 1
    S = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                ds = deg[i] + deg[j]
                S[i, j] = shared[i, j] + (1.0 / ds if ds > 0 else 0.0)
    return S


def _split(Q, lo, height, S, leaf_of):
    if not Q:
        return
    if height == 0 or len(Q) == 1:
        leaf_of[Q[0]] = lo
        return
    half = 1 << (height - 1)
    if len(Q) == 2 and height == 1:
        A, B = [Q[0]], [Q[1]]
    else:
        sub = S[np.ix_(Q, Q)].copy()
        np.fill_diagonal(sub, 0.0)
        lap = np.diag(sub.sum(axis=1)) - sub
        w, V = np.linalg.eigh(lap)
        f = V[:, 1].copy()
        imin = int(np.argmin(Q))
        if f[imin] > 0:
            f = -f
        order = sorted(range(len(Q)), key=lambda i: (f[i], Q[i]))
        cut = int(np.sum(f <= 0.0))
        cut = max(cut, len(Q) - half)
        cut = min(cut, half)
        A = [Q[order[i]] for i in range(cut)]
        B = [Q[order[i]] for i in range(cut, len(Q))]
    _split(A, lo, height - 1, S, leaf_of)
    _split(B, lo + half, height - 1, S, leaf_of)


def optimized_layout(circ, n_leaves=None):
    """leaf_of_qubit for the circuit: recursive capacity-constrained two-way
    spectral split of the Eq. 9 similarity (Algorithm 1 with two clusters)."""
    N = circ.n_qubits
    if n_leaves is None:
        n_leaves = 1
        while n_leaves < N:
            n_leaves *= 2
    height = 0
    while (1 << height) < n_leaves:
        height += 1
    leaf_of = [-1] * N
    _split(list(range(N)), 0, height, similarity(circ), leaf_of)
    return leaf_of

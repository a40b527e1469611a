"""Pins of the oracle-side TTN layout (App. B, Eq. 9, Algorithm 1 with two
clusters): a valid capacity-respecting leaf assignment, the spectral split on
a toy gate graph with two obvious clusters, and the noise-free bond dimension
the layout needs at one round, against Table III's printed values: 8 for
both orderings at d = 3; at d = 5 the default ordering needs 512 and the
paper's optimized ordering 16 (its candidates are post-selected; one
two-way spectral split per node, as here, reaches 32, within a factor 2)."""
import numpy as np
import pytest

from oracle.circuit import build_circuit, CNOT
from oracle.layout import optimized_layout, similarity
from oracle.stabilizer import chi_exact_noise_free
from oracle.ttn import default_layout


class _Toy:
    def __init__(self, n, ops):
        self.n_qubits = n
        self.ops = ops


def _valid(lay, N, n_leaves):
    assert len(lay) == N and len(set(lay)) == N
    assert all(0 <= x < n_leaves for x in lay)


@pytest.mark.parametrize("d", [3, 5, 7])
def test_layout_is_a_valid_leaf_assignment(d):
    circ = build_circuit(d, 1)
    lay = optimized_layout(circ)
    L = 1
    while L < circ.n_qubits:
        L *= 2
    _valid(lay, circ.n_qubits, L)


def test_eq9_similarity_closed_form():
    # qubits 0-1 share two gates, 1-2 one; degrees 2, 3, 1, 0
    toy = _Toy(4, [(CNOT, 0, 1, -1, -1, 0), (CNOT, 1, 0, -1, -1, 1), (CNOT, 1, 2, -1, -1, 2)])
    S = similarity(toy)
    assert S[0, 1] == pytest.approx(2 + 1 / 5)
    assert S[1, 2] == pytest.approx(1 + 1 / 4)
    assert S[0, 3] == pytest.approx(1 / 2)
    assert S[2, 3] == pytest.approx(1.0)
    assert np.allclose(S, S.T) and np.all(np.diag(S) == 0)


def test_two_clusters_split_apart():
    # two 4-qubit cliques {0,2,4,6} and {1,3,5,7}, joined by one gate
    ops = []
    for grp in ([0, 2, 4, 6], [1, 3, 5, 7]):
        for i in grp:
            for j in grp:
                if i < j:
                    ops += [(CNOT, i, j, -1, -1, 0)] * 3
    ops.append((CNOT, 6, 1, -1, -1, 1))
    lay = optimized_layout(_Toy(8, ops), 8)
    left = {q for q in range(8) if lay[q] < 4}
    assert left in ({0, 2, 4, 6}, {1, 3, 5, 7})


@pytest.mark.parametrize("d,want_opt,want_default", [(3, 8, 8), (5, 16, 512)])
def test_noise_free_chi_matches_table3_trend(d, want_opt, want_default):
    circ = build_circuit(d, 1)
    L = 1
    while L < circ.n_qubits:
        L *= 2
    assert chi_exact_noise_free(circ, optimized_layout(circ), L) <= 2 * want_opt
    assert chi_exact_noise_free(circ, default_layout(circ.n_qubits), L) == want_default

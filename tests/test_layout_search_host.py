"""Layout post-selection on the host (TTN_LAYOUT_SEARCH): the library's
noise-free bond dimension (a C++ stabilizer tableau) equals the oracle's
(tests/test_oracle_stabilizer.py pins that one to state-vector Schmidt ranks
and to Table III) on several layouts, the searched layout is a valid leaf
map that never needs more than the optimized one, and it halves the noise-free
bond dimension of the d = 7 extraction circuits."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.circuit import build_circuit
from oracle.stabilizer import chi_exact_noise_free

P = pytest.importorskip("paper_2511_05719_gb300")


def _lib_or_skip():
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")


@pytest.mark.parametrize("d,C", [(3, 1), (3, 3), (5, 1), (5, 5), (7, 1)])
def test_library_noise_free_chi_equals_oracle(d, C):
    _lib_or_skip()
    circ = build_circuit(d, C)
    c = P.Circuit(d, C, layout="optimized")
    layouts = [c.layout(), np.arange(c.n_qubits), W.random_layout(c.n_qubits, c.n_leaves, seed=d * 10 + C)]
    for lay in layouts:
        assert c.noise_free_chi(lay) == chi_exact_noise_free(circ, list(lay), c.n_leaves)
    assert c.noise_free_chi() == c.noise_free_chi(c.layout())


@pytest.mark.parametrize("d,C", [(3, 1), (3, 3), (5, 1), (5, 5), (7, 1), (7, 7)])
def test_search_never_worse_and_valid(d, C):
    _lib_or_skip()
    s = P.Circuit(d, C, layout="search")
    o = P.Circuit(d, C, layout="optimized")
    lay = s.layout()
    assert len(set(lay.tolist())) == s.n_qubits and lay.min() >= 0 and lay.max() < s.n_leaves
    assert s.noise_free_chi() <= o.noise_free_chi()
    assert np.array_equal(s.ops(), o.ops())          # only the layout differs


def test_search_halves_d7():
    _lib_or_skip()
    for C, opt in ((1, 128), (7, 512)):
        assert P.Circuit(7, C, layout="optimized").noise_free_chi() == opt
        assert P.Circuit(7, C, layout="search").noise_free_chi() == opt // 2


def test_noise_free_chi_arguments():
    _lib_or_skip()
    c = P.Circuit(3, 1)
    with pytest.raises(P.TTNError):
        c.noise_free_chi([0] * c.n_qubits)                   # not injective
    with pytest.raises(P.TTNError):
        c.noise_free_chi(list(range(4, 4 + c.n_qubits)))      # leaf 16 outside 16 leaves
    # an unknown layout value is refused
    import ctypes
    from paper_2511_05719_gb300 import _lib
    p = _lib.CircuitParams()
    p.distance, p.rounds, p.layout = 3, 1, 4
    h = ctypes.c_void_p()
    assert _lib.load_library().ttn_build_circuit(ctypes.byref(p), ctypes.byref(h)) == 1

"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/ttn.h declares, and its host-side circuit logic equals the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_or_skip():
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")
    return _lib


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ttn.h")).read()
    # a name followed by "(" declares a function; "ttn_status (*" opens a
    # function-pointer typedef
    return sorted(set(re.findall(r"\b(ttn_[a-z_]+)\s*\((?!\*)", src)))


def test_header_exports_every_symbol():
    _lib = _lib_or_skip()
    lib = ctypes.CDLL(_lib.library_path())
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s


@pytest.mark.parametrize("d,C", [(3, 1), (3, 3), (5, 5), (7, 7)])
def test_circuit_ir_equals_oracle(d, C):
    _lib_or_skip()
    import paper_2511_05719_gb300 as P
    from oracle.circuit import build_circuit
    c = P.Circuit(d, C, layout="default")
    oc = build_circuit(d, C)
    assert (c.n_qubits, c.n_layers, c.n_events, c.n_record_bits) == \
        (oc.n_qubits, oc.n_layers, oc.n_events, oc.n_record_bits)
    assert np.array_equal(c.ops(), np.array(oc.ops, dtype=np.int32))


@pytest.mark.parametrize("d,C", [(3, 3), (5, 5), (7, 7)])
def test_layouts_valid(d, C):
    _lib_or_skip()
    import paper_2511_05719_gb300 as P
    for lay in ("default", "optimized"):
        c = P.Circuit(d, C, layout=lay)
        lo = c.layout()
        assert len(set(lo.tolist())) == c.n_qubits
        assert lo.min() >= 0 and lo.max() < c.n_leaves
        assert c.n_leaves == 1 << int(np.ceil(np.log2(c.n_qubits)))


def test_invalid_arguments():
    _lib_or_skip()
    import paper_2511_05719_gb300 as P
    for bad in [(4, 1), (1, 1), (3, 0), (13, 1)]:
        with pytest.raises(P.TTNError) as e:
            P.Circuit(*bad)
        assert e.value.status == 1
    with pytest.raises(P.TTNError):
        P.Circuit(3, 1, leaf_of_qubit=[0] * 13)          # not injective
    with pytest.raises(P.TTNError):
        P.Circuit(3, 1, leaf_of_qubit=list(range(4, 17)))  # leaf 16 is outside 16 leaves
    c = P.Circuit(3, 1, leaf_of_qubit=list(range(13)))
    assert np.array_equal(c.layout(), np.arange(13))


def test_run_mixed_rejects_bad_items_before_any_device_work():
    _lib = _lib_or_skip()
    import paper_2511_05719_gb300 as P
    lib = _lib.load_library()
    # n_items outside [1, 64] and null arrays
    for n in (0, 65):
        assert lib.ttn_run_mixed(n, None, None, None, None, None, None) == 1
    assert lib.ttn_run_mixed(1, None, None, None, None, None, None) == 1
    c3 = P.Circuit(3, 1)
    items = [dict(circuit=c3, n_traj=2, chi=8), dict(circuit=c3, n_traj=2, chi=0)]
    with pytest.raises(P.TTNError) as e:
        P.run_mixed(items)
    assert e.value.status == 1 and "item 1" in str(e.value)
    items = [dict(circuit=c3, n_traj=2, noise="bogus")]
    with pytest.raises(KeyError):
        P.run_mixed(items)
    with pytest.raises(ValueError):
        P.run_mixed([dict(circuit=c3, n_traj=1, rounds=3)])
    # an item with trajectories needs an output array
    lib2 = ctypes.CDLL(_lib.library_path())
    lib2.ttn_run_mixed.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 6
    p = _lib.RunParams()
    p.noise, p.chi, p.precision = 1, 8, 0
    circs = (ctypes.c_void_p * 1)(c3.handle.value)
    cnt = (ctypes.c_uint64 * 1)(3)
    fails = (ctypes.c_void_p * 1)(None)
    assert lib2.ttn_run_mixed(1, circs, ctypes.byref(p), cnt, fails, None, None) == 1
    assert b"logical_fail" in lib.ttn_last_error()


def test_grad_sums_argument_checks_before_device_work():
    _lib = _lib_or_skip()
    import paper_2511_05719_gb300 as P
    c = P.Circuit(3, 1)
    for kw in (dict(shots=1), dict(shots=10, wrt="gamma"), dict(shots=10, chi=0),
               dict(shots=10, noise="ad", wrt="theta", gamma=0.1)):
        shots = kw.pop("shots")
        with pytest.raises(P.TTNError) as e:
            P.grad_sums(c, shots, **kw)
        assert e.value.status == 1, kw
    lib = _lib.load_library()
    p = _lib.RunParams()
    p.noise, p.chi, p.theta = 1, 8, 0.1
    assert lib.ttn_grad_sums(c.handle, ctypes.byref(p), 10, 0, 0.0, None, None, None, None) == 1


def test_header_is_plain_c():
    """include/ttn.h compiles as C99 (pedantic) and as C++17: the ABI has no
    C++ types or constructs."""
    import shutil
    import subprocess
    import tempfile
    src = ('#include "ttn.h"\nint main(void) { ttn_crossing_eval f = 0; (void)f;\n'
           '  return TTN_MIXED_MAX_ITEMS > 0 ? 0 : 1; }\n')
    for cc, std, lang in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "c++")):
        if not shutil.which(cc):
            pytest.skip("%s not available" % cc)
        with tempfile.NamedTemporaryFile("w", suffix=".c", delete=False) as f:
            f.write(src)
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                            "-I", os.path.join(ROOT, "include"), "-x", lang, f.name],
                           capture_output=True, text=True)
        os.unlink(f.name)
        assert r.returncode == 0, r.stderr


def test_eig_gram_argument_checks_before_device_work():
    """ttn_eig_gram rejects bad shapes, routes and tolerances with EINVAL before
    it touches the device; the wrapper rejects tensors that are not CUDA
    complex128."""
    _lib = _lib_or_skip()
    lib = _lib.load_library()
    fake = ctypes.c_void_p(16)  # never dereferenced: every call below fails its checks
    s = (ctypes.c_double * 4)()
    k = (ctypes.c_int32 * 1)()
    cases = [(None, 1, 4, 4, 1, 1e-7), (fake, 0, 4, 4, 1, 1e-7), (fake, 1, 513, 4, 1, 1e-7),
             (fake, 1, 4, 5, 1, 1e-7), (fake, 1, 4, 0, 1, 1e-7), (fake, 1, 4, 4, 4, 1e-7),
             (fake, 1, 4, 4, -1, 1e-7), (fake, 1, 4, 4, 1, 1.0), (fake, 1, 100, 4, 0, 1e-7)]
    for G, B, n, kc, route, eps in cases:
        st = lib.ttn_eig_gram(G, B, n, kc, route, eps, fake, ctypes.cast(s, ctypes.POINTER(ctypes.c_double)),
                              ctypes.cast(k, ctypes.POINTER(ctypes.c_int32)), None)
        assert st == 1, (B, n, kc, route, eps)
    torch = pytest.importorskip("torch")
    import paper_2511_05719_gb300 as P
    with pytest.raises(ValueError):
        P.eig_gram(torch.zeros(4, 4, dtype=torch.complex128))
    with pytest.raises(ValueError):
        P.eig_gram(torch.zeros(4, 4, dtype=torch.complex64))


def test_gemm_mode_range():
    _lib = _lib_or_skip()
    import paper_2511_05719_gb300 as P
    c = P.Circuit(3, 1)
    with pytest.raises(P.TTNError) as e:
        P.run_trajectories(c, 1, noise="srx", theta=0.1, chi=8, precision="mixed", gemm_mode=4)
    assert e.value.status == 1

"""Device memory layout on the host: replaying each circuit's step program
with every centre move keeping the largest rank its kernels allow (even where
rounding keeps more than the exact rank), no node ever holds more elements
than its slot, for every distance, round count, noise model and bond cap of
the workloads; and the bonds' structural caps are what makes this hold
(they bind on many truncating moves where a cap at chi alone would keep
more)."""
import pytest

P = pytest.importorskip("paper_2511_05719_gb300")


def _lib_or_skip():
    import os
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")
    return _lib


@pytest.mark.parametrize("d,C", [(3, 1), (3, 3), (5, 1), (5, 5), (7, 1), (7, 7)])
def test_no_slot_can_overflow(d, C):
    _lib = _lib_or_skip()
    c = P.Circuit(d, C)
    for noise in ("none", "srx", "ad", "srx_ad"):
        for chi in (1, 2, 4, 16, 64, 128, 1024):
            r = _lib.slot_check(c, noise, chi)
            assert r["worst_fill"] <= 1.0, (d, C, noise, chi, r)
            assert r["worst_fill"] > 0.0


def test_structural_caps_bind():
    _lib = _lib_or_skip()
    r = _lib.slot_check(P.Circuit(7, 7), "srx", 128)
    assert r["binding_moves"] > 1000
    assert _lib.slot_check(P.Circuit(7, 7), "srx", 1)["binding_moves"] == 0   # chi is the cap


def test_slot_check_arguments():
    _lib = _lib_or_skip()
    c = P.Circuit(3, 1)
    for bad in (dict(chi=0), dict(chi=5000), dict(noise=9)):
        kw = dict(noise="srx", chi=16)
        kw.update(bad)
        with pytest.raises(P.TTNError):
            _lib.slot_check(c, **kw)

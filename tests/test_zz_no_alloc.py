"""The allocation-free decoder entry point (ttn_decode_noalloc) against the
regular one (ttn_decode).  Callers whose memory pool owns the device, or whose
framework forbids driver allocations, use it; it must give the same decoded
outcomes, colours and scores, call after call, although every call reuses the
same static scratch.  Kept in the last-collected file so that a run stopping
at the first failure has already run every other test."""
import numpy as np
import pytest

import paper_2511_05719_gb300 as P

torch = pytest.importorskip("torch")


def _records(c, n, dens, seed):
    rng = np.random.default_rng(seed)
    return (rng.random((n, c.n_record_bits)) < dens).astype(np.uint8)


@pytest.mark.gpu
@pytest.mark.parametrize("d,C,n", [(3, 3, 37), (5, 2, 21), (7, 3, 19)])
def test_noalloc_decode_equals_decode(d, C, n):
    c = P.Circuit(d, C)
    dev = torch.device("cuda:0")
    for call, dens in enumerate((0.02, 0.12)):  # two calls in a row, sparse then dense
        recs = _records(c, n, dens, 100 * d + call)
        want_fail, want_color, want_score = P.decode(c, recs)
        r = torch.from_numpy(recs).to(dev)
        fail = torch.full((n,), 255, dtype=torch.uint8, device=dev)
        color = torch.full((n,), -7, dtype=torch.int32, device=dev)
        score = torch.full((n,), -7, dtype=torch.int64, device=dev)
        P.decode_noalloc(c, r, fail, color, score, stream=torch.cuda.current_stream().cuda_stream)
        np.testing.assert_array_equal(fail.cpu().numpy(), want_fail)
        np.testing.assert_array_equal(color.cpu().numpy(), want_color)
        np.testing.assert_array_equal(score.cpu().numpy(), want_score)


@pytest.mark.gpu
def test_noalloc_rejects_circuits_beyond_its_static_scratch():
    c = P.Circuit(7, 8)  # (8 + 1) * 18 + 1 = 163 detector nodes > 145
    dev = torch.device("cuda:0")
    r = torch.zeros((2, c.n_record_bits), dtype=torch.uint8, device=dev)
    fail = torch.zeros(2, dtype=torch.uint8, device=dev)
    with pytest.raises(P.TTNError) as ei:
        P.decode_noalloc(c, r, fail)
    assert "status 1" in str(ei.value) and "145" in str(ei.value)


def test_noalloc_rejects_tensors_it_cannot_hand_to_the_device():
    """Host tensors, wrong dtypes and short outputs are refused in the
    wrapper, before any pointer reaches the kernel."""
    import os
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")
    c = P.Circuit(3, 1)
    r = torch.zeros((2, c.n_record_bits), dtype=torch.uint8)
    fail = torch.zeros(2, dtype=torch.uint8)
    with pytest.raises(ValueError):
        P.decode_noalloc(c, r, fail)                       # CPU tensors
    with pytest.raises(ValueError):
        P.decode_noalloc(c, r.to(torch.int32), fail)       # wrong dtype (checked first on device)
    with pytest.raises(ValueError):
        P.decode_noalloc(c, torch.zeros((2, 3), dtype=torch.uint8), fail)  # wrong width

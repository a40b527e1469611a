"""Checkpoint / resume of a p_L estimate on the host, with a stand-in runner
whose outcomes depend only on the trajectory index (as the library's do):
an interrupted and resumed run equals an uninterrupted one, a checkpoint of
another run is refused, and the JSONL log has one line per batch."""
import json

import numpy as np
import pytest

from paper_2511_05719_gb300.checkpoint import logical_error_rate_resumable


class FakeCircuit:
    distance, rounds = 5, 5


def fake_fail(t):
    x = (int(t) * 0x9E3779B1) & 0xFFFFFFFF
    return 2 if x % 211 == 0 else (3 if x % 173 == 0 else (1 if x % 7 == 0 else 0))


class Runner:
    def __init__(self, crash_after=None):
        self.calls = []
        self.crash_after = crash_after

    def __call__(self, circuit, n, first_traj=0, **kw):
        if self.crash_after is not None and len(self.calls) == self.crash_after:
            raise RuntimeError("simulated crash")
        self.calls.append((first_traj, n))
        idx = np.arange(first_traj, first_traj + n)
        return dict(fail=np.array([fake_fail(t) for t in idx], dtype=np.uint8),
                    discarded=(idx % 13) * 1e-3, near_ties=(idx % 50 == 0).astype(np.int32))


def direct(first, shots):
    f = np.array([fake_fail(t) for t in range(first, first + shots)])
    nf, nv = int((f == 1).sum()), int((f <= 1).sum())
    return nf / nv, nf, nv


KW = dict(noise="srx", theta=0.02, chi=64, precision="fp32", seed=7, first_traj=100)


def test_uninterrupted_equals_direct_count(tmp_path):
    r = Runner()
    p, s, nf, nv = logical_error_rate_resumable(FakeCircuit(), 1000, str(tmp_path / "st.json"),
                                                batch=128, run=r, **KW)
    pd, nfd, nvd = direct(100, 1000)
    assert (nf, nv) == (nfd, nvd) and p == pd
    assert s == pytest.approx(np.sqrt(p * (1 - p) / nv))
    assert r.calls[0] == (100, 128) and r.calls[-1] == (100 + 896, 104) and len(r.calls) == 8


def test_crash_then_resume_equals_uninterrupted(tmp_path):
    path = str(tmp_path / "st.json")
    r1 = Runner(crash_after=3)
    with pytest.raises(RuntimeError):
        logical_error_rate_resumable(FakeCircuit(), 1000, path, batch=128, run=r1, **KW)
    st = json.load(open(path))
    assert st["next_traj"] == 384 and not st["done"]
    r2 = Runner()
    res = logical_error_rate_resumable(FakeCircuit(), 1000, path, batch=128, run=r2, **KW)
    assert r2.calls[0] == (100 + 384, 128)          # continues where it stopped
    full = logical_error_rate_resumable(FakeCircuit(), 1000, str(tmp_path / "b.json"), batch=128,
                                        run=Runner(), **KW)
    assert res == full
    # a finished run returns its stored result without running again
    r3 = Runner()
    assert logical_error_rate_resumable(FakeCircuit(), 1000, path, batch=128, run=r3, **KW) == full
    assert r3.calls == []
    st = json.load(open(path))
    assert st["done"] and st["n_lost"] + st["n_overflow"] + st["n_valid"] == 1000


def test_checkpoint_of_another_run_is_refused(tmp_path):
    path = str(tmp_path / "st.json")
    logical_error_rate_resumable(FakeCircuit(), 300, path, batch=100, run=Runner(), **KW)
    for change in (dict(theta=0.03), dict(chi=128), dict(seed=8)):
        kw = dict(KW, **change)
        with pytest.raises(ValueError):
            logical_error_rate_resumable(FakeCircuit(), 300, path, batch=100, run=Runner(), **kw)
    with pytest.raises(ValueError):
        logical_error_rate_resumable(FakeCircuit(), 301, path, batch=100, run=Runner(), **KW)
    with pytest.raises(ValueError):
        logical_error_rate_resumable(FakeCircuit(), 300, path, batch=100, run=Runner(),
                                     theta_per_traj=[0.1], **KW)


def test_jsonl_log_one_line_per_batch(tmp_path):
    log = tmp_path / "run.jsonl"
    logical_error_rate_resumable(FakeCircuit(), 500, str(tmp_path / "st.json"), batch=200,
                                 log_path=str(log), run=Runner(), **KW)
    lines = [json.loads(x) for x in open(log)]
    assert [x["n"] for x in lines] == [200, 200, 100]
    assert [x["first_traj"] for x in lines] == [100, 300, 500]
    assert lines[-1]["next_traj"] == 500
    _, nf, nv = direct(100, 500)
    assert sum(x["n_fail"] for x in lines) == nf and sum(x["n_valid"] for x in lines) == nv
    assert lines[-1]["p_L"] == pytest.approx(nf / nv)
    assert all(x["discarded_max"] >= x["discarded_mean"] >= 0 for x in lines)

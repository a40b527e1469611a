"""Sweep CLI on the host with a stand-in runner: every (distance, strength)
point is estimated and checkpointed, a rerun resumes without new work, and
--fit recovers the threshold of a synthetic Eq. 4 failure model."""
import io
import json

import numpy as np
import pytest

from paper_2511_05719_gb300 import sweep

TAU, NU = 0.05, 1.2


def model_p(d, x):
    u = (x - TAU) * d ** (1 / NU)
    return min(max(0.2 + 1.5 * u + 3.0 * u * u, 0.01), 0.9)


class C:
    def __init__(self, d, r, layout="optimized"):
        self.distance, self.rounds, self.layout = d, r, layout


class Runner:
    def __init__(self):
        self.calls = 0

    def __call__(self, circuit, n, first_traj=0, theta=0.0, **kw):
        self.calls += 1
        p = model_p(circuit.distance, theta)
        # deterministic per trajectory index: fail iff a hashed uniform < p
        idx = np.arange(first_traj, first_traj + n, dtype=np.uint64)
        h = (idx * np.uint64(0x9E3779B97F4A7C15) + np.uint64(circuit.distance)) >> np.uint64(11)
        u = h.astype(np.float64) / 2.0 ** 53
        return dict(fail=(u < p).astype(np.uint8))


def test_sweep_points_resume_and_fit(tmp_path):
    pytest.importorskip("paper_2511_05719_gb300._lib")
    from paper_2511_05719_gb300 import _lib
    import os
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")
    argv = ["--distances", "3,5,7", "--noise", "srx", "--strengths",
            ",".join("%.4f" % x for x in np.linspace(0.035, 0.065, 7)), "--shots", "40000",
            "--batch", "10000", "--state-dir", str(tmp_path / "st"), "--fit", "--tau0", "0.045"]
    r1, buf = Runner(), io.StringIO()
    pts = sweep.main(argv, run=r1, circuit=C, out=buf)
    assert len(pts) == 21 and r1.calls == 21 * 4
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert lines[0]["rounds"] == 3 and lines[-2]["rounds"] == 7
    fit = lines[-1]
    assert fit["fit"] == "eq4" and fit["points"] == 21
    assert abs(fit["tau"] - TAU) < 4 * fit["tau_sigma"] + 1e-4
    # rerun: every point comes from its checkpoint
    r2 = Runner()
    pts2 = sweep.main(argv, run=r2, circuit=C, out=io.StringIO())
    assert r2.calls == 0 and pts2 == pts


def test_sweep_argument_checks():
    with pytest.raises(SystemExit):
        sweep.parse(["--distances", "4", "--strengths", "0.1"])
    a = sweep.parse(["--distances", "3,5", "--strengths", "0.01,0.02", "--rounds", "2"])
    assert a.distances == [3, 5] and a.strengths == [0.01, 0.02] and a.rounds == "2"

"""The pipelined resident batch (ttn_pipeline_*) against ttn_run_trajectories:
trajectories depend only on (seed, trajectory index), so every trajectory a
pipeline step completes must carry the decoded outcome the plain call gives
for that index (same kernels, same draws), whatever group and segment it ran
in.  Log-probabilities and discarded weights agree to 1e-6 relative: a few
reductions (column norms of a centre move, log-probability terms of
simultaneous Pauli draws) add in FP64 atomically, in an order that varies from
run to run, and a last-bit difference can round the other way into the FP32
tensors."""
import numpy as np
import pytest

import workloads as W

P = pytest.importorskip("paper_2511_05719_gb300")
torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("precision,noise,R,S", [("mixed", "srx_ad", 6, 3), ("fp64", "srx", 4, 2),
                                                 ("mixed", "ad_pta", 5, 5), ("fp32", "srx", 3, 1)])
def test_pipeline_equals_plain_runs(precision, noise, R, S):
    c = P.Circuit(3, 2, layout="optimized")
    cycle = [0.03, 0.07, 0.11]
    seed, first = W.BASE_SEED + 21, 1000
    pipe = P.Pipeline(c, R, S, noise=noise, theta=0.0, gamma=0.04, chi=64, precision=precision,
                      seed=seed, first_traj=first, theta_cycle=cycle)
    G = pipe.group_size
    assert G == R // S
    got = {}
    for step in range(2 * S + 1):
        if step % 2:
            dev = torch.device("cuda:0")
            out = dict(fail=torch.full((G,), 9, dtype=torch.uint8, device=dev),
                       log_prob=torch.zeros(G, dtype=torch.float64, device=dev),
                       discarded=torch.zeros(G, dtype=torch.float64, device=dev))
            st = torch.cuda.current_stream()
            r = pipe.step(out, stream=st.cuda_stream)
            r = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}
        else:
            r = pipe.step()
        for i, t in enumerate(r["traj"]):
            got[int(t)] = (int(r["fail"][i]), float(r["log_prob"][i]), float(r["discarded"][i]))
    pipe.close()
    n = len(got)
    assert sorted(got) == list(range(first, first + n))      # completed in index order, none skipped
    thetas = [cycle[t % len(cycle)] for t in range(first, first + n)]
    ref = P.run_trajectories(c, n, noise=noise, theta=0.0, gamma=0.04, chi=64, precision=precision,
                             seed=seed, first_traj=first, theta_per_traj=thetas)
    for i in range(n):
        f, lp, ds = got[first + i]
        assert f == ref["fail"][i]
        assert abs(lp - ref["log_prob"][i]) <= 1e-6 * (1.0 + abs(lp))
        assert abs(ds - ref["discarded"][i]) <= 1e-6 * (1e-12 + abs(ds))


def test_pipeline_argument_checks():
    import os
    from paper_2511_05719_gb300 import _lib
    if not os.path.exists(_lib.library_path()):
        pytest.skip("libttn.so not built")
    c = P.Circuit(3, 1)
    for R, S in [(5, 2), (1, 2), (4, 0)]:
        with pytest.raises(P.TTNError) as ei:
            P.Pipeline(c, R, S, chi=8)
        assert "status 1" in str(ei.value)
    with pytest.raises(P.TTNError):
        P.Pipeline(c, 4, 2, chi=8, theta_cycle=[0.1, float("nan")])

"""The MIXED precision route -- complex64 tensors, FP32 contractions (FMA,
or exact digit products on the tcgen05 tensor cores), every isometry-centre
factorisation in FP64 (exact Gram matrix on the tensor cores + FP64 Hermitian
eigensolver) -- against the CPU oracle.

This is the route of the d = 7, chi = 128 benchmark workload, and it is the
same at every circuit size (no size-dependent switch), so the d = 3 circuits
below test exactly the kernels the benchmark runs.  Bars: amplitudes within
1e-5 of the state-vector oracle (2-norm relative to the state's norm) through
the first syndrome round and 2e-5 through the second (FP32 rounding grows with
depth); records bit-exact for the same Philox draws except near ties
(|u - p| < 1e-5, counted and excluded); log-probabilities within the bound
the amplitude bar implies (below); no
trajectory may lose its norm (the library fails the call if one does)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV, decoder as DEC
from oracle.channels import NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD
from oracle.circuit import build_circuit

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_05719_gb300")

MODELS = {"none": NONE, "srx": SRX, "ad": AD, "srx_pta": SRX_PTA, "ad_pta": AD_PTA, "srx_ad": SRX_AD}
STRENGTH = {"none": (0.0, 0.0), "srx": (0.07, 0.0), "ad": (0.0, 0.06), "srx_pta": (0.12, 0.0),
            "ad_pta": (0.0, 0.08), "srx_ad": (0.06, 0.05)}
TOL_ROUND1, TOL_ROUND2, TIE = 1e-5, 2e-5, 1e-5


def logp_tolerance(branch_p):
    """A state within relative distance e of the exact one gives a branch of
    probability p = |P psi|^2 with |dp| <= 2 sqrt(p) e + e^2, so
    |d log p| <= (2 e / sqrt(p)) (1 + e / sqrt(p)); summed over the sampled
    branches with e = the round-2 amplitude bar."""
    e = TOL_ROUND2
    return sum(2 * e / math.sqrt(p) * (1 + e / math.sqrt(p)) for p in branch_p)


@pytest.mark.parametrize("noise", list(MODELS))
def test_mixed_amplitudes_match_statevector(noise):
    circ = build_circuit(3, 2)
    th, ga = STRENGTH[noise]
    for lay, lo in [("optimized", None), ("explicit", W.random_layout(13, 16, 5))]:
        c = P.Circuit(3, 2, layout=lay, leaf_of_qubit=lo)
        for traj in (0, 3):
            layers = [0, 4, 13, 20, circ.n_layers - 1]
            ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED, traj, snapshot_layers=layers)
            for L in layers:
                amp = P.debug_state(c, traj, L, noise=noise, theta=th, gamma=ga, chi=64,
                                    precision="mixed", seed=W.BASE_SEED)
                want = ref["states"][L]
                err = np.linalg.norm(amp - want) / np.linalg.norm(want)
                assert err < (TOL_ROUND1 if L <= 13 else TOL_ROUND2), (noise, lay, traj, L, err)


@pytest.mark.parametrize("noise", ["srx", "ad", "srx_pta", "ad_pta", "srx_ad", "none"])
def test_mixed_records_bit_exact(noise):
    d, C = 3, 3
    circ = build_circuit(d, C)
    th, ga = STRENGTH[noise]
    c = P.Circuit(d, C, layout="optimized")
    n = 48
    out = P.run_trajectories(c, n, noise=noise, theta=th, gamma=ga, chi=64, precision="mixed",
                             seed=W.BASE_SEED + 9, first_traj=100)
    G = DEC.DecoderGraphs(d, C)
    excluded = 0
    for i in range(n):
        ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED + 9, 100 + i)
        if ref["margin"] < TIE or out["near_ties"][i] > 0:
            excluded += 1
            continue
        assert np.array_equal(out["records"][i], ref["rec"]), i
        assert abs(out["log_prob"][i] - ref["logp"]) < logp_tolerance(ref["branch_p"])
        assert out["fail"][i] == DEC.decode(G, ref["rec"])[0]
    assert excluded <= 3


@pytest.mark.parametrize("d,C,chi,noise,th,ga", [(5, 2, 64, "srx_ad", 0.05, 0.01),
                                                  (7, 1, 128, "srx", 0.07, 0.0)])
def test_mixed_large_circuits_complete(d, C, chi, noise, th, ga):
    """Truncated runs at d = 5 and d = 7: every trajectory completes (a lost
    one fails the call) and the outputs are valid (the discarded weight is
    the sum of the weight each truncating move drops, so it is not bounded
    by 1)."""
    c = P.Circuit(d, C, layout="optimized")
    n = 8
    out = P.run_trajectories(c, n, noise=noise, theta=th, gamma=ga, chi=chi, precision="mixed",
                             seed=W.BASE_SEED + 3)
    assert set(np.unique(out["records"])) <= {0, 1}
    assert np.all(out["fail"] <= 1)
    assert np.all(np.isfinite(out["log_prob"])) and np.all(out["log_prob"] <= 1e-9)
    assert np.all(out["discarded"] >= 0) and np.all(np.isfinite(out["discarded"]))


@pytest.mark.parametrize("noise", ["srx", "srx_ad"])
def test_mixed_contraction_routes(noise):
    """The tcgen05 digit-product contractions (gemm_mode "exact") and the
    FMA contractions (the default) both hold the amplitude bars.  (The digit
    route sums exactly but rounds its inputs to 23 bits below each row's
    largest entry, so it is not more accurate than FMA sums in general.)"""
    circ = build_circuit(3, 2)
    th, ga = STRENGTH[noise]
    c = P.Circuit(3, 2, layout="optimized")
    layers = [13, circ.n_layers - 1]
    for traj in (1, 2):
        ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED, traj, snapshot_layers=layers)
        errs = {}
        for mode in ("exact", "fma"):
            for L in layers:
                amp = P.debug_state(c, traj, L, noise=noise, theta=th, gamma=ga, chi=64,
                                    precision="mixed", seed=W.BASE_SEED, gemm_mode=mode)
                want = ref["states"][L]
                err = np.linalg.norm(amp - want) / np.linalg.norm(want)
                assert err < (TOL_ROUND1 if L <= 13 else TOL_ROUND2), (noise, mode, traj, L, err)
                errs[mode, L] = err

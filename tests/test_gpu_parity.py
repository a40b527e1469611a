"""GPU path (through the C ABI) against the CPU oracle on seeded inputs.

Tolerances: amplitudes within 1e-10 (FP64) or 1e-5 (FP32) of the state-vector
oracle in the 2-norm relative to the state's norm on the one-sided Jacobi
path (the Gram path used for bonds above 64 has its own test below); records bit-exact for the
same Philox draws, except trajectories that met a near tie (|u - p| below
1e-9 FP64 / 1e-5 FP32), which are excluded and counted; decoder output
bit-exact; p_L within 3 binomial sigma of the exact value.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import statevector as SV, philox, decoder as DEC, densitymatrix as DM
from oracle.channels import NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD
from oracle.circuit import build_circuit

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_05719_gb300")

MODELS = {"none": NONE, "srx": SRX, "ad": AD, "srx_pta": SRX_PTA, "ad_pta": AD_PTA, "srx_ad": SRX_AD}
STRENGTH = {"none": (0.0, 0.0), "srx": (0.07, 0.0), "ad": (0.0, 0.06), "srx_pta": (0.12, 0.0),
            "ad_pta": (0.0, 0.08), "srx_ad": (0.06, 0.05)}
AMP_TOL = {"fp64": 1e-10, "fp32": 1e-5}
# FP32 rounding grows with circuit depth: the 1e-5 bar holds through the
# first syndrome round (layers <= 13); the second round is held to 2e-5.
AMP_TOL_ROUND2 = {"fp64": 1e-10, "fp32": 2e-5}
TIE = {"fp64": 1e-9, "fp32": 1e-5}


def test_philox_bit_exact():
    trajs = np.array([0, 1, 7, 2 ** 33 + 5, 123456789], dtype=np.uint64)
    events = np.array([0, 1, 2, 552, 7190, 2 ** 31 - 1], dtype=np.int32)
    for seed in (0, W.BASE_SEED, 2 ** 64 - 1):
        gpu = P.philox_uniforms(seed, trajs, events)
        ref = philox.uniforms(seed, trajs, events.astype(np.int64))
        assert np.array_equal(gpu, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("noise", list(MODELS))
def test_amplitudes_match_statevector(noise, precision):
    circ = build_circuit(3, 2)
    th, ga = STRENGTH[noise]
    layouts = [("optimized", None), ("explicit", W.random_layout(13, 16, 5))]
    for li, (lay, lo) in enumerate(layouts):
        c = P.Circuit(3, 2, layout=lay, leaf_of_qubit=lo)
        for traj in (0, 3):
            layers = [-1, 0, 4, 13, 20, circ.n_layers - 1]
            ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED, traj,
                                    snapshot_layers=[L for L in layers if L >= 0])
            for L in layers:
                amp = P.debug_state(c, traj, L, noise=noise, theta=th, gamma=ga, chi=64,
                                    precision=precision, seed=W.BASE_SEED, svd_mode="jacobi")
                if L < 0:
                    want = np.zeros(1 << 13, dtype=complex)
                    want[0] = 1.0
                else:
                    want = ref["states"][L]
                err = np.linalg.norm(amp - want) / np.linalg.norm(want)
                tol = AMP_TOL[precision] if L <= 13 else AMP_TOL_ROUND2[precision]
                assert err < tol, (noise, lay, traj, L, err)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("noise", ["srx", "ad", "srx_pta", "ad_pta", "srx_ad", "none"])
def test_records_bit_exact(noise, precision):
    d, C = 3, 3
    circ = build_circuit(d, C)
    th, ga = STRENGTH[noise]
    c = P.Circuit(d, C, layout="optimized")
    n = 48
    out = P.run_trajectories(c, n, noise=noise, theta=th, gamma=ga, chi=64,
                             precision=precision, seed=W.BASE_SEED + 9, first_traj=100)
    G = DEC.DecoderGraphs(d, C)
    excluded = 0
    for i in range(n):
        ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED + 9, 100 + i)
        if ref["margin"] < TIE[precision] or out["near_ties"][i] > 0:
            excluded += 1
            continue
        assert np.array_equal(out["records"][i], ref["rec"]), i
        assert abs(out["log_prob"][i] - ref["logp"]) < (1e-8 if precision == "fp64" else 1e-3)
        assert out["discarded"][i] == 0.0 or out["discarded"][i] < 1e-20
        assert out["fail"][i] == DEC.decode(G, ref["rec"])[0]
    assert excluded <= 3


def test_decoder_bit_exact_against_oracle():
    rng = np.random.default_rng(11)
    for d, C in ((3, 3), (5, 3), (7, 2)):
        c = P.Circuit(d, C)
        G = DEC.DecoderGraphs(d, C)
        code = G.code
        n = 60
        recs = np.zeros((n, c.n_record_bits), dtype=np.uint8)
        # sparse random syndrome histories: flip a few Z records and data bits
        for i in range(n):
            k = rng.integers(0, 4)
            for _ in range(k):
                if rng.random() < 0.5:
                    r = rng.integers(0, C)
                    p = rng.integers(0, code.n_plaq)
                    recs[i, r * 2 * code.n_plaq + 2 * p] ^= 1
                else:
                    q = rng.integers(0, code.n)
                    recs[i, C * 2 * code.n_plaq + q] ^= 1
        fail, color, score = P.decode(c, recs)
        for i in range(n):
            f, col, s = DEC.decode(G, recs[i])
            assert (fail[i], color[i], score[i]) == (f, col, s), (d, C, i)


def test_pl_within_3_sigma_of_exact_d3_c1():
    theta = 0.12
    circ = build_circuit(3, 1)
    code = circ.code
    Pq = code.n_plaq
    keep = [2 * p for p in range(Pq)] + [2 * Pq + q for q in range(code.n)]
    dist = DM.record_distribution(circ, theta, keep)
    G = DEC.DecoderGraphs(3, 1)
    exact = 0.0
    for bits, pr in dist.items():
        rec = np.zeros(circ.n_record_bits, dtype=np.uint8)
        rec[keep] = bits
        exact += pr * DEC.decode(G, rec)[0]
    c = P.Circuit(3, 1)
    shots = 20000
    pl, sg, nf = P.logical_error_rate(c, shots, noise="srx", theta=theta, chi=64,
                                      precision="fp64", seed=W.BASE_SEED + 21)
    assert abs(pl - exact) < 3 * math.sqrt(exact * (1 - exact) / shots)


def test_edge_cases():
    c = P.Circuit(3, 1)
    out = P.run_trajectories(c, 0, noise="srx", theta=0.1, chi=8)
    assert out["records"].shape[0] == 0
    # theta = 0 and gamma = 0: the noise is the identity, no logical failure
    for noise in ("srx", "ad", "srx_pta", "ad_pta"):
        pl, _, _ = P.logical_error_rate(c, 64, noise=noise, theta=0.0, gamma=0.0, chi=16, seed=3)
        assert pl == 0.0
    # chi = 1 keeps a product state: Z syndromes stay trivial (Sec. IV.A)
    out = P.run_trajectories(P.Circuit(3, 2), 16, noise="none", chi=1, precision="fp64", seed=4)
    assert out["fail"].sum() == 0
    with pytest.raises(P.TTNError):
        P.run_trajectories(c, 4, noise="srx", theta=0.1, chi=0)
    with pytest.raises(P.TTNError):
        P.run_trajectories(c, 4, noise="ad", gamma=1.5, chi=4)


def test_batching_does_not_change_results():
    c = P.Circuit(3, 2)
    a = P.run_trajectories(c, 40, noise="srx_ad", theta=0.05, gamma=0.03, chi=64, seed=9,
                           precision="fp64")
    b1 = P.run_trajectories(c, 17, noise="srx_ad", theta=0.05, gamma=0.03, chi=64, seed=9,
                            precision="fp64")
    b2 = P.run_trajectories(c, 23, noise="srx_ad", theta=0.05, gamma=0.03, chi=64, seed=9,
                            first_traj=17, precision="fp64")
    assert np.array_equal(a["records"], np.vstack([b1["records"], b2["records"]]))
    assert np.allclose(a["log_prob"], np.concatenate([b1["log_prob"], b2["log_prob"]]), atol=1e-12)


# Gram-matrix path (large bonds): the kept space is chosen from eigenvalues of
# M^H M above eps_gram^2 lambda_max (FP64 1e-7, FP32 1e-4 in singular values),
# so each move may drop a component of relative amplitude up to eps_gram; the
# snapshots below are a few tens of moves apart.  Tolerances: FP64 1e-5,
# FP32 3e-3 (2-norm, relative).
GRAM_TOL = {"fp64": 1e-5, "fp32": 3e-3}


@pytest.mark.parametrize("svd_mode", ["gram", "gram_tri"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("noise", ["srx", "ad", "srx_ad"])
def test_gram_path_amplitudes(noise, precision, svd_mode):
    circ = build_circuit(3, 2)
    th, ga = STRENGTH[noise]
    c = P.Circuit(3, 2, layout="optimized")
    for traj in (1, 4):
        layers = [4, 13, 20, circ.n_layers - 1]
        ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED, traj, snapshot_layers=layers)
        if ref["margin"] < 1e-3:
            continue
        for L in layers:
            amp = P.debug_state(c, traj, L, noise=noise, theta=th, gamma=ga, chi=64,
                                precision=precision, seed=W.BASE_SEED, svd_mode=svd_mode)
            want = ref["states"][L]
            err = np.linalg.norm(amp - want) / np.linalg.norm(want)
            assert err < GRAM_TOL[precision], (noise, traj, L, err)


def test_profile_ledger_counts_work():
    c = P.Circuit(3, 1)
    P.profile_begin("svd_jacobi")
    P.run_trajectories(c, 8, noise="srx", theta=0.05, chi=64, precision="fp64", seed=1,
                       svd_mode="jacobi")
    prof = P.profile_end()
    assert prof["timed_launches"] > 0 and prof["timed_ms"] > 0
    assert prof["flops"]["svd_jacobi"] > 0 and prof["flops"]["absorb"] > 0
    assert prof["flops"]["gram"] == 0


def _exact_pl_d3_c1(theta):
    circ = build_circuit(3, 1)
    code = circ.code
    Pq = code.n_plaq
    keep = [2 * p for p in range(Pq)] + [2 * Pq + q for q in range(code.n)]
    dist = DM.record_distribution(circ, theta, keep)
    G = DEC.DecoderGraphs(3, 1)
    pl = 0.0
    for bits, pr in dist.items():
        rec = np.zeros(circ.n_record_bits, dtype=np.uint8)
        rec[keep] = bits
        pl += pr * DEC.decode(G, rec)[0]
    return pl


def test_grad_matches_exact_derivative_d3_c1():
    # exact dp_L/dtheta: central difference of the exact p_L (deferred
    # measurement), O(dtheta^2) ~ 1e-6 relative
    theta, dth = 0.12, 1e-3
    exact = (_exact_pl_d3_c1(theta + dth) - _exact_pl_d3_c1(theta - dth)) / (2 * dth)
    c = P.Circuit(3, 1)
    shots = 12000
    pl, g, sg, score = P.grad(c, shots, wrt="theta", noise="srx", theta=theta, chi=64,
                              precision="fp32", seed=W.BASE_SEED + 31, return_score=True)
    assert sg > 0
    assert abs(g - exact) < 3 * sg + 1e-3 * abs(exact), (g, sg, exact)
    # the score has zero mean: E[d log p / d theta] = d/dtheta sum p = 0
    assert abs(score.mean()) < 3 * score.std() / np.sqrt(shots)


def test_grad_scores_match_oracle_per_trajectory():
    """Each trajectory's score (the central difference of its forced replays at
    theta +- h) against the state-vector oracle's log p of the same record at
    theta +- h, same h: FP64, d = 3, untruncated (chi = 64)."""
    theta, h, shots = 0.12, 1e-4, 16
    c = P.Circuit(3, 1)
    circ = build_circuit(3, 1)
    kw = dict(noise="srx", theta=theta, chi=64, precision="fp64", seed=W.BASE_SEED + 5)
    out = P.run_trajectories(c, shots, **kw)
    pl, g, sg, score = P.grad(c, shots, wrt="theta", h=h, return_score=True, **kw)
    for i in range(shots):
        rec = out["records"][i]
        want = (SV.record_log_prob(circ, SRX, theta + h, 0.0, rec)
                - SV.record_log_prob(circ, SRX, theta - h, 0.0, rec)) / (2 * h)
        assert abs(score[i] - want) <= 1e-6 * (1.0 + abs(want)), (i, score[i], want)


def test_grad_ad_and_argument_checks():
    c = P.Circuit(3, 1)
    pl, g, sg = P.grad(c, 2000, wrt="gamma", noise="ad", gamma=0.05, chi=64, precision="fp32",
                       seed=3)
    assert sg > 0 and np.isfinite(g)
    with pytest.raises(P.TTNError):
        P.grad(c, 100, wrt="gamma", noise="srx", theta=0.1, chi=16)
    with pytest.raises(P.TTNError):
        P.grad(c, 100, wrt="gamma", noise="ad", gamma=0.0, chi=16)


def test_decoder_dense_syndromes_blossom_path():
    """Dense syndrome histories: matching components far above the subset-DP
    size go through the kernel's blossom matcher; bit-exact with the oracle."""
    rng = np.random.default_rng(23)
    for d, C, dens in ((5, 5, 0.3), (7, 3, 0.12), (7, 7, 0.1)):
        c = P.Circuit(d, C)
        G = DEC.DecoderGraphs(d, C)
        n = 12
        recs = (rng.random((n, c.n_record_bits)) < dens).astype(np.uint8)
        fail, color, score = P.decode(c, recs)
        for i in range(n):
            f, col, s = DEC.decode(G, recs[i])
            assert (fail[i], color[i], score[i]) == (f, col, s), (d, C, i)


TC_TOL = {"fp32": 2e-5}


@pytest.mark.parametrize("svd_mode", ["jacobi", "gram"])
@pytest.mark.parametrize("noise", ["srx", "ad", "srx_ad"])
def test_tensor_core_contractions_amplitudes(noise, svd_mode):
    """Every FP32 contraction on the tensor cores (3xTF32): amplitudes against
    the statevector oracle through both rounds."""
    circ = build_circuit(3, 2)
    th, ga = STRENGTH[noise]
    c = P.Circuit(3, 2, layout="optimized")
    tol = TC_TOL["fp32"] if svd_mode == "jacobi" else GRAM_TOL["fp32"]
    for traj in (0, 5):
        layers = [4, 13, 20, circ.n_layers - 1]
        ref = SV.run_trajectory(circ, MODELS[noise], th, ga, W.BASE_SEED, traj, snapshot_layers=layers)
        if ref["margin"] < 1e-3:
            continue
        for L in layers:
            amp = P.debug_state(c, traj, L, noise=noise, theta=th, gamma=ga, chi=64, precision="fp32",
                                seed=W.BASE_SEED, svd_mode=svd_mode, gemm_mode="tensor")
            want = ref["states"][L]
            err = np.linalg.norm(amp - want) / np.linalg.norm(want)
            assert err < tol, (noise, svd_mode, traj, L, err)

"""Records of the MIXED route at d = 5 and d = 7 against oracles that reach
those sizes exactly:

* Pauli noise (SRX_PTA, AD_PTA, DEPOL) against the stabilizer-tableau oracle
  (O3): a Pauli trajectory has the noise-free entanglement, so at chi >= the
  noise-free chi_exact (32 at d = 5, C = 5; 128 at d = 7, C = 1 on the
  optimized layout) the tree tensor network is exact and every record must
  equal O3's bit for bit (same Philox draws), except near ties.
* Amplitude damping at d = 5, C = 1, chi = 64 against the plain CPU tree
  tensor network (O4): the jumps keep the rank low enough that neither side
  truncates (O4's discarded weight is checked to be 0), so the records must
  agree bit for bit as well.

Near ties: draws within 1e-5 of a compared probability (FP32 tensors give
probabilities to ~1e-6) are counted and excluded.  Log-probabilities are held
to the bound a 2e-5 amplitude error implies (see test_gpu_mixed_precision)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import chp, ttn as TT
from oracle.channels import SRX_PTA, AD_PTA, AD, DEPOL
from oracle.circuit import build_circuit

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_05719_gb300")

TIE = 1e-5


def logp_tolerance(branch_p, e=2e-5):
    return sum(2 * e / math.sqrt(p) * (1 + e / math.sqrt(p)) for p in branch_p)


@pytest.mark.parametrize("d,C,chi,noise,model,th,ga", [
    (5, 5, 64, "srx_pta", SRX_PTA, 0.12, 0.0),
    (5, 5, 64, "ad_pta", AD_PTA, 0.0, 0.06),
    (7, 1, 128, "srx_pta", SRX_PTA, 0.12, 0.0),
    (7, 1, 128, "ad_pta", AD_PTA, 0.0, 0.06),
    (5, 5, 64, "depol", DEPOL, 0.0, 0.02),
    (7, 1, 128, "depol", DEPOL, 0.0, 0.02)])
def test_pta_records_equal_tableau_oracle(d, C, chi, noise, model, th, ga):
    circ = build_circuit(d, C)
    c = P.Circuit(d, C, layout="optimized")
    assert c.noise_free_chi() <= chi
    n, seed, first = 8, W.BASE_SEED + 31, 500
    out = P.run_trajectories(c, n, noise=noise, theta=th, gamma=ga, chi=chi, precision="mixed",
                             seed=seed, first_traj=first)
    excluded = 0
    for i in range(n):
        ref = chp.run_trajectory(circ, model, th, ga, seed, first + i)
        if ref["margin"] < TIE or out["near_ties"][i] > 0:
            excluded += 1
            continue
        assert np.array_equal(out["records"][i], ref["rec"]), (d, C, noise, i)
        assert abs(out["log_prob"][i] - ref["logp"]) < logp_tolerance(ref["branch_p"])
        assert out["discarded"][i] < 1e-9
    assert excluded <= 2


def test_ad_records_equal_ttn_oracle_d5():
    d, C, chi, ga = 5, 1, 64, 0.05
    circ = build_circuit(d, C)
    c = P.Circuit(d, C, layout="optimized")
    lay = list(c.layout())
    n, seed = 6, W.BASE_SEED + 41
    out = P.run_trajectories(c, n, noise="ad", gamma=ga, chi=chi, precision="mixed", seed=seed)
    compared = 0
    for i in range(n):
        ref = TT.run_trajectory(circ, AD, 0.0, ga, seed, i, chi, leaf_of_qubit=lay)
        if ref["discarded"] > 0 or ref["margin"] < TIE or out["near_ties"][i] > 0:
            continue
        compared += 1
        assert np.array_equal(out["records"][i], ref["rec"]), i
        assert abs(out["log_prob"][i] - ref["logp"]) < logp_tolerance(ref["branch_p"])
    assert compared >= 4

"""Seeded synthetic workloads shared by the tests, smoke() and bench.py.

Holds only input generation (configuration constants, seeds, trajectory
ranges, per-trajectory noise strengths, qubit-to-leaf layouts for parity
cases); none of the simulation's arithmetic.  The paper runs no dataset: its
workloads are synthetic circuits (Sec. III), restated here.
"""
import numpy as np

BASE_SEED = 2511057190

# d=3 hexagonal color code, 3 rounds, SRX theta = 0.05 rad, chi = 16, complex128
M1 = dict(name="d3_C3_srx_chi16_fp64", distance=3, rounds=3, noise="srx", theta=0.05,
          gamma=0.0, chi=16, precision="fp64", shots=1000, seed=BASE_SEED + 0)
# d=5, 5 rounds, AD gamma sweep and its twirl, chi = 64, complex64
M2 = dict(name="d5_C5_ad_chi64_fp32", distance=5, rounds=5, noise="ad",
          gammas=[1e-3, 3e-3, 1e-2, 2e-2], chi=64, precision="fp32", shots=100000,
          seed=BASE_SEED + 1)
# d=7, 7 rounds, SRX theta sweep (8 points in [0.01, 0.15] rad), chi = 128,
# complex64 tensors with tcgen05 digit-product contractions and the FP64 centre (MIXED)
M3 = dict(name="d7_C7_srx_chi128", distance=7, rounds=7, noise="srx",
          thetas=list(np.linspace(0.01, 0.15, 8)), chi=128, precision="mixed",
          shots=100000, seed=BASE_SEED + 2)
# mixed batch: d ~ U{3,5,7}, chi ~ U{16,64,128}, SRX theta ~ U[0.01, 0.1] then AD
M4 = dict(name="mixed_4096", n=4096, distances=[3, 5, 7], chis=[16, 64, 128],
          theta_range=(0.01, 0.1), gamma_range=(1e-3, 1e-2), seed=BASE_SEED + 3)
# gradient workload
M5 = dict(name="grad_srx", distances=[5, 7], chis=[64, 128], shots=50000, dtheta=1e-3,
          theta0=0.027, seed=BASE_SEED + 4)


def mixed_batch(n=4096, seed=M4["seed"]):
    """Per-trajectory (d, chi, theta, gamma) of the mixed workload."""
    rng = np.random.default_rng(seed)
    d = rng.choice(M4["distances"], size=n)
    chi = rng.choice(M4["chis"], size=n)
    theta = rng.uniform(*M4["theta_range"], size=n)
    gamma = rng.uniform(*M4["gamma_range"], size=n)
    return d, chi, theta, gamma


def theta_sweep_per_traj(n, thetas):
    """Trajectory i of a batch runs at thetas[i % len(thetas)]."""
    t = np.asarray(thetas, dtype=np.float64)
    return t[np.arange(n) % t.size]


def random_layout(n_qubits, n_leaves, seed):
    """A seeded random injective qubit -> leaf map (a parity input)."""
    rng = np.random.default_rng(seed)
    return rng.permutation(n_leaves)[:n_qubits].astype(np.int32)

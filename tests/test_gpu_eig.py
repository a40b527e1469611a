"""The centre move's Gram eigensolver on its own (ttn_eig_gram) against
numpy's Hermitian eigensolver: singular values, orthonormality and
invariance of the kept subspace, on random, degenerate, rank-deficient,
split (block-diagonal) and near-degenerate spectra, and on every Gram matrix
of a d = 3 trajectory of the CPU tree tensor network (Sec. III.B: the centre
moves by the Schmidt decomposition of a bond matrix)."""
import math
import sys
import os

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2511_05719_gb300")

pytestmark = pytest.mark.gpu

ROUTES = ["jacobi", "tridiagonal", "tridiagonal_split", "mixed"]


def _unitary(rng, n):
    z = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _gram(rng, lam):
    U = _unitary(rng, len(lam))
    G = (U * lam) @ U.conj().T
    return 0.5 * (G + G.conj().T)


def _check(G, V, s, k, eps_keep, tol, kcap=None, route="tridiagonal"):
    """Kept subspace: orthonormal, invariant under G, its Rayleigh quotient's
    spectrum the top-k eigenvalues; singular values match numpy's.  The
    Jacobi route skips rotations against directions whose diagonal entry is
    below eps_keep^2 tr(G) / n (their coupling to a kept direction a is at
    most sqrt(a eps_keep^2 tr(G) / n)): its residual is held to eps_keep |G|
    beside the rounding bar."""
    n = G.shape[0]
    lam = np.linalg.eigvalsh(G)[::-1]
    s_ref = np.sqrt(np.maximum(lam, 0.0))
    gn = max(lam[0], 1e-300)
    assert np.max(np.abs(s ** 2 - s_ref ** 2)) <= tol * gn, (s[:8], s_ref[:8])
    want_k = max(1, int(np.sum(s_ref > eps_keep * s_ref[0])))
    if kcap is not None:
        want_k = min(want_k, kcap)
    # ranks agree except where a singular value sits on the threshold
    if int(k) != want_k:
        edge = eps_keep * s_ref[0]
        lo, hi = sorted((int(k), want_k))
        assert np.all(np.abs(s_ref[lo:hi] - edge) <= 1e-6 * s_ref[0]), (int(k), want_k)
    k = int(k)
    Vk = V[:, :k]
    if k < V.shape[1]:
        assert np.max(np.abs(V[:, k:])) == 0.0
    orth = np.linalg.norm(Vk.conj().T @ Vk - np.eye(k))
    assert orth <= tol * math.sqrt(k), orth
    H = Vk.conj().T @ G @ Vk
    resid = np.linalg.norm(G @ Vk - Vk @ H)
    rtol = tol + (eps_keep if route == "jacobi" else 0.0)
    assert resid <= rtol * gn * math.sqrt(k), (route, resid)
    ev = np.sort(np.linalg.eigvalsh(0.5 * (H + H.conj().T)))[::-1]
    assert np.max(np.abs(ev - lam[:k])) <= tol * gn * math.sqrt(k)
    # columns are eigenvectors up to rotations within groups of close
    # eigenvalues (at most 1e-3 of the largest apart): the diagonal of H
    # descends up to that width
    d = np.real(np.diag(H))
    assert np.all(np.diff(d) <= 2e-3 * gn), d[:8]


def _run(Gs, route, kcap=None, eps_keep=1e-7):
    G = torch.as_tensor(np.stack(Gs), dtype=torch.complex128, device="cuda")
    V, s, k = P.eig_gram(G, kcap=kcap, route=route, eps_keep=eps_keep)
    torch.cuda.synchronize()
    return V.cpu().numpy(), s.cpu().numpy(), k.cpu().numpy()


def _tol(route, fp64=1e-10):
    """The split and MIXED routes round V_k to complex64 (2^-24 per entry)."""
    return 1e-6 if route in ("tridiagonal_split", "mixed") else fp64


def _routes_for(n):
    return [r for r in ROUTES if r != "jacobi" or n * n <= 8192]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 90, 129, 300, 512])
def test_random_spectrum(n):
    rng = np.random.default_rng(100 + n)
    Gs = [_gram(rng, rng.uniform(0.0, 1.0, n) ** 3) for _ in range(3)]
    for route in _routes_for(n):
        V, s, k = _run(Gs, route)
        for b in range(3):
            _check(Gs[b], V[b], s[b], k[b], 1e-7, _tol(route, 1e-11), route=route)


@pytest.mark.parametrize("n", [4, 16, 48, 96, 256])
def test_degenerate_and_rank_deficient(n):
    """Stabiliser-like flat spectra: a few exactly repeated eigenvalues and a
    null space (a pure stabiliser state's bond has 2^r equal Schmidt values)."""
    rng = np.random.default_rng(7 + n)
    specs = []
    r = max(1, n // 4)
    specs.append(np.r_[np.full(r, 1.0 / r), np.zeros(n - r)])
    specs.append(np.r_[np.full(n // 2, 0.5), np.full(n - n // 2, 0.25)])
    lam = np.zeros(n)
    lam[: n // 2] = np.repeat([0.4, 0.2, 0.1, 0.05], max(1, n // 8))[: n // 2]
    specs.append(lam)
    Gs = [_gram(rng, sp) for sp in specs]
    for route in _routes_for(n):
        V, s, k = _run(Gs, route)
        for b in range(len(Gs)):
            _check(Gs[b], V[b], s[b], k[b], 1e-7, _tol(route), route=route)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 64, 200])
def test_rank_one_and_two(n):
    """Bonds right after a measurement: one or two nonzero Schmidt values and
    an (n-1)- or (n-2)-fold zero eigenvalue."""
    rng = np.random.default_rng(300 + n)
    Gs = [_gram(rng, np.r_[0.7, np.zeros(n - 1)])]
    if n >= 2:
        Gs.append(_gram(rng, np.r_[0.6, 0.4, np.zeros(n - 2)]))
        Gs.append(_gram(rng, np.r_[0.5, 0.5, np.zeros(n - 2)]))
    for route in _routes_for(n):
        V, s, k = _run(Gs, route)
        for b in range(len(Gs)):
            _check(Gs[b], V[b], s[b], k[b], 1e-7, _tol(route), route=route)


@pytest.mark.parametrize("n", [6, 32, 100])
def test_block_diagonal_and_near_degenerate(n):
    """Direct sums (the tridiagonal form splits into blocks with equal
    eigenvalues in different blocks) and pairs split by 1e-14 relative."""
    rng = np.random.default_rng(31 + n)
    h = n // 2
    a = _gram(rng, np.linspace(1.0, 0.1, h))
    G1 = np.zeros((n, n), complex)
    G1[:h, :h] = a
    G1[h:, h:] = a[: n - h, : n - h] if n - h == h else _gram(rng, np.linspace(1.0, 0.1, n - h))
    lam = np.repeat(np.linspace(1.0, 0.2, n // 2), 2)[:n] * (1 + 1e-14 * np.tile([0, 1], n)[:n])
    G2 = _gram(rng, lam)
    G3 = np.diag(np.repeat([0.5, 0.25], [n // 2, n - n // 2])).astype(complex)
    for route in _routes_for(n):
        V, s, k = _run([G1, G2, G3], route)
        for b, G in enumerate([G1, G2, G3]):
            _check(G, V[b], s[b], k[b], 1e-7, _tol(route), route=route)


def test_kcap_and_threshold():
    rng = np.random.default_rng(5)
    n = 40
    lam = np.r_[np.geomspace(1.0, 1e-20, n // 2), np.zeros(n - n // 2)]
    G = _gram(rng, lam)
    for route in _routes_for(n):
        V, s, k = _run([G], route, kcap=8)
        assert int(k[0]) == 8
        _check(G, V[0], s[0], k[0], 1e-7, _tol(route), kcap=8, route=route)


def test_trajectory_gram_matrices():
    """Every bond Gram matrix of a d = 3 SRX trajectory of the CPU tree
    tensor network, through the tridiagonal routes and the MIXED runs'
    combination."""
    from oracle import ttn as OT
    from oracle.layout import optimized_layout
    from oracle.channels import SRX
    from oracle.circuit import build_circuit
    import workloads as W

    circ = build_circuit(3, 2)
    mats = []
    orig = OT.TTN.move

    def move(self, v, w, cap=None):
        leg = self._leg_of(v, w)
        Tm = np.moveaxis(self.T[v], leg, 2)
        M = Tm.reshape(-1, Tm.shape[2])
        if M.shape[1] >= 2:
            mats.append(M.conj().T @ M)
        return orig(self, v, w, cap)

    OT.TTN.move = move
    try:
        for traj in (1, 4):
            OT.run_trajectory(circ, SRX, 0.07, 0.0, W.BASE_SEED, traj, 64, leaf_of_qubit=optimized_layout(circ))
    finally:
        OT.TTN.move = orig
    by_n = {}
    for G in mats:
        by_n.setdefault(G.shape[0], []).append(G)
    for n, Gs in sorted(by_n.items()):
        for route in ("tridiagonal", "tridiagonal_split", "mixed"):
            V, s, k = _run(Gs, route)
            for b, G in enumerate(Gs):
                _check(G, V[b], s[b], k[b], 1e-7, _tol(route), route=route)

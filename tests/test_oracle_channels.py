"""Pins of the error channels (Eqs. 1-3) and their Pauli twirls (Sec. IV.C)."""
import numpy as np
import pytest

from oracle import channels as ch


def rand_rho(rng):
    A = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    r = A @ A.conj().T
    return r / np.trace(r)


@pytest.mark.parametrize("theta,gamma", [(0.0, 0.0), (0.05, 0.02), (0.3, 0.4), (1.0, 0.9)])
def test_trace_preserving_and_expansion(theta, gamma):
    rng = np.random.default_rng(3)
    for model in (ch.SRX, ch.AD, ch.SRX_AD):
        K = ch.kraus_of(model, theta, gamma)
        assert np.allclose(sum(k.conj().T @ k for k in K), np.eye(2), atol=1e-14)
        eta = ch.pauli_chi_matrix(K)
        assert np.allclose(eta, eta.conj().T, atol=1e-15)
        for _ in range(5):
            rho = rand_rho(rng)
            direct = ch.apply_channel(K, rho)
            expanded = sum(eta[i, j] * ch.PAULIS[i] @ rho @ ch.PAULIS[j]
                           for i in range(4) for j in range(4))
            assert np.allclose(direct, expanded, atol=1e-14)


@pytest.mark.parametrize("theta", [0.0, 0.01, 0.05, 0.15, 1.2])
def test_srx_twirl_closed_form(theta):
    eta = ch.pauli_chi_matrix(ch.kraus_of(ch.SRX, theta, 0.0))
    assert np.allclose(np.real(np.diag(eta)), ch.pta_probs(ch.SRX_PTA, theta, 0.0), atol=1e-15)
    # SRX is coherent: the off-diagonal I-X term is i sin cos, dropped by the PTA
    assert abs(eta[0, 1]) == pytest.approx(abs(np.sin(theta) * np.cos(theta)), abs=1e-15)


@pytest.mark.parametrize("gamma", [0.0, 1e-3, 1e-2, 0.2, 0.9])
def test_ad_twirl_closed_form(gamma):
    eta = ch.pauli_chi_matrix(ch.kraus_of(ch.AD, 0.0, gamma))
    p = ch.pta_probs(ch.AD_PTA, 0.0, gamma)
    assert np.allclose(np.real(np.diag(eta)), p, atol=1e-15)
    assert p.sum() == pytest.approx(1.0, abs=1e-15)


def test_identity_at_zero_strength():
    assert np.allclose(ch.srx_unitary(0.0), np.eye(2))
    K0, K1 = ch.ad_kraus(0.0)
    assert np.allclose(K0, np.eye(2)) and np.allclose(K1, 0)
    # theta convention: exp(-i theta X), so theta = pi/2 is a full bit flip
    U = ch.srx_unitary(np.pi / 2)
    assert abs(U[1, 0]) == pytest.approx(1.0)


def test_depolarizing_closed_form():
    """DEPOL's Pauli mixture (1 - g, g/3, g/3, g/3) is the depolarizing map
    rho -> (1 - 4g/3) rho + (4g/3) Tr(rho) I / 2, and trace preserving."""
    from oracle.channels import DEPOL, pta_probs, PAULIS, apply_channel
    rng = np.random.default_rng(3)
    for g in (0.0, 0.01, 0.2, 0.75):
        p = pta_probs(DEPOL, 0.0, g)
        assert np.isclose(p.sum(), 1.0)
        kraus = [np.sqrt(pi) * P for pi, P in zip(p, PAULIS)]
        A = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        rho = A @ A.conj().T
        rho /= np.trace(rho)
        want = (1 - 4 * g / 3) * rho + (4 * g / 3) * np.trace(rho) * np.eye(2) / 2
        assert np.allclose(apply_channel(kraus, rho), want, atol=1e-14)

"""Single-qubit error channels and their Pauli-twirled approximations.

Oracle (test infrastructure only).

  SRX  (Eq. 1):   E[rho] = exp(-i theta X) rho exp(+i theta X), theta in [0, pi)
  AD   (Eqs. 2-3): Kraus K0 = [[1,0],[0,sqrt(1-gamma)]], K1 = [[0,sqrt(gamma)],[0,0]]
  PTA  (Sec. IV.C): write the channel as sum_ij eta_ij P_i rho P_j in the Pauli
       basis and keep only the diagonal eta_ii.

theta is the angle of Eq. 1 itself (exp(-i theta X), not R_X(theta) =
exp(-i theta X / 2)); the paper reports it in units of pi.

`pauli_chi_matrix` computes eta from the Kraus operators by the definition
(c_ki = Tr(P_i K_k)/2, eta_ij = sum_k c_ki conj(c_kj)); `pta_probs` gives the
closed forms
    SRX: p = (cos^2 t, sin^2 t, 0, 0)
    AD : p = ((1+sqrt(1-g))^2/4, g/4, g/4, (1-sqrt(1-g))^2/4)
Both are pinned in tests/test_oracle_channels.py: the Pauli expansion
reproduces the channel on random density matrices, the diagonal matches the
closed forms, the channels are trace preserving, theta = 0 / gamma = 0 is the
identity.

  DEPOL (Sec. III.A, the Pauli benchmark model, single-qubit form at every
       location): p = (1 - g, g/3, g/3, g/3).

Noise-model numbering (shared vocabulary of the C-ABI):
NONE=0, SRX=1, AD=2, SRX_PTA=3, AD_PTA=4, SRX_AD=5 (SRX then AD at each
location), DEPOL=6.
"""
import numpy as np

NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD, DEPOL = 0, 1, 2, 3, 4, 5, 6
PAULI_MODELS = (SRX_PTA, AD_PTA, DEPOL)  # channels that are a Pauli mixture

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0)
PAULIS = (I2, X, Y, Z)


def srx_unitary(theta: float) -> np.ndarray:
    """exp(-i theta X) = cos(theta) I - i sin(theta) X (X^2 = I)."""
    return np.cos(theta) * I2 - 1j * np.sin(theta) * X


def ad_kraus(gamma: float):
    K0 = np.array([[1.0, 0.0], [0.0, np.sqrt(1.0 - gamma)]], dtype=np.complex128)
    K1 = np.array([[0.0, np.sqrt(gamma)], [0.0, 0.0]], dtype=np.complex128)
    return [K0, K1]


def kraus_of(model: int, theta: float, gamma: float):
    """Kraus operators of the (non-twirled) channel at one location."""
    if model == SRX:
        return [srx_unitary(theta)]
    if model == AD:
        return ad_kraus(gamma)
    if model == SRX_AD:
        U = srx_unitary(theta)
        return [K @ U for K in ad_kraus(gamma)]
    if model == NONE:
        return [I2.copy()]
    raise ValueError("no Kraus form for a twirled model")


def apply_channel(kraus, rho):
    return sum(K @ rho @ K.conj().T for K in kraus)


def pauli_chi_matrix(kraus) -> np.ndarray:
    """eta_ij with E[rho] = sum_ij eta_ij P_i rho P_j (P = I, X, Y, Z)."""
    c = np.array([[np.trace(P @ K) / 2.0 for P in PAULIS] for K in kraus])
    return c.T @ c.conj()


def pta_probs(model: int, theta: float, gamma: float) -> np.ndarray:
    """Closed-form diagonal of eta for the twirled models, order (I, X, Y, Z)."""
    if model == SRX_PTA:
        c, s = np.cos(theta), np.sin(theta)
        return np.array([c * c, s * s, 0.0, 0.0])
    if model == AD_PTA:
        r = np.sqrt(1.0 - gamma)
        return np.array([(1 + r) ** 2 / 4, gamma / 4, gamma / 4, (1 - r) ** 2 / 4])
    if model == DEPOL:
        return np.array([1.0 - gamma, gamma / 3, gamma / 3, gamma / 3])
    raise ValueError("not a Pauli channel")

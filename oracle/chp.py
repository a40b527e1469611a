"""O3: stabilizer-tableau trajectories for Pauli-twirled noise.

Oracle (test infrastructure only).  With Pauli noise (the Pauli-twirled
channels of Sec. IV.C, SRX_PTA and AD_PTA, and depolarizing noise, DEPOL)
the extraction circuit is Clifford
plus sampled Paulis, so every trajectory stays a stabilizer state and is
simulated exactly at any code distance.  This is the repository's own
version of the paper's comparison with a Clifford simulator (Sec. IV.C,
Fig. 5); the tableau algorithm is Aaronson and Gottesman's (Phys. Rev. A 70,
052328 (2004), the CHP simulator).

State: 2n generators (destabilizers 0..n-1, stabilizers n..2n-1), each a
Pauli string with bits x, z (Python integers, bit q = qubit q) and a sign
bit r.  Gates: H swaps x_q and z_q (sign flips where both are set); CNOT
c -> t updates x_t ^= x_c, z_c ^= z_t with the sign rule of the paper;
Pauli X_q / Z_q / Y_q flip the sign of the generators that anticommute with
them.  Z measurement of q: if a stabilizer has x_q = 1 the outcome is
random -- every other generator with x_q = 1 is multiplied by it (the
"rowsum" with its phase bookkeeping), it moves to the destabilizers and Z_q
with sign = outcome takes its place; otherwise the outcome is determined by
the product of the stabilizers the destabilizers with x_q = 1 pair with.

Trajectory semantics and draws are those of the state-vector oracle
(oracle/statevector.py): Philox4x32-10 uniforms per event; a measurement
gives 1 iff u >= P(0), which for a random outcome (P(0) = 1/2) is u >= 0.5;
a Pauli location draws I, X, Y, Z by the inverse CDF of pta_probs; reset =
X if the qubit's last recorded outcome was 1, then H for an X preparation.

Pinned (tests/test_oracle_chp.py): identical records and log-probabilities
to the state-vector oracle on the same draws at d = 3 for both twirled
models (the two share no code but the circuit and the draws); noise off, Z
syndromes vanish and X syndromes repeat at d = 3, 5, 7; closed-form single-
and two-qubit cases (Bell pair correlations, GHZ parities).
"""
import math

import numpy as np

from . import philox
from .channels import SRX_PTA, AD_PTA, DEPOL, NONE, PAULI_MODELS, pta_probs
from .circuit import PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X, NOISE


class Tableau:
    def __init__(self, n):
        self.n = n
        self.x = [0] * (2 * n)
        self.z = [0] * (2 * n)
        self.r = [0] * (2 * n)
        for i in range(n):
            self.x[i] = 1 << i          # destabilizer X_i
            self.z[n + i] = 1 << i      # stabilizer Z_i  (|0...0>)

    # ---- Clifford gates
    def h(self, q):
        m = 1 << q
        for i in range(2 * self.n):
            xi, zi = self.x[i] & m, self.z[i] & m
            if xi and zi:
                self.r[i] ^= 1
            if bool(xi) != bool(zi):
                self.x[i] ^= m
                self.z[i] ^= m

    def cnot(self, c, t):
        mc, mt = 1 << c, 1 << t
        for i in range(2 * self.n):
            xc = 1 if self.x[i] & mc else 0
            zt = 1 if self.z[i] & mt else 0
            xt = 1 if self.x[i] & mt else 0
            zc = 1 if self.z[i] & mc else 0
            if xc and zt and (xt ^ zc ^ 1):
                self.r[i] ^= 1
            if xc:
                self.x[i] ^= mt
            if zt:
                self.z[i] ^= mc

    def pauli(self, q, k):
        """k = 1 X, 2 Y, 3 Z: flips the sign of anticommuting generators."""
        m = 1 << q
        for i in range(2 * self.n):
            xb, zb = self.x[i] & m, self.z[i] & m
            if (k == 1 and zb) or (k == 3 and xb) or (k == 2 and (bool(xb) != bool(zb))):
                self.r[i] ^= 1

    # ---- measurement
    @staticmethod
    def _g_sum(x1, z1, x2, z2):
        """sum over qubits of the exponent of i in P1 * P2 (Aaronson-Gottesman g)."""
        y1 = x1 & z1
        xo = x1 & ~z1
        zo = z1 & ~x1
        return ((y1 & z2 & ~x2).bit_count() - (y1 & x2 & ~z2).bit_count()
                + (xo & z2 & x2).bit_count() - (xo & z2 & ~x2).bit_count()
                + (zo & x2 & ~z2).bit_count() - (zo & x2 & z2).bit_count())

    def _rowsum(self, h, i, xs=None):
        """generator h <- generator i * generator h (h = -1: the scratch row xs)."""
        if h < 0:
            xh, zh, rh = xs
        else:
            xh, zh, rh = self.x[h], self.z[h], self.r[h]
        e = (2 * rh + 2 * self.r[i] + self._g_sum(self.x[i], self.z[i], xh, zh)) % 4
        assert e in (0, 2)
        out = (xh ^ self.x[i], zh ^ self.z[i], e // 2)
        if h < 0:
            return out
        self.x[h], self.z[h], self.r[h] = out
        return None

    def measure_z(self, q, u):
        """Returns (outcome, probability of that outcome, margin |u - P(0)|
        or None when deterministic)."""
        n, m = self.n, 1 << q
        p = next((i for i in range(n, 2 * n) if self.x[i] & m), None)
        if p is not None:
            out = 1 if u >= 0.5 else 0
            for i in range(2 * n):
                if i != p and (self.x[i] & m):
                    self._rowsum(i, p)
            self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p], self.z[p], self.r[p]
            self.x[p], self.z[p], self.r[p] = 0, m, out
            return out, 0.5, abs(u - 0.5)
        xs = (0, 0, 0)
        for i in range(n):
            if self.x[i] & m:
                xs = self._rowsum(-1, i + n, xs)
        return xs[2], 1.0, None


def run_trajectory(circ, model, theta, gamma, seed, traj):
    """One trajectory of a Pauli-noise model (NONE, SRX_PTA, AD_PTA, DEPOL).
    Returns dict(rec, logp, margin, branch_p) as the state-vector oracle."""
    if model != NONE and model not in PAULI_MODELS:
        raise ValueError("the tableau oracle runs Pauli noise only (NONE, SRX_PTA, AD_PTA, DEPOL)")
    N = circ.n_qubits
    tb = Tableau(N)
    last = np.zeros(N, dtype=np.int64)
    rec = np.zeros(circ.n_record_bits, dtype=np.uint8)
    logp, margin, branch_p = 0.0, math.inf, []
    events = [op[3] for op in circ.ops if op[3] >= 0]
    us = dict(zip(events, philox.uniforms(seed, [traj], events)[0])) if events else {}
    probs = pta_probs(model, theta, gamma) if model != NONE else None
    cum = np.cumsum(probs) if probs is not None else None
    for (kind, a, b, e, r, layer) in circ.ops:
        if kind in (PREP_Z, PREP_X):
            if last[a]:
                tb.pauli(a, 1)
                last[a] = 0
            if kind == PREP_X:
                tb.h(a)
        elif kind == CNOT:
            tb.cnot(a, b)
        elif kind in (MEAS_Z, MEAS_X):
            if kind == MEAS_X:
                tb.h(a)
            out, pm, mg = tb.measure_z(a, us[e])
            if mg is not None:
                margin = min(margin, mg)
            else:
                # deterministic: the draw u is compared with P(0) in {0, 1}
                margin = min(margin, abs(us[e] - (1.0 - out)))
            logp += math.log(pm)
            branch_p.append(pm)
            rec[r] = out
            last[a] = out
        elif kind == NOISE and probs is not None:
            u = us[e]
            k = 3
            for i in range(3):
                if u < cum[i]:
                    k = i
                    break
            if k > 0:
                tb.pauli(a, k)
            logp += math.log(probs[k])
            branch_p.append(float(probs[k]))
            margin = min(margin, float(min(abs(u - c) for c in cum[:3])))
    return dict(rec=rec, logp=logp, margin=margin, branch_p=branch_p)

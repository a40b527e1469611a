"""O4: plain binary Tree Tensor Network trajectories (numpy, complex128).

Oracle (test infrastructure only).  Follows Sec. III.B ("Emulation of quantum
circuits with Tree Tensor Networks"), Fig. 6 and App. B: a complete binary
tree whose leaves are the qubits (unused leaves allowed), bond dimension
capped at chi, two-qubit gates whose cost grows with the tree distance of
their leaves, truncation that discards the smallest Schmidt coefficients.
The trajectory semantics (draws, outcome rules, Kraus unravelling) are those
of the state-vector oracle.

Representation.  L = 2^D leaves, heap numbering: internal node v in 1..L-1 has
children 2v, 2v+1 and parent v // 2; leaf j sits at position L + j.  Node v
holds T_v[l, r, u] (l, r: bonds to its children, u: bond to its parent; the
root keeps u = 1 instead of being absorbed into a child -- an equivalent
form).  A leaf bond has dimension 2 when the leaf holds a qubit, else 1.
One node (the isometry centre) is general, every other tensor is an isometry
towards the centre.

Primitive: move(v -> w) across one bond: SVD of T_v with that bond as the
column index, keep the singular values above eps * s_max (and at most `cap`),
T_v <- U, the neighbour absorbs S V^dag; with a cap it truncates, records the
discarded weight sum_{i>=k} s_i^2 / sum s^2, and renormalises.

Two-qubit gate on leaves a, b (Sec. III.B; the paper delegates this step to
its library, so the procedure is this project's): move the centre to
c = LCA(a, b); write G = sum_k A_k (x) B_k (operator-Schmidt form, rank 2
for CNOT); apply A_k at a's node, B_k at b's node, and carry the index k
through every tensor on the path (the path bonds grow by the factor K);
restore the isometries with exact moves from each leaf node up to c; then
truncate the path bonds to chi by capped moves from c down to b's node, move
back to c, and from c down to a's node.  If a and b share a node the 4x4
gate is applied there directly.

Pinned (tests/test_oracle_ttn.py): with chi >= chi_exact the TTN amplitudes
equal the state-vector oracle's to 1e-12 and the records are identical for
the same draws; chi = 1 keeps a product state; the discarded weight is
zero when chi is large enough.
"""
import math
import time

import numpy as np

from . import philox
from .channels import (NONE, SRX, AD, SRX_PTA, AD_PTA, SRX_AD, PAULI_MODELS,
                       srx_unitary, pta_probs, X, Y, Z, H)
from .circuit import PREP_Z, PREP_X, CNOT, MEAS_Z, MEAS_X, NOISE

P0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
P1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)
CNOT_FACTORS = ([P0, P1], [np.eye(2, dtype=np.complex128), X])


def tree_depth(n_qubits):
    D = 1
    while (1 << D) < n_qubits:
        D += 1
    return D


def default_layout(n_qubits):
    return list(range(n_qubits))


class TTN:
    def __init__(self, n_qubits, leaf_of_qubit, chi, eps=1e-13):
        self.N = n_qubits
        self.D = tree_depth(n_qubits)
        self.L = 1 << self.D
        self.leaf_of_qubit = list(leaf_of_qubit)
        self.chi = chi
        self.eps = eps
        occupied = [False] * self.L
        for q in range(n_qubits):
            occupied[self.leaf_of_qubit[q]] = True
        self.T = [None] * self.L
        for v in range(1, self.L):
            dl = self._leafdim(2 * v, occupied)
            dr = self._leafdim(2 * v + 1, occupied)
            t = np.zeros((dl, dr, 1), dtype=np.complex128)
            t[0, 0, 0] = 1.0
            self.T[v] = t
        self.center = 1
        self.discarded = 0.0

    def _leafdim(self, pos, occupied):
        if pos >= self.L:
            return 2 if occupied[pos - self.L] else 1
        return 1

    # ---------------- tree navigation
    def pos(self, q):
        return self.L + self.leaf_of_qubit[q]

    def path(self, v, w):
        """Node sequence from v to w (both internal nodes)."""
        up_v, up_w = [v], [w]
        a, b = v, w
        while a != b:
            if a > b:
                a //= 2
                up_v.append(a)
            else:
                b //= 2
                up_w.append(b)
        return up_v + up_w[-2::-1]

    # ---------------- primitive move
    def _leg_of(self, v, w):
        """Which leg of v points to neighbour w: 0 = l, 1 = r, 2 = u."""
        if w == 2 * v:
            return 0
        if w == 2 * v + 1:
            return 1
        return 2

    def move(self, v, w, cap=None):
        leg = self._leg_of(v, w)
        T = self.T[v]
        Tm = np.moveaxis(T, leg, 2)             # bond to w last
        sh = Tm.shape
        M = Tm.reshape(sh[0] * sh[1], sh[2])
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
        if s.size == 0 or s[0] == 0.0:
            k = 1
        else:
            k = int(np.sum(s > self.eps * s[0]))
            k = max(k, 1)
        if cap is not None and k > cap:
            tot = float(np.sum(s ** 2))
            disc = float(np.sum(s[cap:] ** 2)) / tot
            self.discarded += disc
            k = cap
            scale = 1.0 / math.sqrt(1.0 - disc) if disc < 1.0 else 1.0
        else:
            scale = 1.0
        U = U[:, :k]
        R = (s[:k, None] * Vh[:k, :]) * scale    # k x dim(bond)
        self.T[v] = np.moveaxis(U.reshape(sh[0], sh[1], k), 2, leg)
        wleg = self._leg_of(w, v)
        Tw = np.moveaxis(self.T[w], wleg, 0)
        Tw = np.tensordot(R, Tw, axes=([1], [0]))
        self.T[w] = np.moveaxis(Tw, 0, wleg)
        self.center = w

    def move_center(self, target):
        p = self.path(self.center, target)
        for a, b in zip(p[:-1], p[1:]):
            self.move(a, b)

    # ---------------- gates
    def apply1(self, q, U):
        pos = self.pos(q)
        v, leg = pos // 2, pos % 2
        T = np.moveaxis(self.T[v], leg, 0)
        T = np.tensordot(U, T, axes=([1], [0]))
        self.T[v] = np.moveaxis(T, 0, leg)

    def prob1(self, q):
        """P(q = 1); the centre must be at q's node."""
        pos = self.pos(q)
        v, leg = pos // 2, pos % 2
        assert self.center == v
        T = np.moveaxis(self.T[v], leg, 0)
        n1 = float(np.sum(np.abs(T[1]) ** 2))
        n = float(np.sum(np.abs(T) ** 2))
        return n1 / n

    def apply_at_center(self, q, K, scale):
        self.apply1(q, K * scale)

    def gate2(self, a, b, A, B):
        """sum_k A[k] (x) B[k] on qubits a, b."""
        pa, pb = self.pos(a), self.pos(b)
        va, vb = pa // 2, pb // 2
        K = len(A)
        if va == vb:
            v = va
            self.move_center(v)
            G = sum(np.kron(A[k], B[k]) for k in range(K))   # (a' b') x (a b)
            G = G.reshape(2, 2, 2, 2)
            T = self.T[v]
            if pa % 2 == 0:    # a on leg l, b on leg r
                T = np.einsum("xyab,abu->xyu", G, T)
            else:
                T = np.einsum("yxba,abu->xyu", G, T)
            self.T[v] = T
            return
        c = va
        x, y = va, vb
        while x != y:
            if x > y:
                x //= 2
            else:
                y //= 2
        c = x
        self.move_center(c)
        side_a = self._branch(va, c)
        side_b = self._branch(vb, c)
        # apply factors at the leaf nodes: new up bond index = k * d + u
        for (pos, nodes, F) in ((pa, side_a, A), (pb, side_b, B)):
            v0 = nodes[0]
            leg = pos % 2
            T = np.moveaxis(self.T[v0], leg, 0)               # (x, y, u)
            parts = [np.tensordot(F[k], T, axes=([1], [0])) for k in range(K)]
            Tn = np.concatenate(parts, axis=2)                 # u-index k*du+u
            self.T[v0] = np.moveaxis(Tn, 0, leg)
            # thread k through the remaining path nodes (block diagonal)
            prev = v0
            for v in nodes[1:] + [c]:
                leg_c = self._leg_of(v, prev)
                T = np.moveaxis(self.T[v], leg_c, 0)           # (x_child, y, u)
                dx = T.shape[0]
                if v == c:
                    continue
                out = np.zeros((K * dx,) + T.shape[1:2] + (K * T.shape[2],),
                               dtype=np.complex128)
                du = T.shape[2]
                for k in range(K):
                    out[k * dx:(k + 1) * dx, :, k * du:(k + 1) * du] = T
                self.T[v] = np.moveaxis(out, 0, leg_c)
                prev = v
        # the LCA: both child legs carry k, diagonal
        T = self.T[c]
        la = self._leg_of(c, side_a[-1])
        lb = self._leg_of(c, side_b[-1])
        Tc = np.moveaxis(T, (la, lb), (0, 1))                  # (xa, xb, u)
        dxa, dxb, du = Tc.shape
        out = np.zeros((K * dxa, K * dxb, du), dtype=np.complex128)
        for k in range(K):
            out[k * dxa:(k + 1) * dxa, k * dxb:(k + 1) * dxb, :] = Tc
        self.T[c] = np.moveaxis(out, (0, 1), (la, lb))
        # restore isometries from the leaf nodes up to c (exact moves)
        for nodes in (side_a, side_b):
            for v, w in zip(nodes, nodes[1:] + [c]):
                self.center = v
                self.move(v, w)
        self.center = c
        # truncate: c -> b's node, back to c, c -> a's node
        seq = [c] + side_b[::-1]
        for v, w in zip(seq[:-1], seq[1:]):
            self.move(v, w, cap=self.chi)
        self.move_center(c)
        seq = [c] + side_a[::-1]
        for v, w in zip(seq[:-1], seq[1:]):
            self.move(v, w, cap=self.chi)

    def _branch(self, v0, c):
        nodes = [v0]
        v = v0
        while v // 2 != c:
            v //= 2
            nodes.append(v)
        return nodes

    # ---------------- state extraction
    def amplitudes(self):
        """Little-endian amplitude vector (qubit q = bit q of the index)."""
        def sub(v):
            T = self.T[v]
            if 2 * v >= self.L:
                return T                                   # (leaf, leaf, u)
            A, B = sub(2 * v), sub(2 * v + 1)
            R = np.tensordot(A, T, axes=([A.ndim - 1], [0]))          # (.a, r, u)
            R = np.tensordot(R, B, axes=([R.ndim - 2], [B.ndim - 1]))  # (.a, u, .b)
            return np.moveaxis(R, A.ndim - 1, -1)                     # (.a, .b, u)
        full = sub(1)[..., 0]
        occ = sorted(self.leaf_of_qubit)
        st = full.reshape((2,) * len(occ))
        rank = {j: i for i, j in enumerate(occ)}
        st = np.transpose(st, [rank[self.leaf_of_qubit[q]] for q in range(self.N)])
        return st.transpose(tuple(range(self.N - 1, -1, -1))).reshape(-1).copy()

    def max_bond(self):
        m = 1
        for v in range(1, self.L):
            m = max(m, max(self.T[v].shape))
        return m


def apply_noise_ttn(tt, q, model, theta, gamma, u):
    if model == NONE:
        return 0.0, None
    if model in (SRX, SRX_AD):
        tt.apply1(q, srx_unitary(theta))
        if model == SRX:
            return 0.0, None
    if model in (AD, SRX_AD):
        tt.move_center(tt.pos(q) // 2)
        P1v = tt.prob1(q)
        p1 = gamma * P1v
        if u < p1:
            K1 = np.array([[0, 1], [0, 0]], dtype=np.complex128)
            tt.apply1(q, K1 / math.sqrt(P1v))
            return math.log(p1), abs(u - p1)
        K0 = np.array([[1, 0], [0, math.sqrt(1 - gamma)]], dtype=np.complex128)
        tt.apply1(q, K0 / math.sqrt(1.0 - p1))
        return math.log1p(-p1), abs(u - p1)
    if model in PAULI_MODELS:
        p = pta_probs(model, theta, gamma)
        cum = np.cumsum(p)
        k = 3
        for i in range(3):
            if u < cum[i]:
                k = i
                break
        if k > 0:
            tt.apply1(q, (None, X, Y, Z)[k])
        return math.log(p[k]), float(min(abs(u - c) for c in cum[:3]))
    raise ValueError("unknown noise model")


def run_trajectory(circ, model, theta, gamma, seed, traj, chi, leaf_of_qubit=None,
                   snapshot_layers=(), eps=1e-13, max_ops=None, deadline=None, on_op=None):
    """One trajectory on the numpy TTN.  max_ops / deadline (a time.time()
    value) stop the run early, for bounded timing samples; `ops_done` in the
    result counts the ops run.  on_op(i), if given, is called after op i
    (a timing hook; it does not touch the state)."""
    N = circ.n_qubits
    if leaf_of_qubit is None:
        leaf_of_qubit = default_layout(N)
    tt = TTN(N, leaf_of_qubit, chi, eps)
    last = np.zeros(N, dtype=np.int64)
    rec = np.zeros(circ.n_record_bits, dtype=np.uint8)
    logp = 0.0
    margin = math.inf
    branch_p = []
    states = {}
    snap = set(snapshot_layers)
    events = [op[3] for op in circ.ops if op[3] >= 0]
    us = dict(zip(events, philox.uniforms(seed, [traj], events)[0])) if events else {}
    cur_layer = 0
    ops_done = len(circ.ops)
    for i, (kind, a, b, e, r, layer) in enumerate(circ.ops):
        if (max_ops is not None and i >= max_ops) or (deadline is not None and time.time() > deadline):
            ops_done = i
            break
        if layer != cur_layer:
            if cur_layer in snap:
                states[cur_layer] = tt.amplitudes()
            cur_layer = layer
        if kind in (PREP_Z, PREP_X):
            if last[a]:
                tt.apply1(a, X)
                last[a] = 0
            if kind == PREP_X:
                tt.apply1(a, H)
        elif kind == CNOT:
            tt.gate2(a, b, *CNOT_FACTORS)
        elif kind in (MEAS_Z, MEAS_X):
            if kind == MEAS_X:
                tt.apply1(a, H)
            tt.move_center(tt.pos(a) // 2)
            p1 = tt.prob1(a)
            p0 = 1.0 - p1
            u = us[e]
            m = 1 if u >= p0 else 0
            margin = min(margin, abs(u - p0))
            pm = p1 if m else p0
            tt.apply1(a, (P1 if m else P0) / math.sqrt(pm))
            logp += math.log(pm)
            branch_p.append(pm)
            rec[r] = m
            last[a] = m
        elif kind == NOISE:
            lp, dist = apply_noise_ttn(tt, a, model, theta, gamma, us[e])
            logp += lp
            if dist is not None:
                margin = min(margin, dist)
                branch_p.append(math.exp(lp))
        if on_op is not None:
            on_op(i)
    if cur_layer in snap:
        states[cur_layer] = tt.amplitudes()
    return dict(rec=rec, logp=logp, margin=margin, states=states, ttn=tt, branch_p=branch_p,
                discarded=tt.discarded, ops_done=ops_done)

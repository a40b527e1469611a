"""Concatenated minimum-weight perfect-matching decoder of the color code.

Oracle (test infrastructure only).  Follows App. A.2 ("Decoding"): for each
colour c, (1) MWPM on the restricted lattice of the checks whose colour is
not c; (2) the edges predicted by (1), together with the c-coloured checks,
define a second problem, also solved by MWPM; the lowest-weight of the three
candidate corrections is the output.  The paper defers the details to a
reference that is not available; the reading below is this project's.

Detectors (Z-memory experiment, data start in |0>^n, Sec. III):
    D[t][p] = mZ[t][p] xor mZ[t-1][p]          t = 0..C-1, mZ[-1] = 0
    D[C][p] = parity(data bits on face p) xor mZ[C-1][p]
Node id of (t, p) is t * P + p; the boundary has id (C + 1) * P.

Stage 1 (colour c): nodes (t, p) with colour(p) != c.  Space edge at layer t
for every data qubit q whose non-c faces are {f1, f2} (edge f1-f2) or {f1}
(edge f1-boundary); its qubit set Q(e) = all qubits with that same non-c face
set.  Time edges (t, p)-(t+1, p).  Unit weights.

Stage 2 (colour c): nodes (t, g) with colour(g) = c, plus the boundary.  Each
stage-1 space edge e in the matching at layer t contributes its default
qubit q1 = min Q(e) (flipping the c-face of q1); the residual c-syndrome is
D xor those flips.  Edges at layer t:
  * e matched in stage 1: weight-0 "choice" edges g(q1)-g(qj), qj in Q(e)
    (swap the default qubit; non-c syndrome unchanged);
  * e not matched: weight-2 "pair" edges g(qi)-g(qj) for qi < qj in Q(e)
    (flip both; non-c syndrome unchanged);
  * qubits with no non-c face: weight-1 edge g(q)-boundary;
  a qubit with no c-face maps to the boundary.  Time edges (t,g)-(t+1,g),
  weight 1.
Score(c) = stage-1 weight + stage-2 weight; the smallest score wins, ties to
the lowest c.  fail = parity(all data bits) xor parity(#corrected qubits):
Z-bar = Z^{x n} (App. A.1) is flipped by an odd number of X corrections.

Exactness / uniqueness: every matching weight is W = w * 2^40 + h(a, b),
h a 28-bit splitmix64 hash of the node pair, stage and colour, so the
optimum is unique with overwhelming probability and any exact MWPM solver
finds the same one.  Paths: the canonical shortest path from the smaller
node id to the larger walks, at each step, to the smallest-id neighbour that
stays on a shortest path (distances compared as (weight, hops)).

MWPM here is exact: the optimum splits over connected components of the
pairs cheaper than sending both defects to the boundary; each component is
solved by a subset dynamic programme (<= 14 defects) or by networkx's
weighted blossom with integer weights (a library routine as one step).

Pinned (tests/test_oracle_decoder.py): DP matching == brute-force enumeration
of perfect matchings; the component split equals the undecomposed DP and
the blossom; every code-capacity X error of weight <= (d-1)/2
decodes without a logical flip (d = 3, 5, 7); noise-free records decode to no
flip.  Parity against the paper's own decoder is unpinned (its definition is
not in the paper).
"""
import heapq
from collections import deque
from functools import lru_cache

import numpy as np

from .colorcode import color_code

MASK64 = (1 << 64) - 1
WUNIT = 1 << 40
MAX_DP_DEFECTS = 22


def pair_hash(a, b, stage, color):
    """28-bit hash of an unordered node pair (splitmix64 finaliser)."""
    if a > b:
        a, b = b, a
    x = (a * 0x9E3779B97F4A7C15 + b * 0xBF58476D1CE4E5B9
         + (stage * 3 + color + 1) * 0x94D049BB133111EB) & MASK64
    x ^= x >> 30
    x = (x * 0xBF58476D1CE4E5B9) & MASK64
    x ^= x >> 27
    x = (x * 0x94D049BB133111EB) & MASK64
    x ^= x >> 31
    return x >> 36


class DecoderGraphs:
    """Static stage-1 graphs and qubit sets for one (d, C)."""

    def __init__(self, d, rounds):
        code = color_code(d)
        self.code = code
        self.C = rounds
        self.P = code.n_plaq
        self.T = rounds + 1
        self.B = self.T * self.P
        P = self.P
        self.stage1 = []
        for c in range(3):
            # non-c face set of every qubit, and the qubit sets per face set
            qsets = {}
            for q in range(code.n):
                S = tuple(f for f in code.qubit_plaqs[q] if code.plaq_color[f] != c)
                qsets.setdefault(S, []).append(q)
            cface = []
            for q in range(code.n):
                g = [f for f in code.qubit_plaqs[q] if code.plaq_color[f] == c]
                cface.append(g[0] if g else -1)
            nodes = [t * P + p for t in range(self.T) for p in range(P)
                     if code.plaq_color[p] != c]
            adj = {v: set() for v in nodes}
            adj[self.B] = set()
            space = {}   # (t, S) -> sorted qubit list
            for S, qs in qsets.items():
                if len(S) == 0:
                    continue
                for t in range(self.T):
                    if len(S) == 2:
                        u, v = t * P + S[0], t * P + S[1]
                    else:
                        u, v = t * P + S[0], self.B
                    adj[u].add(v)
                    adj[v].add(u)
                    space[(t, S)] = sorted(qs)
            for t in range(self.T - 1):
                for p in range(P):
                    if code.plaq_color[p] != c:
                        u, v = t * P + p, (t + 1) * P + p
                        adj[u].add(v)
                        adj[v].add(u)
            adj = {v: sorted(ns) for v, ns in adj.items()}
            dist = {}
            for s in adj:
                dist[s] = bfs(adj, s)
            self.stage1.append(dict(adj=adj, dist=dist, qsets=qsets, cface=cface,
                                    nodes=nodes))


def bfs(adj, s):
    d = {s: 0}
    dq = deque([s])
    while dq:
        u = dq.popleft()
        for v in adj[u]:
            if v not in d:
                d[v] = d[u] + 1
                dq.append(v)
    return d


def edge_key(u, v):
    return (u, v) if u < v else (v, u)


def canonical_path_unit(adj, dist_to_target, src, dst):
    """Walk from src to dst on unit-weight edges, smallest-id next hop."""
    path = []
    u = src
    while u != dst:
        du = dist_to_target[u]
        nxt = None
        for v in adj[u]:
            if dist_to_target.get(v, None) == du - 1:
                nxt = v
                break
        path.append(edge_key(u, nxt))
        u = nxt
    return path


def mwpm_dp(defects, wpair, wbound):
    """Exact minimum-weight matching of `defects` (sorted ids); each defect is
    paired with another or with the boundary.  wpair(i, j), wbound(i) are
    perturbed integer weights or None when unreachable.  Returns list of
    (i, j) index pairs, j = -1 for the boundary, and the total weight.
    Subset dynamic programme (small instances)."""
    k = len(defects)
    if k > MAX_DP_DEFECTS:
        raise ValueError("too many defects for the DP oracle: %d" % k)
    INF = float("inf")
    W = [[wpair(i, j) if i != j else None for j in range(k)] for i in range(k)]
    Wb = [wbound(i) for i in range(k)]

    @lru_cache(maxsize=None)
    def f(mask):
        if mask == 0:
            return (0, ())
        i = (mask & -mask).bit_length() - 1
        rest = mask & ~(1 << i)
        best = (INF, ())
        if Wb[i] is not None:
            sub = f(rest)
            cand = Wb[i] + sub[0]
            if cand < best[0]:
                best = (cand, ((i, -1),) + sub[1])
        m = rest
        while m:
            j = (m & -m).bit_length() - 1
            m &= m - 1
            if W[i][j] is None:
                continue
            sub = f(rest & ~(1 << j))
            cand = W[i][j] + sub[0]
            if cand < best[0]:
                best = (cand, ((i, j),) + sub[1])
        return best

    tot, pairs = f((1 << k) - 1)
    f.cache_clear()
    if tot == INF:
        raise ValueError("no perfect matching")
    return list(pairs), tot


def mwpm_blossom(k, wpair, wbound):
    """Exact minimum-weight matching with boundary through networkx's
    weighted blossom on the graph of defects and boundary copies (integer
    weights, so the library's dual updates stay exact)."""
    import networkx as nx
    G = nx.Graph()
    maxw = 0
    edges = []
    for i in range(k):
        wb = wbound(i)
        if wb is not None:
            edges.append((("d", i), ("b", i), wb))
        for j in range(i + 1, k):
            w = wpair(i, j)
            if w is not None:
                edges.append((("d", i), ("d", j), w))
            edges.append((("b", i), ("b", j), 0))
    for (_, _, w) in edges:
        maxw = max(maxw, w)
    for (a, b, w) in edges:
        G.add_edge(a, b, weight=maxw + 1 - w)
    M = nx.max_weight_matching(G, maxcardinality=True)
    pairs, tot = [], 0
    for (a, b) in M:
        if a[0] == "d" and b[0] == "d":
            i, j = sorted((a[1], b[1]))
            pairs.append((i, j))
            tot += wpair(i, j)
        elif a[0] != b[0]:
            i = a[1] if a[0] == "d" else b[1]
            pairs.append((i, -1))
            tot += wbound(i)
    if sum(2 if j >= 0 else 1 for (_, j) in pairs) != k:
        raise ValueError("no perfect matching")
    return pairs, tot


def mwpm(defects, wpair, wbound):
    """Exact minimum-weight matching with boundary.  A pair with
    w(i, j) >= wb(i) + wb(j) is never better than sending both defects to the
    boundary, so the optimum splits over connected components of the other
    pairs; each component is solved exactly (DP when small, blossom
    otherwise)."""
    k = len(defects)
    useful = [[] for _ in range(k)]
    for i in range(k):
        for j in range(i + 1, k):
            w = wpair(i, j)
            if w is None:
                continue
            bi, bj = wbound(i), wbound(j)
            if bi is not None and bj is not None and w >= bi + bj:
                continue
            useful[i].append(j)
            useful[j].append(i)
    seen = [False] * k
    pairs, tot = [], 0
    for r in range(k):
        if seen[r]:
            continue
        comp, stack = [], [r]
        seen[r] = True
        while stack:
            x = stack.pop()
            comp.append(x)
            for y in useful[x]:
                if not seen[y]:
                    seen[y] = True
                    stack.append(y)
        comp.sort()
        wp = lambda a, b: wpair(comp[a], comp[b])
        wb = lambda a: wbound(comp[a])
        if len(comp) <= 14:
            cp, ct = mwpm_dp(list(range(len(comp))), wp, wb)
        else:
            cp, ct = mwpm_blossom(len(comp), wp, wb)
        for (a, b) in cp:
            pairs.append((comp[a], comp[b] if b >= 0 else -1))
        tot += ct
    return pairs, tot


def detectors(record, code, rounds):
    """Z detectors D[t][p] from a record [syndrome bits | data bits]."""
    P = code.n_plaq
    rec = np.asarray(record, dtype=np.int64)
    mz = np.zeros((rounds, P), dtype=np.int64)
    for r in range(rounds):
        for p in range(P):
            mz[r, p] = rec[r * 2 * P + 2 * p]
    data = rec[rounds * 2 * P: rounds * 2 * P + code.n]
    D = np.zeros((rounds + 1, P), dtype=np.int64)
    prev = np.zeros(P, dtype=np.int64)
    for r in range(rounds):
        D[r] = mz[r] ^ prev
        prev = mz[r]
    for p in range(P):
        D[rounds, p] = (int(np.sum(data[code.plaq_support[p]])) & 1) ^ prev[p]
    return D


def dijkstra_wh(adj_w, src):
    """(weight, hops) lexicographic distances from src; adj_w[u] = [(v, w)]."""
    dist = {src: (0, 0)}
    pq = [(0, 0, src)]
    while pq:
        w, h, u = heapq.heappop(pq)
        if dist.get(u) != (w, h):
            continue
        for v, ew in adj_w[u]:
            cand = (w + ew, h + 1)
            if v not in dist or cand < dist[v]:
                dist[v] = cand
                heapq.heappush(pq, (cand[0], cand[1], v))
    return dist


def canonical_path_wh(adj_w, dist_to_target, src, dst):
    path = []
    u = src
    while u != dst:
        du = dist_to_target[u]
        nxt = None
        for v, ew in adj_w[u]:   # adj_w[u] sorted by (v, w)
            dv = dist_to_target.get(v)
            if dv is not None and (dv[0] + ew, dv[1] + 1) == du:
                nxt = (v, ew)
                break
        path.append((edge_key(u, nxt[0]), nxt[1]))
        u = nxt[0]
    return path


def decode_color(G, D, c):
    """One colour's candidate.  Returns (score, corrected-qubit parity)."""
    P, T, B = G.P, G.T, G.B
    code = G.code
    s1 = G.stage1[c]
    adj, dist = s1["adj"], s1["dist"]
    defects = sorted(t * P + p for t in range(T) for p in range(P)
                     if code.plaq_color[p] != c and D[t][p])

    def wp(i, j):
        a, b = defects[i], defects[j]
        w = dist[a].get(b)
        return None if w is None else w * WUNIT + pair_hash(a, b, 0, c)

    def wb(i):
        a = defects[i]
        w = dist[a].get(B)
        return None if w is None else w * WUNIT + pair_hash(a, B, 0, c)

    pairs, tot1 = mwpm(defects, wp, wb)
    score1 = tot1 // WUNIT
    # stage-1 edges (XOR of canonical paths, from the smaller id)
    e1 = {}
    for (i, j) in pairs:
        a = defects[i]
        b = B if j < 0 else defects[j]
        src, dst = (a, b) if a < b else (b, a)
        for ek in canonical_path_unit(adj, dist[dst], src, dst):
            e1[ek] = e1.get(ek, 0) ^ 1
    e1 = {ek for ek, m in e1.items() if m}

    # stage 2 graph
    cface = s1["cface"]
    corr_parity = 0
    resid = {t * P + g: int(D[t][g]) for t in range(T) for g in range(P)
             if code.plaq_color[g] == c}

    def cnode(t, q):
        g = cface[q]
        return B if g < 0 else t * P + g

    adj_w = {v: {} for v in resid}
    adj_w[B] = {}

    def add_edge(u, v, w):
        if u == v:
            return
        for (x, y) in ((u, v), (v, u)):
            if y not in adj_w[x] or w < adj_w[x][y]:
                adj_w[x][y] = w

    for S, qs in s1["qsets"].items():
        qs = sorted(qs)
        for t in range(T):
            if len(S) == 0:
                for q in qs:
                    add_edge(cnode(t, q), B, 1)
                continue
            u = t * P + S[0]
            v = t * P + S[1] if len(S) == 2 else B
            if edge_key(u, v) in e1:
                q1 = qs[0]
                corr_parity ^= 1
                n1 = cnode(t, q1)
                if n1 != B:
                    resid[n1] ^= 1
                for qj in qs[1:]:
                    add_edge(n1, cnode(t, qj), 0)
            else:
                for i in range(len(qs)):
                    for j in range(i + 1, len(qs)):
                        add_edge(cnode(t, qs[i]), cnode(t, qs[j]), 2)
    for t in range(T - 1):
        for g in range(P):
            if code.plaq_color[g] == c:
                add_edge(t * P + g, (t + 1) * P + g, 1)
    adj_l = {u: sorted(nb.items()) for u, nb in adj_w.items()}

    defects2 = sorted(v for v, m in resid.items() if m)
    dists = {v: dijkstra_wh(adj_l, v) for v in defects2 + [B]}

    def wp2(i, j):
        a, b = defects2[i], defects2[j]
        dd = dists[a].get(b)
        return None if dd is None else dd[0] * WUNIT + pair_hash(a, b, 1, c)

    def wb2(i):
        a = defects2[i]
        dd = dists[a].get(B)
        return None if dd is None else dd[0] * WUNIT + pair_hash(a, B, 1, c)

    pairs2, tot2 = mwpm(defects2, wp2, wb2)
    score2 = tot2 // WUNIT
    for (i, j) in pairs2:
        a = defects2[i]
        b = B if j < 0 else defects2[j]
        src, dst = (a, b) if a < b else (b, a)
        for (ek, w) in canonical_path_wh(adj_l, dists[dst], src, dst):
            # choice edges swap one qubit for another (parity unchanged);
            # pair edges flip two qubits; weight-1 edges are one qubit
            # (boundary) or a time edge (no data qubit).
            if w == 1 and (ek[1] == B or ek[0] == B):
                corr_parity ^= 1
    return score1 + score2, corr_parity


def decode(G, record):
    """Returns (fail bit, winning colour, score)."""
    D = detectors(record, G.code, G.C)
    best = None
    for c in range(3):
        score, par = decode_color(G, D, c)
        if best is None or score < best[0]:
            best = (score, c, par)
    data = np.asarray(record)[G.C * 2 * G.P: G.C * 2 * G.P + G.code.n]
    fail = (int(np.sum(data)) & 1) ^ best[2]
    return fail, best[1], best[0]

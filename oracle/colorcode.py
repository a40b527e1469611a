"""Triangular hexagonal (6.6.6) color code, [[ (3d^2+1)/4, 1, d ]].

Oracle (test infrastructure only).  Follows Sec. II.A ("The hexagonal color
code") and App. A.1 ("The topological formulation of the color code"): qubits
sit on the vertices of a honeycomb lattice, every face (plaquette) carries one
X and one Z stabilizer acting on its vertices, faces are 3-colorable, and a
triangular patch gives weight-6 bulk and weight-4 boundary plaquettes with
one logical qubit.

Construction (the paper's figure is not available, so the patch is built from
its geometric definition): on the triangular lattice a*e1 + b*e2, take the
points with a, b >= 0 and a + b <= M, M = 3(d-1)/2.  Points with
(a - b) mod 3 == 1 are face centres, the rest are honeycomb vertices (qubits).
A face's qubits are its six lattice neighbours that lie in the patch.  Face
colour = a mod 3.  Qubits and faces are numbered row by row (b, then a).

Pinned by tests/test_oracle_code.py against closed forms: n = (3d^2+1)/4,
#faces = (n-1)/2, sum of weights 12/42/90, weights in {4,6}, all X/Z checks
commute, k = 1 (GF(2) rank), and the code distance (brute force).
"""
from dataclasses import dataclass, field

# Neighbour directions of a lattice point, in a fixed order; the CNOT schedule
# uses this index as the time slot of a face's CNOT with that neighbour.
DIRS = ((1, 0), (0, 1), (-1, 1), (-1, 0), (0, -1), (1, -1))


@dataclass
class ColorCode:
    d: int
    n: int                      # data qubits
    n_plaq: int                 # plaquettes (faces)
    qubit_pos: list             # (a, b) lattice point of each data qubit
    plaq_pos: list              # (a, b) lattice point of each face centre
    plaq_dir: list              # per face: 6 entries, data qubit or -1
    plaq_color: list            # per face: 0, 1, 2
    plaq_support: list = field(default_factory=list)   # per face: sorted qubits
    qubit_plaqs: list = field(default_factory=list)    # per qubit: sorted faces


def color_code(d: int) -> ColorCode:
    if d < 3 or d % 2 == 0:
        raise ValueError("distance must be odd and >= 3")
    M = 3 * (d - 1) // 2
    pts = [(a, b) for b in range(M + 1) for a in range(M + 1 - b)]
    is_face = lambda p: (p[0] - p[1]) % 3 == 1
    qpos = sorted([p for p in pts if not is_face(p)], key=lambda p: (p[1], p[0]))
    fpos = sorted([p for p in pts if is_face(p)], key=lambda p: (p[1], p[0]))
    qidx = {p: i for i, p in enumerate(qpos)}
    pdir = []
    for (a, b) in fpos:
        pdir.append([qidx.get((a + da, b + db), -1) for (da, db) in DIRS])
    code = ColorCode(d=d, n=len(qpos), n_plaq=len(fpos), qubit_pos=qpos,
                     plaq_pos=fpos, plaq_dir=pdir,
                     plaq_color=[a % 3 for (a, b) in fpos])
    code.plaq_support = [sorted(q for q in row if q >= 0) for row in pdir]
    code.qubit_plaqs = [[] for _ in range(code.n)]
    for p, sup in enumerate(code.plaq_support):
        for q in sup:
            code.qubit_plaqs[q].append(p)
    return code


def check_matrix(code: ColorCode):
    """Face-qubit incidence matrix H (n_plaq x n) over GF(2), as 0/1 ints.

    The code is self-dual CSS: H is the check matrix of both the X and the Z
    stabilizers (App. A.1)."""
    H = [[0] * code.n for _ in range(code.n_plaq)]
    for p, sup in enumerate(code.plaq_support):
        for q in sup:
            H[p][q] = 1
    return H


def n_qubits_total(code: ColorCode) -> int:
    """Data plus one Z- and one X-ancilla per plaquette (Sec. II.A)."""
    return code.n + 2 * code.n_plaq

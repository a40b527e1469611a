// Host-side construction of the color code, its syndrome-extraction circuit,
// the qubit-to-leaf layout and the per-trajectory step program.
//
// Color code: triangular 6.6.6 patch [[ (3d^2+1)/4, 1, d ]] (Sec. II.A, App. A.1)
// built from its geometric definition -- lattice points a*e1 + b*e2 with
// a, b >= 0, a + b <= 3(d-1)/2; points with (a - b) mod 3 == 1 are face
// centres, the others are qubits; a face acts on its lattice neighbours in the
// patch; face colour = a mod 3; qubits and faces numbered row by row.
//
// Circuit: C cycles of non-fault-tolerant extraction (Sec. III, Fig. 1a):
// per face one |0> ancilla (Z check, CNOT data -> ancilla) and one |+>
// ancilla (X check, CNOT ancilla -> data); a geometric schedule in which slot
// s = 0..5 of each block runs every face's CNOT with its neighbour in lattice
// direction s; an error location after every layer on every qubit the layer
// does not measure (Fig. 1b-d); final Z readout of the data.  Qubits: data
// 0..n-1, Z ancilla of face p at n + 2p, X ancilla at n + 2p + 1.
//
// Layout: the recursive binary split of App. B (Algorithm 1) with the
// similarity of Eq. 9, f(qi, qj) = |G(qi) ^ G(qj)| + 1 / (|G(qi)| + |G(qj)|),
// clustered by spectral bisection (Fiedler vector of the similarity
// Laplacian) and cut to the subtree capacity.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

#include "internal.h"

namespace ttn {

static const int DIRS[6][2] = {{1, 0}, {0, 1}, {-1, 1}, {-1, 0}, {0, -1}, {1, -1}};

Code build_code(int d) {
  Code code;
  code.d = d;
  const int M = 3 * (d - 1) / 2;
  std::vector<std::pair<int, int>> qpos, fpos;  // (b, a): row-major sort keys
  for (int b = 0; b <= M; ++b)
    for (int a = 0; a + b <= M; ++a) {
      int cls = ((a - b) % 3 + 3) % 3;
      if (cls == 1) fpos.push_back({b, a});
      else qpos.push_back({b, a});
    }
  std::sort(qpos.begin(), qpos.end());
  std::sort(fpos.begin(), fpos.end());
  std::map<std::pair<int, int>, int> qidx;  // (a, b) -> qubit
  for (size_t i = 0; i < qpos.size(); ++i) qidx[{qpos[i].second, qpos[i].first}] = (int)i;
  code.n = (int)qpos.size();
  code.P = (int)fpos.size();
  code.dir.resize(code.P);
  code.color.resize(code.P);
  code.support.resize(code.P);
  code.qplaqs.assign(code.n, {});
  for (int p = 0; p < code.P; ++p) {
    int a = fpos[p].second, b = fpos[p].first;
    code.color[p] = a % 3;
    for (int s = 0; s < 6; ++s) {
      auto it = qidx.find({a + DIRS[s][0], b + DIRS[s][1]});
      code.dir[p][s] = it == qidx.end() ? -1 : it->second;
      if (it != qidx.end()) code.support[p].push_back(it->second);
    }
    std::sort(code.support[p].begin(), code.support[p].end());
    for (int q : code.support[p]) code.qplaqs[q].push_back(p);
  }
  return code;
}

std::vector<Op> build_ops(const Code& code, int rounds, int* n_layers, int* n_events,
                          int* n_locations) {
  const int n = code.n, P = code.P, N = n + 2 * P;
  std::vector<Op> ops;
  int ev = 0, loc = 0, layer = 0;
  auto noise = [&](int upto) {
    for (int q = 0; q < upto; ++q) ops.push_back({NOISE, q, loc++, ev++, -1, layer});
  };
  auto zanc = [&](int p) { return n + 2 * p; };
  auto xanc = [&](int p) { return n + 2 * p + 1; };
  for (int r = 0; r < rounds; ++r) {
    if (r == 0)
      for (int q = 0; q < n; ++q) ops.push_back({PREP_Z, q, -1, -1, -1, layer});
    for (int p = 0; p < P; ++p) {
      ops.push_back({PREP_Z, zanc(p), -1, -1, -1, layer});
      ops.push_back({PREP_X, xanc(p), -1, -1, -1, layer});
    }
    noise(N);
    ++layer;
    for (int s = 0; s < 6; ++s) {
      for (int p = 0; p < P; ++p)
        if (code.dir[p][s] >= 0) ops.push_back({CNOT, code.dir[p][s], zanc(p), -1, -1, layer});
      noise(N);
      ++layer;
    }
    for (int s = 0; s < 6; ++s) {
      for (int p = 0; p < P; ++p)
        if (code.dir[p][s] >= 0) ops.push_back({CNOT, xanc(p), code.dir[p][s], -1, -1, layer});
      noise(N);
      ++layer;
    }
    for (int p = 0; p < P; ++p) {
      ops.push_back({MEAS_Z, zanc(p), -1, ev++, r * 2 * P + 2 * p, layer});
      ops.push_back({MEAS_X, xanc(p), -1, ev++, r * 2 * P + 2 * p + 1, layer});
    }
    noise(n);
    ++layer;
  }
  for (int q = 0; q < n; ++q) ops.push_back({MEAS_Z, q, -1, ev++, rounds * 2 * P + q, layer});
  ++layer;
  *n_layers = layer;
  *n_events = ev;
  *n_locations = loc;
  return ops;
}

// Symmetric eigenproblem by cyclic Jacobi rotations (host, small n).  Returns
// eigenvalues ascending with eigenvectors as columns of V (row-major n x n).
static void sym_eig(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (i != j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        double zeta = (aqq - app) / (2.0 * apq);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  w.resize(n);
  std::vector<double> V2((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)idx[j] * n + idx[j]];
    for (int k = 0; k < n; ++k) V2[(size_t)k * n + j] = V[(size_t)k * n + idx[j]];
  }
  V.swap(V2);
}

// Recursive capacity-constrained spectral bisection (App. B, Algorithm 1).
static void split_rec(const std::vector<int>& Q, int lo, int height, const std::vector<double>& S,
                      int N, std::vector<int>& leaf_of) {
  if (Q.empty()) return;
  if (height == 0) {
    leaf_of[Q[0]] = lo;
    return;
  }
  const int half = 1 << (height - 1);
  if ((int)Q.size() == 1) {
    leaf_of[Q[0]] = lo;
    return;
  }
  std::vector<int> A, B;
  if ((int)Q.size() == 2 && height == 1) {
    A = {Q[0]};
    B = {Q[1]};
  } else {
    const int m = (int)Q.size();
    std::vector<double> Lap((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        if (i != j) {
          double s = S[(size_t)Q[i] * N + Q[j]];
          Lap[(size_t)i * m + j] = -s;
          Lap[(size_t)i * m + i] += s;
        }
    std::vector<double> w, V;
    sym_eig(m, Lap, w, V);
    std::vector<double> f(m);
    for (int i = 0; i < m; ++i) f[i] = V[(size_t)i * m + (m > 1 ? 1 : 0)];
    // orientation: the lowest-numbered qubit gets a non-positive value
    int imin = (int)(std::min_element(Q.begin(), Q.end()) - Q.begin());
    if (f[imin] > 0)
      for (double& x : f) x = -x;
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      if (f[a] != f[b]) return f[a] < f[b];
      return Q[a] < Q[b];
    });
    int cut = 0;
    for (int i = 0; i < m; ++i) cut += f[i] <= 0.0;
    cut = std::max(cut, m - half);
    cut = std::min(cut, half);
    for (int i = 0; i < m; ++i) (i < cut ? A : B).push_back(Q[ord[i]]);
  }
  split_rec(A, lo, height - 1, S, N, leaf_of);
  split_rec(B, lo + half, height - 1, S, N, leaf_of);
}

static std::vector<double> gate_similarity(const std::vector<Op>& ops, int N) {
  std::vector<double> shared((size_t)N * N, 0.0);
  std::vector<int> deg(N, 0);
  for (const Op& op : ops)
    if (op.kind == CNOT) {
      shared[(size_t)op.a * N + op.b] += 1.0;
      shared[(size_t)op.b * N + op.a] += 1.0;
      deg[op.a]++;
      deg[op.b]++;
    }
  std::vector<double> S((size_t)N * N, 0.0);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      if (i != j) {
        int dsum = deg[i] + deg[j];
        S[(size_t)i * N + j] = shared[(size_t)i * N + j] + (dsum > 0 ? 1.0 / dsum : 0.0);
      }
  return S;
}

static std::vector<int> layout_from_similarity(const std::vector<double>& S, int N, int n_leaves) {
  int height = 0;
  while ((1 << height) < n_leaves) ++height;
  std::vector<int> Q(N), leaf_of(N, -1);
  std::iota(Q.begin(), Q.end(), 0);
  split_rec(Q, 0, height, S, N, leaf_of);
  return leaf_of;
}

std::vector<int> optimized_layout(const Code& code, const std::vector<Op>& ops, int N,
                                  int n_leaves) {
  (void)code;
  return layout_from_similarity(gate_similarity(ops, N), N, n_leaves);
}

// ---------------------------------------------------------------- layout search
// Noise-free bond dimension of a layout.  Without noise the extraction
// circuit is Clifford with Z/X measurements, so its state is a stabilizer
// state at every layer: N generators in binary symplectic form (x | z bit
// rows; signs do not affect entanglement), updated per H (swap x_q, z_q),
// CNOT c->t (x_t ^= x_c, z_c ^= z_t) and Z measurement (a generator with
// x_q = 1 is multiplied into the others with x_q = 1 and replaced by Z_q;
// none: deterministic, unchanged) after Aaronson and Gottesman (2004).
// Across the bond above a tree node, A = the qubits of its subtree, the
// entanglement is rank_GF2(generators restricted to A) - |A| bits (Fattal et
// al., quant-ph/0406168) and the Schmidt rank 2^that.  PREP finds its qubit
// in a Z eigenstate (initial or just measured): PREP_Z changes nothing,
// PREP_X is H; MEAS_X is H then a Z measurement.
namespace {
struct Tableau {
  int n, W;
  std::vector<uint64_t> x, z;  // [n][W] bit rows
  explicit Tableau(int n_) : n(n_), W((n_ + 63) / 64), x((size_t)n_ * W, 0), z((size_t)n_ * W, 0) {
    for (int i = 0; i < n; ++i) z[(size_t)i * W + i / 64] |= 1ull << (i % 64);
  }
  bool bit(const std::vector<uint64_t>& m, int r, int q) const {
    return (m[(size_t)r * W + q / 64] >> (q % 64)) & 1ull;
  }
  void h(int q) {
    const uint64_t msk = 1ull << (q % 64);
    for (int r = 0; r < n; ++r) {
      uint64_t& xw = x[(size_t)r * W + q / 64];
      uint64_t& zw = z[(size_t)r * W + q / 64];
      const uint64_t d = (xw ^ zw) & msk;
      xw ^= d;
      zw ^= d;
    }
  }
  void cnot(int c, int t) {
    for (int r = 0; r < n; ++r) {
      if (bit(x, r, c)) x[(size_t)r * W + t / 64] ^= 1ull << (t % 64);
      if (bit(z, r, t)) z[(size_t)r * W + c / 64] ^= 1ull << (c % 64);
    }
  }
  void measure_z(int q) {
    int p = -1;
    for (int r = 0; r < n; ++r) {
      if (!bit(x, r, q)) continue;
      if (p < 0) {
        p = r;
        continue;
      }
      for (int w = 0; w < W; ++w) {
        x[(size_t)r * W + w] ^= x[(size_t)p * W + w];
        z[(size_t)r * W + w] ^= z[(size_t)p * W + w];
      }
    }
    if (p < 0) return;
    for (int w = 0; w < W; ++w) x[(size_t)p * W + w] = z[(size_t)p * W + w] = 0;
    z[(size_t)p * W + q / 64] |= 1ull << (q % 64);
  }
  // entanglement (bits) between the qubits in A and the rest
  int entropy(const std::vector<int>& A) const {
    const int a = (int)A.size();
    if (a == 0 || a == n) return 0;
    const int cols = 2 * a, CW = (cols + 63) / 64;
    std::vector<uint64_t> M((size_t)n * CW, 0);
    for (int r = 0; r < n; ++r)
      for (int j = 0; j < a; ++j) {
        if (bit(x, r, A[j])) M[(size_t)r * CW + j / 64] |= 1ull << (j % 64);
        if (bit(z, r, A[j])) M[(size_t)r * CW + (a + j) / 64] |= 1ull << ((a + j) % 64);
      }
    int rank = 0;
    for (int c = 0; c < cols && rank < n; ++c) {
      const uint64_t msk = 1ull << (c % 64);
      int piv = -1;
      for (int r = rank; r < n; ++r)
        if (M[(size_t)r * CW + c / 64] & msk) {
          piv = r;
          break;
        }
      if (piv < 0) continue;
      if (piv != rank)
        for (int w = 0; w < CW; ++w) std::swap(M[(size_t)piv * CW + w], M[(size_t)rank * CW + w]);
      for (int r = rank + 1; r < n; ++r)
        if (M[(size_t)r * CW + c / 64] & msk)
          for (int w = 0; w < CW; ++w) M[(size_t)r * CW + w] ^= M[(size_t)rank * CW + w];
      ++rank;
    }
    return rank - a;
  }
};

uint64_t splitmix64(uint64_t v) {
  v += 0x9E3779B97F4A7C15ull;
  v = (v ^ (v >> 30)) * 0xBF58476D1CE4E5B9ull;
  v = (v ^ (v >> 27)) * 0x94D049BB133111EBull;
  return v ^ (v >> 31);
}
}  // namespace

int noise_free_bond_bits(const std::vector<Op>& ops, int N, int n_leaves, const std::vector<int>& leaf_of) {
  const int L = n_leaves;
  std::vector<std::vector<int>> under(2 * L);
  for (int q = 0; q < N; ++q)
    for (int x = L + leaf_of[q]; x >= 1; x /= 2) under[x].push_back(q);
  Tableau t(N);
  int cur = ops.empty() ? 0 : ops[0].layer, worst = 0;
  auto snap = [&]() {
    for (int v = 2; v < L; ++v) worst = std::max(worst, t.entropy(under[v]));
  };
  for (const Op& op : ops) {
    if (op.layer != cur) {
      snap();
      cur = op.layer;
    }
    switch (op.kind) {
      case PREP_X: t.h(op.a); break;
      case CNOT: t.cnot(op.a, op.b); break;
      case MEAS_Z: t.measure_z(op.a); break;
      case MEAS_X:
        t.h(op.a);
        t.measure_z(op.a);
        break;
      default: break;  // PREP_Z, NOISE: no change of entanglement
    }
  }
  snap();
  return worst;
}

// Algorithm 1 (App. B) as a seeded candidate generator.  At each tree level
// the unassigned qubits are clustered into k = 2, 3, ... groups by spectral
// clustering (rows of the k lowest Laplacian eigenvectors of the Eq. 9
// similarity, normalised, then k-means from a seeded k-means++ start); the
// clusters are merged into two groups by size, largest first into the
// smaller group (reading of the balanced agglomeration the algorithm names);
// the first k whose two groups fit the two subtrees is taken, else a seeded
// random even split; each group then fills one subtree.
namespace {
struct Rng {
  uint64_t s;
  double uniform() {
    s = splitmix64(s);
    return (double)(s >> 11) * (1.0 / 9007199254740992.0);
  }
};

std::vector<int> kmeans_labels(const std::vector<double>& X, int m, int dim, int k, Rng& rng) {
  std::vector<double> cen((size_t)k * dim);
  std::vector<double> dist(m, 0.0);
  // k-means++ start
  int first = std::min(m - 1, (int)(rng.uniform() * m));
  for (int t = 0; t < dim; ++t) cen[t] = X[(size_t)first * dim + t];
  for (int c = 1; c < k; ++c) {
    double tot = 0.0;
    for (int i = 0; i < m; ++i) {
      double best = 1e300;
      for (int cc = 0; cc < c; ++cc) {
        double d2 = 0.0;
        for (int t = 0; t < dim; ++t) {
          const double e = X[(size_t)i * dim + t] - cen[(size_t)cc * dim + t];
          d2 += e * e;
        }
        best = std::min(best, d2);
      }
      dist[i] = best;
      tot += best;
    }
    int pick = m - 1;
    double u = rng.uniform() * tot, acc = 0.0;
    for (int i = 0; i < m; ++i) {
      acc += dist[i];
      if (acc >= u && dist[i] > 0.0) {
        pick = i;
        break;
      }
    }
    for (int t = 0; t < dim; ++t) cen[(size_t)c * dim + t] = X[(size_t)pick * dim + t];
  }
  std::vector<int> lab(m, 0);
  for (int it = 0; it < 100; ++it) {
    bool changed = false;
    for (int i = 0; i < m; ++i) {
      int arg = 0;
      double best = 1e300;
      for (int c = 0; c < k; ++c) {
        double d2 = 0.0;
        for (int t = 0; t < dim; ++t) {
          const double e = X[(size_t)i * dim + t] - cen[(size_t)c * dim + t];
          d2 += e * e;
        }
        if (d2 < best) best = d2, arg = c;
      }
      if (lab[i] != arg) lab[i] = arg, changed = true;
    }
    std::vector<double> sum((size_t)k * dim, 0.0);
    std::vector<int> cnt(k, 0);
    for (int i = 0; i < m; ++i) {
      cnt[lab[i]]++;
      for (int t = 0; t < dim; ++t) sum[(size_t)lab[i] * dim + t] += X[(size_t)i * dim + t];
    }
    for (int c = 0; c < k; ++c)
      if (cnt[c] > 0)
        for (int t = 0; t < dim; ++t) cen[(size_t)c * dim + t] = sum[(size_t)c * dim + t] / cnt[c];
    if (!changed && it > 0) break;
  }
  return lab;
}

void alg1_rec(const std::vector<int>& Q, int lo, int height, const std::vector<double>& S, int N, Rng& rng,
              std::vector<int>& leaf_of) {
  if (Q.empty()) return;
  const int half = height > 0 ? 1 << (height - 1) : 0;
  if (height == 0) {
    leaf_of[Q[0]] = lo;
    return;
  }
  if ((int)Q.size() <= 2) {
    alg1_rec({Q[0]}, lo, height - 1, S, N, rng, leaf_of);
    if (Q.size() == 2) alg1_rec({Q[1]}, lo + half, height - 1, S, N, rng, leaf_of);
    return;
  }
  const int m = (int)Q.size();
  std::vector<double> Lap((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      if (i != j) {
        const double sv = S[(size_t)Q[i] * N + Q[j]];
        Lap[(size_t)i * m + j] = -sv;
        Lap[(size_t)i * m + i] += sv;
      }
  std::vector<double> w, V;
  sym_eig(m, Lap, w, V);
  std::vector<int> A, B;
  for (int k = 2; k <= m && A.empty(); ++k) {
    std::vector<double> X((size_t)m * k);
    for (int i = 0; i < m; ++i) {
      double nrm = 0.0;
      for (int t = 0; t < k; ++t) nrm += V[(size_t)i * m + t] * V[(size_t)i * m + t];
      nrm = nrm > 0.0 ? 1.0 / std::sqrt(nrm) : 1.0;
      for (int t = 0; t < k; ++t) X[(size_t)i * k + t] = V[(size_t)i * m + t] * nrm;
    }
    std::vector<int> lab = kmeans_labels(X, m, k, k, rng);
    std::vector<std::vector<int>> cl(k);
    for (int i = 0; i < m; ++i) cl[lab[i]].push_back(Q[i]);
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cl[a].size() > cl[b].size(); });
    std::vector<int> g0, g1;
    for (int c : order) {
      std::vector<int>& g = g0.size() <= g1.size() ? g0 : g1;
      g.insert(g.end(), cl[c].begin(), cl[c].end());
    }
    if ((int)g0.size() <= half && (int)g1.size() <= half && !g0.empty() && !g1.empty()) {
      A.swap(g0);
      B.swap(g1);
    }
    if (k >= 12) break;  // beyond a dozen clusters the merge is a balanced random split anyway
  }
  if (A.empty()) {  // random even split
    std::vector<int> P(Q);
    for (int i = m - 1; i > 0; --i) std::swap(P[i], P[(int)(rng.uniform() * (i + 1)) % (i + 1)]);
    A.assign(P.begin(), P.begin() + m / 2);
    B.assign(P.begin() + m / 2, P.end());
  }
  alg1_rec(A, lo, height - 1, S, N, rng, leaf_of);
  alg1_rec(B, lo + half, height - 1, S, N, rng, leaf_of);
}
}  // namespace

static std::vector<int> alg1_layout(const std::vector<double>& S, int N, int n_leaves, uint64_t seed) {
  int height = 0;
  while ((1 << height) < n_leaves) ++height;
  std::vector<int> Q(N), leaf_of(N, -1);
  std::iota(Q.begin(), Q.end(), 0);
  Rng rng{seed};
  alg1_rec(Q, 0, height, S, N, rng, leaf_of);
  return leaf_of;
}

// Candidate layouts from the clustering (App. B: the clustering is a
// heuristic, so candidates are sampled and the best is kept): candidate 0 is
// optimized_layout; candidates 1 .. candidates/2 - 1 split a similarity
// whose off-diagonal entries are scaled by independent factors in
// [0.95, 1.05] (seeded by the candidate), which moves the Fiedler cuts
// where they are close; the rest run Algorithm 1 with seeded k-means and
// random splits.  The kept candidate has
// the smallest noise-free bond dimension (a cost evaluated without
// simulating the noisy circuit); ties keep the earlier candidate.
std::vector<int> searched_layout(const Code& code, const std::vector<Op>& ops, int N, int n_leaves,
                                 int candidates) {
  (void)code;
  const std::vector<double> S = gate_similarity(ops, N);
  std::vector<int> best = layout_from_similarity(S, N, n_leaves);
  int best_bits = noise_free_bond_bits(ops, N, n_leaves, best);
  std::vector<double> Sc(S.size());
  for (int c = 1; c < candidates; ++c) {
    std::vector<int> lay;
    if (c < candidates / 2) {
      for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
          const uint64_t h = splitmix64(((uint64_t)c << 40) ^ ((uint64_t)i << 20) ^ (uint64_t)j);
          const double f = 1.0 + 0.1 * ((double)(h >> 11) * (1.0 / 9007199254740992.0) - 0.5);
          Sc[(size_t)i * N + j] = Sc[(size_t)j * N + i] = S[(size_t)i * N + j] * f;
        }
      for (int i = 0; i < N; ++i) Sc[(size_t)i * N + i] = 0.0;
      lay = layout_from_similarity(Sc, N, n_leaves);
    } else {
      lay = alg1_layout(S, N, n_leaves, 0x5EED0000ull + (uint64_t)c);
    }
    const int bits = noise_free_bond_bits(ops, N, n_leaves, lay);
    if (bits < best_bits) {
      best_bits = bits;
      best.swap(lay);
    }
  }
  return best;
}

// ---------------------------------------------------------------- step program
namespace {

struct Compiler {
  const ttn_circuit& c;
  Program prog;
  int center = 1;

  explicit Compiler(const ttn_circuit& cc) : c(cc) {}

  int pos(int q) const { return c.L + c.leaf_of_qubit[q]; }

  std::vector<int> path(int v, int w) const {
    std::vector<int> up_v{v}, up_w{w};
    int a = v, b = w;
    while (a != b) {
      if (a > b) {
        a /= 2;
        up_v.push_back(a);
      } else {
        b /= 2;
        up_w.push_back(b);
      }
    }
    for (int i = (int)up_w.size() - 2; i >= 0; --i) up_v.push_back(up_w[i]);
    return up_v;
  }

  void move(int v, int w, int capped) {
    prog.steps.push_back({S_MOVE, v, w, capped, 0, 0});
    center = w;
  }

  void route(int target) {
    std::vector<int> p = path(center, target);
    for (size_t i = 0; i + 1 < p.size(); ++i) move(p[i], p[i + 1], 0);
  }

  static int leg_of(int v, int w) { return w == 2 * v ? 0 : (w == 2 * v + 1 ? 1 : 2); }

  void cnot(int a, int b) {
    int pa = pos(a), pb = pos(b);
    int va = pa / 2, vb = pb / 2;
    if (va == vb) {
      route(va);
      prog.steps.push_back({S_GATE_NODE, va, (pa % 2 == 0) ? 0 : 1, 0, 0, 0});
      return;
    }
    int x = va, y = vb;
    while (x != y) {
      if (x > y) x /= 2;
      else y /= 2;
    }
    const int lca = x;
    route(lca);
    auto branch = [&](int v0) {
      std::vector<int> nodes{v0};
      int v = v0;
      while (v / 2 != lca) {
        v /= 2;
        nodes.push_back(v);
      }
      return nodes;
    };
    std::vector<int> sa = branch(va), sb = branch(vb);
    for (int side = 0; side < 2; ++side) {
      const std::vector<int>& s = side == 0 ? sa : sb;
      int p = side == 0 ? pa : pb;
      prog.steps.push_back({S_THREAD_LEAF, s[0], p % 2, side, 0, 0});
      for (size_t i = 1; i < s.size(); ++i)
        prog.steps.push_back({S_THREAD_NODE, s[i], leg_of(s[i], s[i - 1]), 0, 0, 0});
    }
    prog.steps.push_back({S_THREAD_LCA, lca, 0, 0, 0, 0});
    for (int side = 0; side < 2; ++side) {
      const std::vector<int>& s = side == 0 ? sa : sb;
      for (size_t i = 0; i < s.size(); ++i) move(s[i], i + 1 < s.size() ? s[i + 1] : lca, 0);
    }
    center = lca;
    move(lca, sb.back(), 1);
    for (int i = (int)sb.size() - 1; i > 0; --i) move(sb[i], sb[i - 1], 1);
    route(lca);
    move(lca, sa.back(), 1);
    for (int i = (int)sa.size() - 1; i > 0; --i) move(sa[i], sa[i - 1], 1);
  }

  // flush the fused single-qubit ops collected for the current layer
  std::vector<std::vector<Op1>> pending;  // per level-1 node (index node - L/2)

  void add1(int q, int kind, int event) {
    int p = pos(q);
    int node = p / 2;
    if (pending.empty()) pending.resize(c.L / 2);
    pending[node - c.L / 2].push_back({p % 2, kind, q, event});
  }

  void flush1() {
    if (pending.empty()) return;
    int b0 = (int)prog.op1.size(), g0 = (int)prog.groups.size();
    for (int i = 0; i < (int)pending.size(); ++i) {
      if (pending[i].empty()) continue;
      int begin = (int)prog.op1.size();
      for (const Op1& o : pending[i]) prog.op1.push_back(o);
      prog.groups.push_back({i + c.L / 2, begin, (int)prog.op1.size(), 0});
    }
    int b1 = (int)prog.op1.size(), g1 = (int)prog.groups.size();
    if (g1 > g0) prog.steps.push_back({S_LAYER1Q, b0, b1, g0, g1, 0});
    pending.clear();
  }
};

}  // namespace

Program compile_program(const ttn_circuit& c, int noise, int last_layer) {
  Compiler cp(c);
  const bool ad = noise == TTN_NOISE_AD || noise == TTN_NOISE_SRX_AD;
  const bool srx = noise == TTN_NOISE_SRX || noise == TTN_NOISE_SRX_AD;
  const bool pta = noise == TTN_NOISE_SRX_PTA || noise == TTN_NOISE_AD_PTA || noise == TTN_NOISE_DEPOL;
  int cur = 0;
  std::vector<int> ad_q, ad_e;
  auto end_layer = [&]() {
    cp.flush1();
    for (size_t i = 0; i < ad_q.size(); ++i) {
      cp.route(cp.pos(ad_q[i]) / 2);
      cp.prog.steps.push_back({S_AD, ad_q[i], ad_e[i], 0, 0, 0});
    }
    ad_q.clear();
    ad_e.clear();
    cp.prog.stop_step_of_layer.push_back((int)cp.prog.steps.size());
  };
  for (const Op& op : c.ops) {
    if (op.layer != cur) {
      end_layer();
      cur = op.layer;
      if (last_layer >= 0 && cur > last_layer) break;
    }
    switch (op.kind) {
      case PREP_Z: cp.add1(op.a, O1_RESET_Z, -1); break;
      case PREP_X: cp.add1(op.a, O1_RESET_X, -1); break;
      case CNOT: cp.cnot(op.a, op.b); break;
      case MEAS_Z:
      case MEAS_X:
        cp.route(cp.pos(op.a) / 2);
        cp.prog.steps.push_back({S_MEASURE, op.a, op.event, op.rec, op.kind == MEAS_X, 0});
        break;
      case NOISE:
        if (srx) cp.add1(op.a, O1_SRX, op.event);
        if (pta) cp.add1(op.a, O1_PTA, op.event);
        if (ad) {
          ad_q.push_back(op.a);
          ad_e.push_back(op.event);
        }
        break;
    }
  }
  if (last_layer < 0 || cur <= last_layer) end_layer();
  return cp.prog;
}

}  // namespace ttn

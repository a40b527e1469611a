// Concatenated minimum-weight perfect-matching decoder (App. A.2) as a
// batched integer kernel: one thread per shot, all three colours.
//
// Definition (the paper defers the details to a reference that is not
// available; this is the reading the library implements):
//   detectors D[t][p] = mZ[t][p] ^ mZ[t-1][p] (t < C, mZ[-1] = 0) and
//   D[C][p] = parity(data on p) ^ mZ[C-1][p]; node id t * P + p, boundary
//   B = (C+1) * P.
//   Stage 1 (colour c): graph on the non-c detectors; space edge per layer for
//   every "non-c face set" S of a data qubit (two faces: edge between them,
//   one face: edge to B), time edges between layers, unit weights; exact MWPM
//   of the defects (each to another defect or to B) on shortest-path
//   distances; the matched edges E1 are the XOR of canonical shortest paths
//   (from the smaller id, stepping to the smallest-id neighbour that stays on
//   a shortest path).
//   Stage 2 (colour c): graph on the c detectors and B.  Each space edge of
//   E1 flips its default qubit q1 = min Q(S) (one correction) and its c-face;
//   choice edges (weight 0) swap q1 for another qubit of Q(S); unmatched
//   classes give pair edges (weight 2, flip two qubits of Q(S)); qubits with
//   no non-c face give weight-1 edges to B; time edges weight 1.  Exact MWPM
//   of the residual c-defects on (weight, hops) shortest paths; weight-1
//   edges at B flip one qubit.
//   Score = stage-1 + stage-2 weight; the lowest score wins (ties: lowest c);
//   fail = parity(data) ^ parity(number of corrected qubits)  (Z-bar = Z^n).
//   Matching weights are w * 2^40 + h(a, b), h a 28-bit splitmix64 hash of
//   the node pair, stage and colour, so the optimum is unique.
// Exact matching: the optimum splits over connected components of the pairs
// cheaper than sending both defects to the boundary; a component of at most
// KCOMP defects is solved by a subset DP, a larger one by the weighted
// blossom algorithm (blossom.cuh) on the defects and their boundary copies.
// At most KMAX defects per instance (beyond that the overflow counter is
// raised and the shot's fail byte is 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "blossom.cuh"
#include "engine.h"

namespace ttn {

static constexpr int KMAX = 128;   // defects per matching instance
static constexpr int KCOMP = 12;   // largest component solved by the subset DP
static_assert(2 * KMAX <= BL_NMAX, "blossom size");
static constexpr int64_t WUNIT = (int64_t)1 << 40;
static constexpr int64_t INF64 = (int64_t)1 << 62;

DecoderTables build_decoder_tables(const Code& code, int rounds) {
  DecoderTables t;
  t.T = rounds + 1;
  t.P = code.P;
  t.B = t.T * t.P;
  t.n_nodes = t.B + 1;
  t.n = code.n;
  t.color = code.color;
  const int P = t.P, T = t.T, B = t.B, NN = t.n_nodes, n = code.n;
  t.support_off.push_back(0);
  for (int p = 0; p < P; ++p) {
    for (int q : code.support[p]) t.support.push_back(q);
    t.support_off.push_back((int)t.support.size());
  }
  std::vector<std::vector<std::vector<int>>> cls_qs(3);
  std::vector<std::vector<std::pair<int, int>>> cls_faces(3);
  t.cface.assign(3 * n, -1);
  for (int c = 0; c < 3; ++c) {
    std::map<std::vector<int>, std::vector<int>> qsets;
    for (int q = 0; q < n; ++q) {
      std::vector<int> S;
      for (int f : code.qplaqs[q]) {
        if (code.color[f] != c) S.push_back(f);
        else t.cface[c * n + q] = f;
      }
      qsets[S].push_back(q);
    }
    for (auto& kv : qsets) {
      cls_qs[c].push_back(kv.second);
      int f1 = kv.first.size() > 0 ? kv.first[0] : -1;
      int f2 = kv.first.size() > 1 ? kv.first[1] : -1;
      cls_faces[c].push_back({f1, f2});
    }
    t.n_cls_max = std::max(t.n_cls_max, (int)qsets.size());
  }
  const int ncm = t.n_cls_max;
  t.cls_off.assign(3 * (ncm + 1), 0);
  t.cls_f.assign(3 * ncm * 2, -1);
  t.n_cls.assign(3, 0);
  for (int c = 0; c < 3; ++c) {
    t.n_cls[c] = (int)cls_qs[c].size();
    for (int i = 0; i <= ncm; ++i) {
      t.cls_off[c * (ncm + 1) + i] = (int)t.cls_q.size();
      if (i < t.n_cls[c]) {
        for (int q : cls_qs[c][i]) t.cls_q.push_back(q);
        t.cls_f[(c * ncm + i) * 2] = cls_faces[c][i].first;
        t.cls_f[(c * ncm + i) * 2 + 1] = cls_faces[c][i].second;
      }
    }
  }
  // stage-1 graphs and all-pairs BFS distances
  t.dist1.assign((size_t)3 * NN * NN, -1);
  t.adj1_off.assign(3 * (NN + 1), 0);
  t.adj1_base.assign(3, 0);
  for (int c = 0; c < 3; ++c) {
    std::vector<std::vector<int>> adj(NN);
    auto link = [&](int u, int v) {
      adj[u].push_back(v);
      adj[v].push_back(u);
    };
    for (int i = 0; i < t.n_cls[c]; ++i) {
      int f1 = cls_faces[c][i].first, f2 = cls_faces[c][i].second;
      if (f1 < 0) continue;
      for (int tt = 0; tt < T; ++tt) link(tt * P + f1, f2 >= 0 ? tt * P + f2 : B);
    }
    for (int tt = 0; tt + 1 < T; ++tt)
      for (int p = 0; p < P; ++p)
        if (code.color[p] != c) link(tt * P + p, (tt + 1) * P + p);
    for (auto& a : adj) {
      std::sort(a.begin(), a.end());
      a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    t.adj1_base[c] = (int)t.adj1.size();
    for (int u = 0; u < NN; ++u) {
      t.adj1_off[c * (NN + 1) + u] = (int)t.adj1.size();
      for (int v : adj[u]) t.adj1.push_back(v);
    }
    t.adj1_off[c * (NN + 1) + NN] = (int)t.adj1.size();
    for (int s = 0; s < NN; ++s) {
      int32_t* dist = &t.dist1[((size_t)c * NN + s) * NN];
      std::deque<int> dq{s};
      dist[s] = 0;
      while (!dq.empty()) {
        int u = dq.front();
        dq.pop_front();
        for (int v : adj[u])
          if (dist[v] < 0) {
            dist[v] = dist[u] + 1;
            dq.push_back(v);
          }
      }
    }
  }
  return t;
}

// ------------------------------------------------------------------ device
struct DecDev {
  int T, P, B, NN, n, n_rec, C, ncm;
  const int32_t* color;
  const int32_t* support_off;
  const int32_t* support;
  const int32_t* dist1;
  const int32_t* adj1_off;
  const int32_t* adj1;
  const int32_t* cls_off;
  const int32_t* cls_q;
  const int32_t* cls_f;
  const int32_t* n_cls;
  const int32_t* clsof;    // [3][P][P+1]
  const int32_t* cface;    // [3][n]
  const int32_t* inc_off;  // [3][P+1]
  const int32_t* inc;      // (cls, q) pairs
  // per-shot scratch
  int64_t* dp_f;
  int8_t* dp_c;
  int64_t* dist2;          // [KMAX + 1][NN]
  uint8_t* e1;             // [T * ncm + T * P]
  uint8_t* resid;          // [NN]
  int* defs;               // [4 * KMAX] defects, partners, components, local ids
  int64_t* wb;             // [KMAX] boundary weights
  size_t dp_stride, d2_stride, e1_stride;
  unsigned char* bls;      // blossom scratch, bl_stride bytes per shot
  size_t bl_stride;
  int32_t* overflow;
};

__device__ __forceinline__ uint64_t pair_hash(int a, int b, int stage, int color) {
  if (a > b) {
    int t = a;
    a = b;
    b = t;
  }
  uint64_t x = (uint64_t)a * 0x9E3779B97F4A7C15ull + (uint64_t)b * 0xBF58476D1CE4E5B9ull +
               (uint64_t)(stage * 3 + color + 1) * 0x94D049BB133111EBull;
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x >> 36;
}

// Exact minimum-weight matching of k defects (each to another defect or to
// the boundary).  A pair with W(i,j) >= Wb(i) + Wb(j) is never better than
// sending both to the boundary, so the optimum decomposes over the connected
// components of the graph of the other pairs; each component is solved
// exactly by a subset DP.  wfun(i, j) / wb[i] return the perturbed weight or
// a negative value when absent.  Returns the total, or -1 when a component
// -2 when no perfect matching exists.  Components above KCOMP defects go to
// the blossom matcher (scratch bl).
template <typename WF>
__device__ int64_t mwpm_exact(int k, WF wfun, const int64_t* wb, int64_t* f, int8_t* ch, int* partner,
                              int* comp, int* loc, void* bl) {
  // union-find by label propagation (k <= KMAX_TOTAL)
  for (int i = 0; i < k; ++i) comp[i] = i;
  bool changed = true;
  while (changed) {
    changed = false;
    for (int i = 0; i < k; ++i)
      for (int j = i + 1; j < k; ++j) {
        if (comp[i] == comp[j]) continue;
        const int64_t w = wfun(i, j);
        if (w < 0) continue;
        if (wb[i] >= 0 && wb[j] >= 0 && w >= wb[i] + wb[j]) continue;
        const int m = min(comp[i], comp[j]);
        comp[i] = comp[j] = m;
        changed = true;
      }
  }
  int64_t total = 0;
  for (int root = 0; root < k; ++root) {
    int s = 0;
    for (int i = 0; i < k; ++i)
      if (comp[i] == root) loc[s++] = i;
    if (s == 0) continue;
    if (s > KCOMP) {
      int* part = reinterpret_cast<int*>(f);  // the DP table is free here
      auto wp = [&](int i, int j) -> int64_t { return wfun(loc[i], loc[j]); };
      auto wbl = [&](int i) -> int64_t { return wb[loc[i]]; };
      const int64_t t = min_matching_boundary(s, wp, wbl, part, bl);
      if (t < 0) return t;
      total += t;
      for (int i = 0; i < s; ++i) partner[loc[i]] = part[i] >= 0 ? loc[part[i]] : -1;
      continue;
    }
    const int full = (1 << s) - 1;
    f[0] = 0;
    for (int mask = 1; mask <= full; ++mask) {
      const int a = __ffs(mask) - 1;
      const int rest = mask & ~(1 << a);
      int64_t best = INF64;
      int bc = -2;
      const int64_t wba = wb[loc[a]];
      if (wba >= 0 && f[rest] < INF64) {
        best = wba + f[rest];
        bc = -1;
      }
      int m = rest;
      while (m) {
        const int c = __ffs(m) - 1;
        m &= m - 1;
        const int64_t w = wfun(loc[a], loc[c]);
        const int sub = rest & ~(1 << c);
        if (w >= 0 && f[sub] < INF64 && w + f[sub] < best) {
          best = w + f[sub];
          bc = c;
        }
      }
      f[mask] = best;
      ch[mask] = (int8_t)bc;
    }
    if (f[full] >= INF64) return -2;
    total += f[full];
    int mask = full;
    while (mask) {
      const int a = __ffs(mask) - 1;
      const int c = ch[mask];
      partner[loc[a]] = c >= 0 ? loc[c] : -1;
      mask &= ~(1 << a);
      if (c >= 0) {
        partner[loc[c]] = loc[a];
        mask &= ~(1 << c);
      }
    }
  }
  return total;
}

__device__ __forceinline__ int edge_id1(const DecDev& d, int c, int u, int w) {
  if (u == d.B || w == d.B || (u / d.P) == (w / d.P)) {
    int x = u == d.B ? w : u;
    int y = u == d.B ? u : w;
    int t = x / d.P, fx = x % d.P;
    int fy = y == d.B ? -1 : y % d.P;
    int f1 = fy < 0 ? fx : min(fx, fy), f2 = fy < 0 ? -1 : max(fx, fy);
    int cls = d.clsof[(c * d.P + f1) * (d.P + 1) + (f2 < 0 ? d.P : f2)];
    return t * d.ncm + cls;
  }
  int lo = min(u, w);
  return d.T * d.ncm + lo;  // time edge (t, p) -> (t + 1, p), lo = t * P + p
}

// Neighbours of stage-2 node x (colour c): min weight per neighbour, sorted.
__device__ int nbrs2(const DecDev& d, int c, const uint8_t* e1, int x, int* ny, int* nw) {
  int cnt = 0;
  auto add = [&](int y, int w) {
    if (y == x) return;
    for (int i = 0; i < cnt; ++i)
      if (ny[i] == y) {
        if (w < nw[i]) nw[i] = w;
        return;
      }
    if (cnt < 256) {
      ny[cnt] = y;
      nw[cnt] = w;
      ++cnt;
    }
  };
  const int P = d.P, n = d.n;
  const int* cf = d.cface + c * n;
  auto cnode = [&](int t, int q) { return cf[q] < 0 ? d.B : t * P + cf[q]; };
  const int* coff = d.cls_off + c * (d.ncm + 1);
  if (x != d.B) {
    const int t = x / P, g = x % P;
    if (t > 0) add(x - P, 1);
    if (t + 1 < d.T) add(x + P, 1);
    const int* io = d.inc_off + c * (P + 1);
    for (int e = io[g]; e < io[g + 1]; ++e) {
      const int cls = d.inc[2 * e], q = d.inc[2 * e + 1];
      const int f1 = d.cls_f[(c * d.ncm + cls) * 2];
      const int b0 = coff[cls], b1 = coff[cls + 1];
      if (f1 < 0) {
        add(d.B, 1);
      } else if (e1[t * d.ncm + cls]) {
        const int q1 = d.cls_q[b0];
        if (q == q1) {
          for (int j = b0 + 1; j < b1; ++j) add(cnode(t, d.cls_q[j]), 0);
        } else {
          add(cnode(t, q1), 0);
        }
      } else {
        for (int j = b0; j < b1; ++j)
          if (d.cls_q[j] != q) add(cnode(t, d.cls_q[j]), 2);
      }
    }
  } else {
    for (int t = 0; t < d.T; ++t)
      for (int cls = 0; cls < d.n_cls[c]; ++cls) {
        const int f1 = d.cls_f[(c * d.ncm + cls) * 2];
        const int b0 = coff[cls], b1 = coff[cls + 1];
        if (f1 < 0) {
          for (int j = b0; j < b1; ++j)
            if (cf[d.cls_q[j]] >= 0) add(cnode(t, d.cls_q[j]), 1);
        } else if (e1[t * d.ncm + cls]) {
          const int q1 = d.cls_q[b0];
          if (cf[q1] < 0)
            for (int j = b0 + 1; j < b1; ++j) add(cnode(t, d.cls_q[j]), 0);
          for (int j = b0 + 1; j < b1; ++j)
            if (cf[d.cls_q[j]] < 0) add(cnode(t, q1), 0);
        } else {
          for (int i = b0; i < b1; ++i)
            for (int j = i + 1; j < b1; ++j) {
              int qi = d.cls_q[i], qj = d.cls_q[j];
              if (cf[qi] < 0) add(cnode(t, qj), 2);
              if (cf[qj] < 0) add(cnode(t, qi), 2);
            }
        }
      }
  }
  // insertion sort by id
  for (int i = 1; i < cnt; ++i) {
    int y = ny[i], w = nw[i], j = i - 1;
    while (j >= 0 && ny[j] > y) {
      ny[j + 1] = ny[j];
      nw[j + 1] = nw[j];
      --j;
    }
    ny[j + 1] = y;
    nw[j + 1] = w;
  }
  return cnt;
}

// (weight, hops) Dijkstra on the stage-2 graph; key = weight * 2^20 + hops.
__device__ void dijkstra2(const DecDev& d, int c, const uint8_t* e1, int src, int64_t* key,
                          uint8_t* done, int* ny, int* nw) {
  for (int x = 0; x < d.NN; ++x) {
    key[x] = INF64;
    done[x] = 0;
  }
  key[src] = 0;
  for (;;) {
    int u = -1;
    int64_t best = INF64;
    for (int x = 0; x < d.NN; ++x)
      if (!done[x] && key[x] < best) {
        best = key[x];
        u = x;
      }
    if (u < 0) break;
    done[u] = 1;
    int cnt = nbrs2(d, c, e1, u, ny, nw);
    for (int i = 0; i < cnt; ++i) {
      int64_t cand = best + ((int64_t)nw[i] << 20) + 1;
      if (cand < key[ny[i]]) key[ny[i]] = cand;
    }
  }
}

__global__ void k_decode(DecDev d, int nb, const uint8_t* records, uint8_t* fail, int32_t* color_out,
                         int64_t* score_out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nb) return;
  const uint8_t* rec = records + (int64_t)s * d.n_rec;
  const int P = d.P, T = d.T, C = d.C, NN = d.NN;
  int64_t* f = d.dp_f + (int64_t)s * d.dp_stride;
  int8_t* ch = d.dp_c + (int64_t)s * d.dp_stride;
  int64_t* dist2 = d.dist2 + (int64_t)s * d.d2_stride;
  uint8_t* e1 = d.e1 + (int64_t)s * d.e1_stride;
  uint8_t* resid = d.resid + (int64_t)s * (2 * NN);
  uint8_t* done = resid + NN;
  int ny[256], nw[256];
  int* defs = d.defs + (int64_t)s * 4 * KMAX;
  int* partner = defs + KMAX;
  int* comp = defs + 2 * KMAX;
  int* loc = defs + 3 * KMAX;
  int64_t* Wb = d.wb + (int64_t)s * KMAX;
  void* bl = d.bls + (int64_t)s * d.bl_stride;
  // detectors into resid scratch temporarily: Dbit(t, p)
  auto Dbit = [&](int t, int p) -> int {
    int cur = t < C ? rec[t * 2 * P + 2 * p] : 0;
    if (t == C) {
      int par = 0;
      for (int i = d.support_off[p]; i < d.support_off[p + 1]; ++i) par ^= rec[C * 2 * P + d.support[i]];
      cur = par;
    }
    int prev = t > 0 ? rec[(t - 1) * 2 * P + 2 * p] : 0;
    return cur ^ prev;
  };
  int best_c = -1, best_par = 0;
  int64_t best_score = INF64;
  bool over = false;
  for (int c = 0; c < 3 && !over; ++c) {
    // ---------------- stage 1
    int k = 0;
    for (int t = 0; t < T && !over; ++t)
      for (int p = 0; p < P; ++p)
        if (d.color[p] != c && Dbit(t, p)) {
          if (k == KMAX) {
            over = true;
            break;
          }
          defs[k++] = t * P + p;
        }
    if (over) break;
    const int32_t* D1 = d.dist1 + (size_t)c * NN * NN;
    for (int i = 0; i < k; ++i) {
      int a = defs[i];
      int db = D1[(size_t)a * NN + d.B];
      Wb[i] = db < 0 ? -1 : (int64_t)db * WUNIT + (int64_t)pair_hash(a, d.B, 0, c);
    }
    auto w1 = [&](int i, int j) -> int64_t {
      const int dd = D1[(size_t)defs[i] * NN + defs[j]];
      return dd < 0 ? -1 : (int64_t)dd * WUNIT + (int64_t)pair_hash(defs[i], defs[j], 0, c);
    };
    int64_t tot1 = mwpm_exact(k, w1, Wb, f, ch, partner, comp, loc, bl);
    if (tot1 < 0) {
      if (tot1 == -2) atomicAdd(d.overflow + 1, 1);
      over = true;
      break;
    }
    for (int i = 0; i < T * d.ncm + T * P; ++i) e1[i] = 0;
    const int* aoff = d.adj1_off + c * (NN + 1);
    for (int i = 0; i < k; ++i) {
      int j = partner[i];
      if (j >= 0 && j < i) continue;
      int a = defs[i], b = j < 0 ? d.B : defs[j];
      int src = min(a, b), dst = max(a, b);
      int u = src;
      while (u != dst) {
        int du = D1[(size_t)u * NN + dst];
        int w = -1;
        for (int e = aoff[u]; e < aoff[u + 1]; ++e) {
          int x = d.adj1[e];
          if (D1[(size_t)x * NN + dst] == du - 1) {
            w = x;
            break;
          }
        }
        if (w < 0) {
          atomicAdd(d.overflow + 1, 1);
          break;
        }
        e1[edge_id1(d, c, u, w)] ^= 1;
        u = w;
      }
    }
    // ---------------- stage 2
    int par = 0;
    for (int x = 0; x < NN; ++x) resid[x] = 0;
    for (int t = 0; t < T; ++t)
      for (int g = 0; g < P; ++g)
        if (d.color[g] == c) resid[t * P + g] = (uint8_t)Dbit(t, g);
    const int* coff = d.cls_off + c * (d.ncm + 1);
    const int* cf = d.cface + c * d.n;
    for (int t = 0; t < T; ++t)
      for (int cls = 0; cls < d.n_cls[c]; ++cls)
        if (d.cls_f[(c * d.ncm + cls) * 2] >= 0 && e1[t * d.ncm + cls]) {
          int q1 = d.cls_q[coff[cls]];
          par ^= 1;
          if (cf[q1] >= 0) resid[t * P + cf[q1]] ^= 1;
        }
    int k2 = 0;
    for (int x = 0; x < d.B; ++x)
      if (resid[x]) {
        if (k2 == KMAX) {
          over = true;
          break;
        }
        defs[k2++] = x;
      }
    if (over) break;
    for (int i = 0; i <= k2; ++i) {
      int srcn = i < k2 ? defs[i] : d.B;
      dijkstra2(d, c, e1, srcn, dist2 + (size_t)i * NN, done, ny, nw);
    }
    for (int i = 0; i < k2; ++i) {
      int a = defs[i];
      int64_t kb = dist2[(size_t)i * NN + d.B];
      Wb[i] = kb >= INF64 ? -1 : (kb >> 20) * WUNIT + (int64_t)pair_hash(a, d.B, 1, c);
    }
    auto w2 = [&](int i, int j) -> int64_t {
      const int64_t kk = dist2[(size_t)i * NN + defs[j]];
      return kk >= INF64 ? -1 : (kk >> 20) * WUNIT + (int64_t)pair_hash(defs[i], defs[j], 1, c);
    };
    int64_t tot2 = mwpm_exact(k2, w2, Wb, f, ch, partner, comp, loc, bl);
    if (tot2 < 0) {
      if (tot2 == -2) atomicAdd(d.overflow + 1, 1);
      over = true;
      break;
    }
    for (int i = 0; i < k2; ++i) {
      int j = partner[i];
      if (j >= 0 && j < i) continue;
      int a = defs[i], b = j < 0 ? d.B : defs[j];
      int src = min(a, b), dst = max(a, b);
      const int64_t* kd = dist2 + (size_t)(dst == d.B ? k2 : (j < 0 ? i : (dst == a ? i : j))) * NN;
      int u = src;
      while (u != dst) {
        int64_t du = kd[u];
        int cnt = nbrs2(d, c, e1, u, ny, nw);
        int v = -1, ew = 0;
        for (int e = 0; e < cnt; ++e) {
          int64_t dv = kd[ny[e]];
          if (dv < INF64 && dv + ((int64_t)nw[e] << 20) + 1 == du) {
            v = ny[e];
            ew = nw[e];
            break;
          }
        }
        if (v < 0) {
          atomicAdd(d.overflow + 1, 1);
          break;
        }
        if (ew == 1 && (u == d.B || v == d.B)) par ^= 1;
        u = v;
      }
    }
    int64_t score = (tot1 / WUNIT) + (tot2 / WUNIT);
    if (score < best_score) {
      best_score = score;
      best_c = c;
      best_par = par;
    }
  }
  if (over) {
    atomicAdd(d.overflow, 1);
    fail[s] = 2;
    if (color_out) color_out[s] = -1;
    if (score_out) score_out[s] = -1;
    return;
  }
  int dpar = 0;
  for (int q = 0; q < d.n; ++q) dpar ^= rec[C * 2 * P + q];
  fail[s] = (uint8_t)(dpar ^ best_par);
  if (color_out) color_out[s] = best_c;
  if (score_out) score_out[s] = best_score;
}

#define CKD(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #call);    \
      return TTN_ECUDA;                                                            \
    }                                                                              \
  } while (0)

template <typename X>
static cudaError_t upload(const std::vector<X>& v, const X** dptr, std::vector<void*>& owned) {
  X* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(X) * std::max<size_t>(1, v.size()));
  if (e != cudaSuccess) return e;
  owned.push_back(p);
  if (!v.empty()) e = cudaMemcpy(p, v.data(), sizeof(X) * v.size(), cudaMemcpyHostToDevice);
  *dptr = p;
  return e;
}

ttn_status decode_device(const ttn_circuit& c, int nb, const uint8_t* d_records, uint8_t* fail,
                         int32_t* color, int64_t* score, void* stream, bool on_device) {
  const DecoderTables& t = c.dec;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<void*> owned;
  auto cleanup = [&]() {
    for (void* p : owned) cudaFree(p);
  };
  DecDev d{};
  d.T = t.T;
  d.P = t.P;
  d.B = t.B;
  d.NN = t.n_nodes;
  d.n = t.n;
  d.n_rec = c.n_rec;
  d.C = c.C;
  d.ncm = t.n_cls_max;
  // class lookup and c-face incidences
  std::vector<int32_t> clsof((size_t)3 * t.P * (t.P + 1), -1);
  std::vector<int32_t> inc_off(3 * (t.P + 1), 0), inc;
  for (int cc = 0; cc < 3; ++cc) {
    for (int i = 0; i < t.n_cls[cc]; ++i) {
      int f1 = t.cls_f[(cc * t.n_cls_max + i) * 2], f2 = t.cls_f[(cc * t.n_cls_max + i) * 2 + 1];
      if (f1 >= 0) clsof[((size_t)cc * t.P + f1) * (t.P + 1) + (f2 < 0 ? t.P : f2)] = i;
    }
    std::vector<std::vector<int>> per(t.P);
    for (int i = 0; i < t.n_cls[cc]; ++i)
      for (int j = t.cls_off[cc * (t.n_cls_max + 1) + i]; j < t.cls_off[cc * (t.n_cls_max + 1) + i + 1]; ++j) {
        int q = t.cls_q[j];
        int g = t.cface[cc * t.n + q];
        if (g >= 0) {
          per[g].push_back(i);
          per[g].push_back(q);
        }
      }
    for (int g = 0; g < t.P; ++g) {
      inc_off[cc * (t.P + 1) + g] = (int)inc.size() / 2;
      for (int x : per[g]) inc.push_back(x);
    }
    inc_off[cc * (t.P + 1) + t.P] = (int)inc.size() / 2;
  }
#define UP(vec, field)                                          \
  do {                                                          \
    cudaError_t e_ = upload(vec, &d.field, owned);              \
    if (e_ != cudaSuccess) {                                    \
      cleanup();                                                \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_)); \
      return TTN_ECUDA;                                         \
    }                                                           \
  } while (0)
  UP(t.color, color);
  UP(t.support_off, support_off);
  UP(t.support, support);
  UP(t.dist1, dist1);
  UP(t.adj1_off, adj1_off);
  UP(t.adj1, adj1);
  UP(t.cls_off, cls_off);
  UP(t.cls_q, cls_q);
  UP(t.cls_f, cls_f);
  UP(t.n_cls, n_cls);
  UP(clsof, clsof);
  UP(t.cface, cface);
  UP(inc_off, inc_off);
  UP(inc, inc);
#undef UP
  d.dp_stride = (size_t)1 << KCOMP;
  d.bl_stride = (boundary_matching_scratch_bytes(KMAX) + 255) / 256 * 256;
  d.d2_stride = (size_t)(KMAX + 1) * t.n_nodes;
  d.e1_stride = (size_t)t.T * t.n_cls_max + (size_t)t.T * t.P;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
    owned.push_back(*p);
    return true;
  };
  const int chunk = std::min(nb, 1024);
  bool ok = alloc((void**)&d.dp_f, sizeof(int64_t) * d.dp_stride * chunk) &&
            alloc((void**)&d.dp_c, d.dp_stride * chunk) &&
            alloc((void**)&d.dist2, sizeof(int64_t) * d.d2_stride * chunk) &&
            alloc((void**)&d.e1, d.e1_stride * chunk) &&
            alloc((void**)&d.resid, (size_t)2 * t.n_nodes * chunk) &&
            alloc((void**)&d.defs, sizeof(int) * 4 * KMAX * chunk) &&
            alloc((void**)&d.wb, sizeof(int64_t) * KMAX * chunk) &&
            alloc((void**)&d.bls, d.bl_stride * chunk) &&
            alloc((void**)&d.overflow, 2 * sizeof(int32_t));
  if (!ok) {
    cleanup();
    set_error("decoder scratch allocation failed");
    return TTN_ENOMEM;
  }
  CKD(cudaMemsetAsync(d.overflow, 0, 2 * sizeof(int32_t), st));
  uint8_t* dfail = nullptr;
  int32_t* dcol = nullptr;
  int64_t* dscore = nullptr;
  if (on_device) {
    dfail = fail;
    dcol = color;
    dscore = score;
  } else {
    if (!alloc((void**)&dfail, nb) || !alloc((void**)&dcol, sizeof(int32_t) * nb) ||
        !alloc((void**)&dscore, sizeof(int64_t) * nb)) {
      cleanup();
      set_error("decoder output allocation failed");
      return TTN_ENOMEM;
    }
  }
  for (int s0 = 0; s0 < nb; s0 += chunk) {
    int m = std::min(chunk, nb - s0);
    k_decode<<<(m + 63) / 64, 64, 0, st>>>(d, m, d_records + (size_t)s0 * c.n_rec, dfail + s0,
                                           dcol ? dcol + s0 : nullptr, dscore ? dscore + s0 : nullptr);
    if (profile().active) profile().kernels += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      cleanup();
      set_error(std::string("CUDA: decode launch: ") + cudaGetErrorString(e));
      return TTN_ECUDA;
    }
  }
  int32_t ovf[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(ovf, d.overflow, sizeof(ovf), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(fail, dfail, nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && color) e = cudaMemcpyAsync(color, dcol, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && score) e = cudaMemcpyAsync(score, dscore, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    set_error(std::string("CUDA: decode: ") + cudaGetErrorString(e));
    return TTN_ECUDA;
  }
  if (ovf[0] > 0) {
    set_error("decoder: " + std::to_string(ovf[0]) + " shot(s) exceed " + std::to_string(KMAX) +
              " defects per matching instance (fail byte set to 2)");
    return TTN_EOVERFLOW;
  }
  if (ovf[1] > 0) {
    set_error("decoder: canonical path or perfect matching not found");
    return TTN_ECUDA;
  }
  return TTN_OK;
}

// ------------------------------------------------------------------ allocation-free decoding
// ttn_decode_noalloc serves callers that must not allocate device memory: an
// application whose memory pool or caching allocator already owns the GPU
// memory, or a host framework whose allocator hooks forbid direct driver
// allocations.  It runs the same decoder kernel, but its tables and per-shot
// scratch live in file-scope static device arrays instead of cudaMalloc'ed
// buffers.  Every GPU that loads the library holds these arrays (about 2 MB)
// until the process exits.  Every call resolves the arrays' device addresses
// on the current device (cudaGetSymbolAddress allocates nothing, and a
// device reset between calls leaves no stale address); the first call on a
// device may also load the module, so make it before any stream capture.
// The first call with a given circuit packs its decoder tables into one host
// array kept with the circuit.  Each call copies that array to the device,
// decodes NA_SHOTS shots per launch (one thread per shot), reads back two
// overflow counters and synchronises its stream.
//
// Limits: at most NA_NODES detector nodes ((rounds + 1) * #faces + 1 <= 145,
// e.g. d = 7 with up to 7 rounds) and NA_TABLE_INTS packed table entries; any
// number of shots, decoded NA_SHOTS at a time, so n shots take ceil(n / 8)
// serial launches.  All calls share the arrays: calls that overlap on the GPU
// (different streams or host threads without ordering) race and corrupt each
// other's results.
static constexpr int NA_SHOTS = 8;
static constexpr int NA_NODES = 145;
static constexpr int NA_TABLE_INTS = 80000;
static constexpr size_t NA_E1_BYTES = 2048;
static constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
static constexpr size_t NA_DPF = na_align(sizeof(int64_t) << KCOMP);
static constexpr size_t NA_DPC = na_align((size_t)1 << KCOMP);
static constexpr size_t NA_D2 = na_align(sizeof(int64_t) * (KMAX + 1) * NA_NODES);
static constexpr size_t NA_E1 = na_align(NA_E1_BYTES);
static constexpr size_t NA_RES = na_align(2 * NA_NODES);
static constexpr size_t NA_DEFS = na_align(sizeof(int) * 4 * KMAX);
static constexpr size_t NA_WB = na_align(sizeof(int64_t) * KMAX);
static constexpr size_t NA_BL = na_align(boundary_matching_scratch_bytes(KMAX));
static constexpr size_t NA_PER_SHOT = NA_DPF + NA_DPC + NA_D2 + NA_E1 + NA_RES + NA_DEFS + NA_WB + NA_BL;
static constexpr size_t NA_SCRATCH_BYTES = NA_PER_SHOT * NA_SHOTS + 256;

static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];
static __device__ __align__(256) int32_t g_na_tables[NA_TABLE_INTS];

DecoderBlob build_decoder_blob(const DecoderTables& t) {
  DecoderBlob b;
  std::vector<int32_t> clsof((size_t)3 * t.P * (t.P + 1), -1);
  std::vector<int32_t> inc_off(3 * (t.P + 1), 0), inc;
  for (int cc = 0; cc < 3; ++cc) {
    for (int i = 0; i < t.n_cls[cc]; ++i) {
      int f1 = t.cls_f[(cc * t.n_cls_max + i) * 2], f2 = t.cls_f[(cc * t.n_cls_max + i) * 2 + 1];
      if (f1 >= 0) clsof[((size_t)cc * t.P + f1) * (t.P + 1) + (f2 < 0 ? t.P : f2)] = i;
    }
    std::vector<std::vector<int>> per(t.P);
    for (int i = 0; i < t.n_cls[cc]; ++i)
      for (int j = t.cls_off[cc * (t.n_cls_max + 1) + i]; j < t.cls_off[cc * (t.n_cls_max + 1) + i + 1]; ++j) {
        int q = t.cls_q[j];
        int g = t.cface[cc * t.n + q];
        if (g >= 0) {
          per[g].push_back(i);
          per[g].push_back(q);
        }
      }
    for (int g = 0; g < t.P; ++g) {
      inc_off[cc * (t.P + 1) + g] = (int)inc.size() / 2;
      for (int x : per[g]) inc.push_back(x);
    }
    inc_off[cc * (t.P + 1) + t.P] = (int)inc.size() / 2;
  }
  const std::vector<int32_t>* parts[14] = {&t.color, &t.support_off, &t.support, &t.dist1, &t.adj1_off,
                                           &t.adj1, &t.cls_off, &t.cls_q, &t.cls_f, &t.n_cls,
                                           &clsof, &t.cface, &inc_off, &inc};
  for (int i = 0; i < 14; ++i) {
    b.off[i] = (int32_t)b.data.size();
    b.data.insert(b.data.end(), parts[i]->begin(), parts[i]->end());
    while (b.data.size() % 4) b.data.push_back(0);  // 16-byte aligned parts
  }
  b.off[14] = (int32_t)b.data.size();
  return b;
}

// Device addresses of the static arrays on the current device.  Resolved on
// every call: cudaGetSymbolAddress allocates nothing, and caching the
// addresses would leave them stale after a device reset.
static std::mutex g_na_mutex;

static ttn_status na_setup(unsigned char** scratch, int32_t** tables) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess) {
    set_error(std::string("CUDA: cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    return TTN_ECUDA;
  }
  void* q = nullptr;
  e = cudaGetSymbolAddress(&q, g_na_tables);
  if (e != cudaSuccess) {
    set_error(std::string("CUDA: cudaGetSymbolAddress(tables): ") + cudaGetErrorString(e));
    return TTN_ECUDA;
  }
  *scratch = (unsigned char*)p;
  *tables = (int32_t*)q;
  return TTN_OK;
}

ttn_status decode_noalloc(const ttn_circuit& c, uint64_t n, const uint8_t* d_records, uint8_t* d_fail,
                          int32_t* d_color, int64_t* d_score, void* stream) {
  const DecoderTables& t = c.dec;
  if (t.n_nodes > NA_NODES) {
    set_error("ttn_decode_noalloc: " + std::to_string(t.n_nodes) + " detector nodes; the static scratch holds " +
              std::to_string(NA_NODES) + " ((rounds + 1) * faces + 1)");
    return TTN_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!c.dec_blob_ready) {
      c.dec_blob = build_decoder_blob(t);
      c.dec_blob_ready = true;
    }
  }
  const DecoderBlob& blob = c.dec_blob;
  if ((int64_t)blob.data.size() > NA_TABLE_INTS ||
      (size_t)t.T * t.n_cls_max + (size_t)t.T * t.P > NA_E1_BYTES) {
    set_error("ttn_decode_noalloc: decoder tables exceed the static table size");
    return TTN_EINVAL;
  }
  unsigned char* scratch = nullptr;
  int32_t* tables = nullptr;
  ttn_status s = na_setup(&scratch, &tables);
  if (s != TTN_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(tables, blob.data.data(), sizeof(int32_t) * blob.data.size(),
                                  cudaMemcpyHostToDevice, st);
  DecDev d{};
  d.T = t.T;
  d.P = t.P;
  d.B = t.B;
  d.NN = t.n_nodes;
  d.n = t.n;
  d.n_rec = c.n_rec;
  d.C = c.C;
  d.ncm = t.n_cls_max;
  d.color = tables + blob.off[0];
  d.support_off = tables + blob.off[1];
  d.support = tables + blob.off[2];
  d.dist1 = tables + blob.off[3];
  d.adj1_off = tables + blob.off[4];
  d.adj1 = tables + blob.off[5];
  d.cls_off = tables + blob.off[6];
  d.cls_q = tables + blob.off[7];
  d.cls_f = tables + blob.off[8];
  d.n_cls = tables + blob.off[9];
  d.clsof = tables + blob.off[10];
  d.cface = tables + blob.off[11];
  d.inc_off = tables + blob.off[12];
  d.inc = tables + blob.off[13];
  // per-shot scratch regions, NA_SHOTS shots side by side
  unsigned char* base = scratch;
  d.dp_f = (int64_t*)base;
  base += NA_DPF * NA_SHOTS;
  d.dp_c = (int8_t*)base;
  base += NA_DPC * NA_SHOTS;
  d.dist2 = (int64_t*)base;
  base += NA_D2 * NA_SHOTS;
  d.e1 = base;
  base += NA_E1 * NA_SHOTS;
  d.resid = base;
  base += NA_RES * NA_SHOTS;
  d.defs = (int*)base;
  base += NA_DEFS * NA_SHOTS;
  d.wb = (int64_t*)base;
  base += NA_WB * NA_SHOTS;
  d.bls = base;
  base += NA_BL * NA_SHOTS;
  d.overflow = (int32_t*)base;  // the last 256 bytes
  d.dp_stride = NA_DPF / sizeof(int64_t);
  d.d2_stride = NA_D2 / sizeof(int64_t);
  d.e1_stride = NA_E1;
  d.bl_stride = NA_BL;
  // the overflow counters must start at zero; the rest is overwritten per shot
  if (e == cudaSuccess) e = cudaMemsetAsync(d.overflow, 0, 2 * sizeof(int32_t), st);
  for (uint64_t s0 = 0; s0 < n && e == cudaSuccess; s0 += NA_SHOTS) {
    const int m = (int)std::min<uint64_t>(NA_SHOTS, n - s0);
    k_decode<<<1, NA_SHOTS, 0, st>>>(d, m, d_records + s0 * c.n_rec, d_fail + s0,
                               d_color ? d_color + s0 : nullptr, d_score ? d_score + s0 : nullptr);
    e = cudaGetLastError();
  }
  int32_t ovf[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(ovf, d.overflow, sizeof(ovf), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("CUDA: ttn_decode_noalloc: ") + cudaGetErrorString(e));
    return TTN_ECUDA;
  }
  if (ovf[0] > 0) {
    set_error("decoder: " + std::to_string(ovf[0]) + " shot(s) exceed " + std::to_string(KMAX) +
              " defects per matching instance (fail byte set to 2)");
    return TTN_EOVERFLOW;
  }
  if (ovf[1] > 0) {
    set_error("decoder: canonical path or perfect matching not found");
    return TTN_ECUDA;
  }
  return TTN_OK;
}

}  // namespace ttn

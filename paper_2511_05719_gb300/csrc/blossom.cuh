// Exact maximum-weight perfect matching on a complete graph of at most
// BL_NMAX vertices by Edmonds' primal-dual blossom algorithm (Edmonds 1965;
// the O(n^3) organisation with least-slack edges per blossom of Gabow 1976
// and Galil, ACM Comput. Surv. 18 (1986)).  Vertices 0..n-1, non-trivial
// blossoms n..2n-1.  Weights are 64-bit integers given by a functor
// wt(u, v) (negative = no edge); slacks use doubled weights so that every
// dual stays integral.
//
// Single-threaded (one GPU thread per instance) and host-compilable, so the
// same code runs in host checks.  The sub-blossoms of a blossom form a linked
// cycle (cnext / cprev); the edge from child x to cnext[x] is (ex[x], ey[x])
// with ex[x] inside x; re-basing a blossom only moves cfirst[b].  No
// recursion: nested work uses explicit stacks inside the scratch.
#pragma once

#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define BL_HD __host__ __device__
#else
#define BL_HD
#endif

namespace ttn {

static constexpr int BL_NMAX = 256;

struct BlossomState {
  int n;
  int64_t* dual;   // [2n] doubled duals of vertices and blossoms
  int16_t* mate;   // [n] matched vertex or -1
  int16_t* inb;    // [n] top-level blossom of a vertex
  int16_t* freeb;  // [n] unused blossom ids
  int16_t* queue;  // [2n] S vertices to scan
  int16_t* label;  // [2n] 0 free, 1 S, 2 T (4: breadcrumb)
  int16_t* lfrom;  // [2n] label edge: vertex outside the (sub)blossom
  int16_t* lto;    // [2n] label edge: vertex inside it
  int16_t* par;    // [2n] parent blossom or -1
  int16_t* base;   // [2n] base vertex (-1: unused blossom id)
  int16_t* cfirst; // [2n] base child
  int16_t* cnext;  // [2n]
  int16_t* cprev;  // [2n]
  int16_t* ex;     // [2n]
  int16_t* ey;     // [2n]
  int16_t* bfrom;  // [2n] least-slack edge to an S vertex: end in this blossom
  int16_t* bto;    // [2n] and the S end
  int16_t* stack;  // [2n] traversal stack
  int16_t* path;   // [2n]
  int nfree, qh, qt;
};

BL_HD constexpr size_t bl_scratch_bytes(int n) {
  return (size_t)2 * n * sizeof(int64_t) + (size_t)3 * n * sizeof(int16_t) +
         (size_t)15 * 2 * n * sizeof(int16_t);
}

BL_HD inline void bl_bind(BlossomState& s, int n, void* scratch) {
  s.n = n;
  s.dual = (int64_t*)scratch;
  int16_t* p = (int16_t*)(s.dual + 2 * n);
  s.mate = p; p += n;
  s.inb = p; p += n;
  s.freeb = p; p += n;
  s.queue = p; p += 2 * n;
  s.label = p; p += 2 * n;
  s.lfrom = p; p += 2 * n;
  s.lto = p; p += 2 * n;
  s.par = p; p += 2 * n;
  s.base = p; p += 2 * n;
  s.cfirst = p; p += 2 * n;
  s.cnext = p; p += 2 * n;
  s.cprev = p; p += 2 * n;
  s.ex = p; p += 2 * n;
  s.ey = p; p += 2 * n;
  s.bfrom = p; p += 2 * n;
  s.bto = p; p += 2 * n;
  s.stack = p; p += 2 * n;
  s.path = p; p += 2 * n;
}

template <typename WT>
struct Blossom {
  BlossomState& s;
  WT wt;

  BL_HD int64_t slack(int u, int v) const { return s.dual[u] + s.dual[v] - 2 * wt(u, v); }

  // vertices of (sub)blossom b, written to out; returns their number
  BL_HD int leaves(int b, int16_t* out) const {
    int top = 0, m = 0;
    s.stack[top++] = (int16_t)b;
    while (top) {
      const int x = s.stack[--top];
      if (x < s.n) {
        out[m++] = (int16_t)x;
        continue;
      }
      int c = s.cfirst[x];
      do {
        s.stack[top++] = (int16_t)c;
        c = s.cnext[c];
      } while (c != s.cfirst[x]);
    }
    return m;
  }

  BL_HD void push_leaves(int b) {
    int top = 0;
    s.stack[top++] = (int16_t)b;
    while (top) {
      const int x = s.stack[--top];
      if (x < s.n) {
        s.queue[s.qt++] = (int16_t)x;
        continue;
      }
      int c = s.cfirst[x];
      do {
        s.stack[top++] = (int16_t)c;
        c = s.cnext[c];
      } while (c != s.cfirst[x]);
    }
  }

  // position of child t in the cycle of b, counted from the base child
  BL_HD int index_of(int b, int t) const {
    int i = 0, c = s.cfirst[b];
    while (c != t) {
      c = s.cnext[c];
      ++i;
    }
    return i;
  }

  BL_HD int child_of(int b, int v) const {
    int t = v;
    while (s.par[t] != b) t = s.par[t];
    return t;
  }

  // Label the top-level blossom of w with t (1 = S, 2 = T) via edge (p, w);
  // a T blossom passes S on to the mate of its base.
  BL_HD void assign_label(int w, int t, int p) {
    for (;;) {
      const int b = s.inb[w];
      s.label[w] = s.label[b] = (int16_t)t;
      s.lfrom[w] = s.lfrom[b] = (int16_t)p;
      s.lto[w] = s.lto[b] = (int16_t)w;
      s.bfrom[w] = s.bfrom[b] = -1;
      if (t == 1) {
        push_leaves(b);
        return;
      }
      const int bs = s.base[b];
      w = s.mate[bs];
      t = 1;
      p = bs;
    }
  }

  // Walk both trees towards their roots; a shared blossom is the base of a
  // new blossom (returned), otherwise the path augments (-1).
  BL_HD int scan_blossom(int v, int w) {
    int np = 0, found = -1;
    while (v != -1 || w != -1) {
      if (v != -1) {
        int b = s.inb[v];
        if (s.label[b] & 4) {
          found = s.base[b];
          break;
        }
        s.path[np++] = (int16_t)b;
        s.label[b] = 5;
        if (s.lfrom[b] == -1) {
          v = -1;  // root
        } else {
          v = s.lfrom[b];
          b = s.inb[v];  // T blossom
          v = s.lfrom[b];
        }
      }
      if (w != -1) {
        const int t = v;
        v = w;
        w = t;
      }
    }
    for (int i = 0; i < np; ++i) s.label[s.path[i]] = 1;
    return found;
  }

  // least-slack edge from blossom b (its leaves) to any S vertex outside it
  BL_HD void best_edge_of(int b) {
    int16_t* lv = s.path;
    const int m = leaves(b, lv);
    int64_t best = 0;
    int bf = -1, bt = -1;
    for (int i = 0; i < m; ++i) {
      const int v = lv[i];
      for (int u = 0; u < s.n; ++u) {
        if (s.inb[u] == b || s.label[s.inb[u]] != 1) continue;
        if (wt(v, u) < 0) continue;
        const int64_t k = slack(v, u);
        if (bf == -1 || k < best) {
          best = k;
          bf = v;
          bt = u;
        }
      }
    }
    s.bfrom[b] = (int16_t)bf;
    s.bto[b] = (int16_t)bt;
  }

  BL_HD void add_blossom(int base_v, int v, int w) {
    const int bb = s.inb[base_v];
    int bv = s.inb[v], bw = s.inb[w];
    const int b = s.freeb[--s.nfree];
    s.base[b] = s.base[bb];
    s.par[b] = -1;
    s.par[bb] = (int16_t)b;
    // cycle: bb, down the v side to inb[v], edge (v, w), inb[w], up to bb
    int np = 0;
    while (bv != bb) {
      s.par[bv] = (int16_t)b;
      s.path[np++] = (int16_t)bv;
      bv = s.inb[s.lfrom[bv]];
    }
    int prev = bb;
    for (int i = np - 1; i >= 0; --i) {
      const int c = s.path[i];
      s.cnext[prev] = (int16_t)c;
      s.cprev[c] = (int16_t)prev;
      s.ex[prev] = s.lfrom[c];
      s.ey[prev] = s.lto[c];
      prev = c;
    }
    s.cnext[prev] = (int16_t)bw;
    s.cprev[bw] = (int16_t)prev;
    s.ex[prev] = (int16_t)v;
    s.ey[prev] = (int16_t)w;
    while (bw != bb) {
      s.par[bw] = (int16_t)b;
      const int up = s.inb[s.lfrom[bw]];
      s.cnext[bw] = (int16_t)up;
      s.cprev[up] = (int16_t)bw;
      s.ex[bw] = s.lto[bw];
      s.ey[bw] = s.lfrom[bw];
      bw = up;
    }
    s.cfirst[b] = (int16_t)bb;
    s.label[b] = 1;
    s.lfrom[b] = s.lfrom[bb];
    s.lto[b] = s.lto[bb];
    s.dual[b] = 0;
    // vertices of former T sub-blossoms become S and are scanned
    int16_t* lv = s.path;
    const int m = leaves(b, lv);
    for (int i = 0; i < m; ++i) {
      const int x = lv[i];
      if (s.label[s.inb[x]] == 2) s.queue[s.qt++] = (int16_t)x;
      s.inb[x] = (int16_t)b;
    }
    int c = bb;
    do {
      s.bfrom[c] = -1;
      c = s.cnext[c];
    } while (c != bb);
    best_edge_of(b);
  }

  BL_HD void free_blossom(int b) {
    s.label[b] = 0;
    s.lfrom[b] = s.lto[b] = -1;
    s.par[b] = -1;
    s.base[b] = -1;
    s.bfrom[b] = -1;
    s.freeb[s.nfree++] = (int16_t)b;
  }

  // the children of b become top-level
  BL_HD void release_children(int b) {
    int c = s.cfirst[b];
    do {
      s.par[c] = -1;
      if (c < s.n) {
        s.inb[c] = (int16_t)c;
      } else {
        int16_t* lv = s.path;
        const int m = leaves(c, lv);
        for (int i = 0; i < m; ++i) s.inb[lv[i]] = (int16_t)c;
      }
      c = s.cnext[c];
    } while (c != s.cfirst[b]);
  }

  // End of a stage: expand b and, transitively, every child blossom with
  // zero dual (the queue is free here and serves as the stack).
  BL_HD void expand_endstage(int b0) {
    int top = 0;
    s.queue[top++] = (int16_t)b0;
    while (top) {
      const int b = s.queue[--top];
      release_children(b);
      int c = s.cfirst[b];
      do {
        if (c >= s.n && s.dual[c] == 0) s.queue[top++] = (int16_t)c;
        c = s.cnext[c];
      } while (c != s.cfirst[b]);
      free_blossom(b);
    }
  }

  // Mid-stage expansion of a T blossom whose dual reached zero: the even
  // path from the entry child to the base child keeps alternating T / S
  // labels, the other children are free unless one of their vertices was
  // reached by a tight edge.
  BL_HD void expand_blossom(int b) {
    release_children(b);
    const int c0 = s.cfirst[b];
    const int entry = s.inb[s.lto[b]];
    const bool fwd = (index_of(b, entry) & 1) != 0;
    int pf = s.lfrom[b], pt = s.lto[b];
    int cur = entry;
    while (cur != c0) {
      s.label[pt] = 0;
      const int nb1 = fwd ? s.cnext[cur] : s.cprev[cur];  // becomes S (mate)
      s.label[nb1] = 0;
      assign_label(pt, 2, pf);
      int nxt;
      if (fwd) {
        pf = s.ex[nb1];
        pt = s.ey[nb1];
        nxt = s.cnext[nb1];
      } else {
        nxt = s.cprev[nb1];
        pf = s.ey[nxt];
        pt = s.ex[nxt];
      }
      cur = nxt;
    }
    // base child: T without passing S to its mate (already S outside)
    s.label[c0] = s.label[pt] = 2;
    s.lfrom[c0] = s.lfrom[pt] = (int16_t)pf;
    s.lto[c0] = s.lto[pt] = (int16_t)pt;
    s.bfrom[c0] = -1;
    int x = fwd ? s.cnext[c0] : s.cprev[c0];
    while (x != entry) {
      if (s.label[x] != 1) {
        int16_t* lv = s.path;
        const int m = leaves(x, lv);
        int hit = -1;
        for (int i = 0; i < m; ++i)
          if (s.label[lv[i]] != 0) {
            hit = lv[i];
            break;
          }
        if (hit >= 0) {
          s.label[hit] = 0;
          s.label[s.mate[s.base[x]]] = 0;
          assign_label(hit, 2, s.lfrom[hit]);
        }
      }
      x = fwd ? s.cnext[x] : s.cprev[x];
    }
    free_blossom(b);
  }

  // Re-base blossom b at vertex v: flip the matched edges on the even path
  // from v's child to the old base child, recursively inside sub-blossoms
  // (explicit stack of (blossom, vertex) frames; frames touch disjoint
  // sub-blossoms, so their order does not matter).
  BL_HD void augment_blossom(int b, int v) {
    int16_t* fb = s.stack;
    int16_t* fv = s.stack + s.n;
    int top = 0;
    fb[top] = (int16_t)b;
    fv[top] = (int16_t)v;
    ++top;
    while (top) {
      --top;
      const int bb = fb[top], vv = fv[top];
      const int t = child_of(bb, vv);
      if (t >= s.n) {
        fb[top] = (int16_t)t;
        fv[top] = (int16_t)vv;
        ++top;
      }
      const int i = index_of(bb, t);
      const int c0 = s.cfirst[bb];
      int cur = t;
      if (i & 1) {  // forward to the base child
        while (cur != c0) {
          const int a = s.cnext[cur];
          const int x = s.ex[a], y = s.ey[a];  // x in a, y in cnext[a]
          const int nb2 = s.cnext[a];
          if (a >= s.n) {
            fb[top] = (int16_t)a;
            fv[top] = (int16_t)x;
            ++top;
          }
          if (nb2 >= s.n) {
            fb[top] = (int16_t)nb2;
            fv[top] = (int16_t)y;
            ++top;
          }
          s.mate[x] = (int16_t)y;
          s.mate[y] = (int16_t)x;
          cur = nb2;
        }
      } else {  // backward to the base child
        while (cur != c0) {
          const int a = s.cprev[cur];
          const int p = s.cprev[a];
          const int x = s.ex[p], y = s.ey[p];  // x in p, y in a
          if (p >= s.n) {
            fb[top] = (int16_t)p;
            fv[top] = (int16_t)x;
            ++top;
          }
          if (a >= s.n) {
            fb[top] = (int16_t)a;
            fv[top] = (int16_t)y;
            ++top;
          }
          s.mate[x] = (int16_t)y;
          s.mate[y] = (int16_t)x;
          cur = p;
        }
      }
      s.cfirst[bb] = (int16_t)t;
      s.base[bb] = (int16_t)vv;
    }
  }

  // Augment along the path through the tight S-S edge (v, w).
  BL_HD void augment(int v, int w) {
    for (int side = 0; side < 2; ++side) {
      int sv = side == 0 ? v : w, p = side == 0 ? w : v;
      for (;;) {
        const int bs = s.inb[sv];
        if (bs >= s.n) augment_blossom(bs, sv);
        s.mate[sv] = (int16_t)p;
        if (s.lfrom[bs] == -1) break;
        const int t = s.lfrom[bs];
        const int bt = s.inb[t];
        const int ns = s.lfrom[bt], j = s.lto[bt];
        if (bt >= s.n) augment_blossom(bt, j);
        s.mate[j] = (int16_t)ns;
        sv = ns;
        p = j;
      }
    }
  }

  // Maximum-weight perfect matching; false when none exists.
  BL_HD bool solve() {
    const int n = s.n;
    int64_t wmax = 0;
    for (int u = 0; u < n; ++u)
      for (int v = u + 1; v < n; ++v) {
        const int64_t w = wt(u, v);
        if (w > wmax) wmax = w;
      }
    for (int u = 0; u < n; ++u) {
      s.mate[u] = -1;
      s.inb[u] = (int16_t)u;
      s.dual[u] = wmax;
    }
    for (int x = 0; x < 2 * n; ++x) {
      s.par[x] = -1;
      s.base[x] = x < n ? (int16_t)x : (int16_t)-1;
      s.label[x] = 0;
      s.lfrom[x] = s.lto[x] = -1;
      s.bfrom[x] = -1;
      if (x >= n) s.dual[x] = 0;
    }
    s.nfree = 0;
    for (int b = 2 * n - 1; b >= n; --b) s.freeb[s.nfree++] = (int16_t)b;
    for (int stage = 0; stage < n; ++stage) {
      int nfreev = 0;
      for (int v = 0; v < n; ++v) nfreev += s.mate[v] == -1;
      if (nfreev == 0) break;
      for (int x = 0; x < 2 * n; ++x) {
        s.label[x] = 0;
        s.bfrom[x] = -1;
      }
      s.qh = s.qt = 0;
      for (int v = 0; v < n; ++v)
        if (s.mate[v] == -1 && s.label[s.inb[v]] == 0) assign_label(v, 1, -1);
      bool augmented = false;
      for (;;) {
        while (s.qh < s.qt && !augmented) {
          const int v = s.queue[s.qh++];
          for (int w = 0; w < n; ++w) {
            if (w == v) continue;
            const int bv = s.inb[v], bw = s.inb[w];
            if (bv == bw || wt(v, w) < 0) continue;
            const int64_t k = slack(v, w);
            if (k <= 0) {
              if (s.label[bw] == 0) {
                assign_label(w, 2, v);
              } else if (s.label[bw] == 1) {
                const int bs = scan_blossom(v, w);
                if (bs >= 0) {
                  add_blossom(bs, v, w);
                } else {
                  augment(v, w);
                  augmented = true;
                  break;
                }
              } else if (s.label[w] == 0) {
                // inside a T blossom: remember how w was reached
                s.label[w] = 2;
                s.lfrom[w] = (int16_t)v;
                s.lto[w] = (int16_t)w;
              }
            } else if (s.label[bw] == 1) {
              if (s.bfrom[bv] == -1 || k < slack(s.bfrom[bv], s.bto[bv])) {
                s.bfrom[bv] = (int16_t)v;
                s.bto[bv] = (int16_t)w;
              }
            } else if (s.label[w] == 0) {
              if (s.bfrom[w] == -1 || k < slack(s.bfrom[w], s.bto[w])) {
                s.bfrom[w] = (int16_t)w;
                s.bto[w] = (int16_t)v;
              }
            }
          }
        }
        if (augmented) break;
        // dual update: the smallest step that makes an edge tight or a
        // T blossom's dual zero
        int dtype = -1, dvert = -1, dblos = -1;
        int64_t delta = 0;
        for (int v = 0; v < n; ++v)
          if (s.label[s.inb[v]] == 0 && s.bfrom[v] != -1) {
            const int64_t d = slack(s.bfrom[v], s.bto[v]);
            if (dtype == -1 || d < delta) {
              delta = d;
              dtype = 2;
              dvert = v;
            }
          }
        for (int b = 0; b < 2 * n; ++b)
          if (s.par[b] == -1 && s.label[b] == 1 && s.bfrom[b] != -1 && (b < n || s.base[b] >= 0)) {
            const int64_t d = slack(s.bfrom[b], s.bto[b]) / 2;
            if (dtype == -1 || d < delta) {
              delta = d;
              dtype = 3;
              dvert = b;
            }
          }
        for (int b = n; b < 2 * n; ++b)
          if (s.base[b] >= 0 && s.par[b] == -1 && s.label[b] == 2) {
            if (dtype == -1 || s.dual[b] < delta) {
              delta = s.dual[b];
              dtype = 4;
              dblos = b;
            }
          }
        if (dtype == -1) return false;  // no augmenting path
        for (int v = 0; v < n; ++v) {
          const int l = s.label[s.inb[v]];
          if (l == 1) s.dual[v] -= delta;
          else if (l == 2) s.dual[v] += delta;
        }
        for (int b = n; b < 2 * n; ++b)
          if (s.base[b] >= 0 && s.par[b] == -1) {
            if (s.label[b] == 1) s.dual[b] += delta;
            else if (s.label[b] == 2) s.dual[b] -= delta;
          }
        s.qh = s.qt = 0;  // the queue is empty here: reuse it from the start
        if (dtype == 2) {
          s.queue[s.qt++] = s.bto[dvert];  // the S end of the edge
        } else if (dtype == 3) {
          s.queue[s.qt++] = s.bfrom[dvert];
        } else {
          expand_blossom(dblos);
        }
      }
      for (int b = n; b < 2 * n; ++b)
        if (s.base[b] >= 0 && s.par[b] == -1 && s.label[b] == 1 && s.dual[b] == 0) expand_endstage(b);
    }
    for (int v = 0; v < n; ++v)
      if (s.mate[v] < 0) return false;
    return true;
  }
};

// Weights of the defect / boundary-copy graph: vertices 0..k-1 are defects,
// k..2k-1 their boundary copies.  Defect pairs carry wp(i, j), defect i and
// its own copy carry wb(i), copies pair with each other at weight 0.  The
// matching maximises top - w, so among perfect matchings it minimises w.
template <typename WP, typename WB>
struct BoundaryWeights {
  WP wp;
  WB wb;
  int k;
  int64_t top;
  BL_HD int64_t raw(int u, int v) const {
    if (u > v) {
      const int t = u;
      u = v;
      v = t;
    }
    if (v < k) return wp(u, v);
    if (u < k) return v == u + k ? wb(u) : -1;
    return 0;
  }
  BL_HD int64_t operator()(int u, int v) const {
    const int64_t r = raw(u, v);
    return r < 0 ? -1 : top - r;
  }
};

BL_HD constexpr size_t boundary_matching_scratch_bytes(int k) { return bl_scratch_bytes(2 * k); }

// Minimum-weight matching of k defects, each paired with another defect
// (wp(i, j) >= 0; negative = no such pair) or sent to the boundary
// (wb(i) >= 0; negative = impossible).  partner[i] = the other defect or -1
// (boundary).  Returns the total weight, -2 if no complete matching exists,
// -1 if 2k exceeds BL_NMAX.
template <typename WP, typename WB>
BL_HD int64_t min_matching_boundary(int k, WP wp, WB wb, int* partner, void* scratch) {
  if (k == 0) return 0;
  if (2 * k > BL_NMAX) return -1;
  BoundaryWeights<WP, WB> W{wp, wb, k, 0};
  int64_t mx = 0;
  for (int u = 0; u < 2 * k; ++u)
    for (int v = u + 1; v < 2 * k; ++v) {
      const int64_t r = W.raw(u, v);
      if (r > mx) mx = r;
    }
  W.top = mx + 1;
  BlossomState st;
  bl_bind(st, 2 * k, scratch);
  Blossom<BoundaryWeights<WP, WB>> B{st, W};
  if (!B.solve()) return -2;
  int64_t total = 0;
  for (int i = 0; i < k; ++i) {
    const int m = st.mate[i];
    if (m < k) {
      partner[i] = m;
      if (m > i) total += wp(i, m);
    } else {
      partner[i] = -1;
      total += wb(i);
    }
  }
  return total;
}

}  // namespace ttn

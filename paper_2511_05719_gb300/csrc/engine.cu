// Batched tree-tensor-network trajectory engine (sm_103a).
//
// Every trajectory of a batch runs the same step program (compiled on the
// host from the circuit and the tree layout); only bond dimensions, tensor
// values and random draws differ.  Kernels take the whole batch (grid.z or
// grid.x = trajectory), read each trajectory's bond dimensions from device
// memory and skip the tiles outside them, so no host synchronisation is
// needed between steps.
//
// Method (Sec. III.B-C): a binary TTN with the isometry centre moved by
// singular value decompositions; a two-qubit gate is applied in
// operator-Schmidt form along the tree path between its leaves and the path
// bonds are re-truncated to chi; measurements and amplitude-damping branches
// are sampled at the centre (Born rule / exact Kraus unravelling) with
// Philox4x32-10 draws keyed by (seed, trajectory, event).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "contract.h"
#include "gram.h"

namespace ttn {

// ------------------------------------------------------------------ complex
template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R x, y;
};

template <typename R>
__device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {  // conj(a) * b
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename R>
__device__ __forceinline__ cx<R> cscale(cx<R> a, R s) {
  return {a.x * s, a.y * s};
}
template <typename R>
__device__ __forceinline__ R cabs2(cx<R> a) {
  return a.x * a.x + a.y * a.y;
}

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 bit
// products, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform in [0, 1) with 53 random bits: counter (traj_lo, traj_hi, event, 0).
__device__ __forceinline__ double draw_uniform(uint64_t seed, uint64_t traj, uint32_t event) {
  uint4 w = philox10(make_uint4((uint32_t)traj, (uint32_t)(traj >> 32), event, 0u),
                     make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  return ((double)(w.x >> 5) * 67108864.0 + (double)(w.y >> 6)) * (1.0 / 9007199254740992.0);
}

__global__ void k_philox_uniforms(uint64_t seed, const uint64_t* trajs, int n_traj,
                                  const int32_t* events, int n_events, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_traj * n_events) return;
  int t = i / n_events, e = i % n_events;
  out[i] = draw_uniform(seed, trajs[t], (uint32_t)events[e]);
}

// ------------------------------------------------------------------ batch state
template <typename R>
struct Dev {
  cx<R>* T;              // node tensors, trajectory b at T + b * tstride + off[v]
  const int64_t* off;    // [L]
  const int64_t* ncap;   // [L] slot capacity of node v (elements)
  int64_t tstride;
  int32_t* dims;         // [B][2L] bond (x, parent(x)) dimension
  int ds;                // 2L
  cx<R>* W;              // [B][wstride] SVD / contraction workspace
  int64_t wstride;
  cx<R>* V;              // [B][vstride] right singular vectors (column-major n x n)
  cx<R>* Rm;             // [B][vstride] factor absorbed by the neighbour (k x n)
  cx<R>* G;              // [B][vstride] Gram matrix / V_k S_k^-1 (Gram path)
  cx<R>* Ts;             // [B][2 vstride] tridiagonal eigensolver scratch
  int64_t vstride;
  double* sv;            // [B][nmax]
  int32_t* perm;         // [B][nmax]
  int nmax;
  int32_t* knew;         // [B] kept rank of the last move
  int32_t* nold;         // [B] previous dimension of that bond
  double* logp;          // [B]
  double* disc;          // [B]
  int32_t* ties;         // [B]
  uint8_t* rec;          // [B][n_rec]
  int n_rec;
  uint8_t* last;         // [B][N] last measured value per qubit
  int N;
  const double* theta;   // [B]
  const double* gamma;   // [B]
  const uint64_t* traj;  // [B] trajectory index
  uint64_t seed;
  int L, chi, noise;
  double eps, tie_eps, tol;
  double eps_gram, tol_gram, tol_abs_gram;
  int svd_mode;
  int eig_smem_bytes;    // dynamic shared memory of k_eig launches
  unsigned long long* ledger;  // [LEDGER_WORDS] algorithmic flops, bytes, eigensolver phase cycles (or null)
  uint8_t* choice;       // [B][n_events] sampled outcome of every stochastic event
  int n_events;
  int forced;            // 1: replay the recorded choices instead of sampling
  double* frob;          // [B] |M|_F^2 of the current Gram-path move
  int32_t* trunc;        // [B] 1 if that move truncated
  int max_sweeps;
  int32_t* err;          // [B] error flags
  int32_t* err_step;     // [B][2] step of the first fatal error, of the first non-convergence
  int cur_step;          // step of the program being launched
  int cur_trunc;         // 1 if that step is a truncating move
  int eig_nsplit;        // > 0: k_eig takes bonds n <= eig_nsplit, k_eig_tri the larger ones
  int defer_bt;          // 1: k_eig_tri leaves the back-transformation to k_eig_bt (reflectors in
                         //    G, phases and tau in V, Z in Ts)
  int2* shape;           // [B] (m, n) of the current move's bond matrix (MIXED runs)
};

enum : int32_t { ERR_ZERO_NORM = 1, ERR_NO_CONVERGE = 2, ERR_CAPACITY = 4, ERR_NAN = 8 };

// Raise an error flag of trajectory b and remember the first failing step.
template <typename R>
__device__ __forceinline__ void flag_err(const Dev<R>& d, int b, int32_t code) {
  atomicOr(&d.err[b], code);
  atomicCAS(&d.err_step[b * 2 + (code == ERR_NO_CONVERGE ? 1 : 0)], -1, d.cur_step);
}

// Gram matrices up to this size are diagonalised in shared memory (k_eig);
// larger ones by the tridiagonal solver (k_eig_tri).
static constexpr int EIG_SMEM_MAX = 131072;
// MIXED runs: FP64 bond Gram matrices up to this dimension go to the
// shared-memory Jacobi solver (36 n^3 flops, short serial chains), larger
// ones to the tridiagonal solver (~12 n^3 flops, longer serial chains).
static constexpr int EIG_JACOBI_N = 64;
static constexpr int TRI_UNROLL = 16;  // loads in flight per thread in L2-resident sweeps
static constexpr int TRI_NB = 8;       // reflectors per compact-WY block of the back-transformation
static constexpr int TRI_INV_ITERS = 2;  // inverse-iteration / orthonormalisation rounds
static constexpr int TRI_INV_EXTRA = 3;  // at most this many further rounds after restarted columns
static constexpr double TRI_CLUSTER_TOL = 1e-3;  // eigenvalue cluster width (relative to |T|)
// the same when V_k is rounded to complex64 afterwards (deferred
// back-transformation): eps_64 / 1e-7 = 2.2e-9 of cross-cluster
// non-orthogonality stays far below the 2^-24 rounding that follows
static constexpr double TRI_CLUSTER_TOL_C64 = 1e-7;
// profiling ledger: flops and bytes per class, then SM cycles per phase of
// the tridiagonal eigensolver (summed over trajectories, thread 0's clock)
static constexpr int LEDGER_WORDS = 2 * NCLASS + EIG_PHASES + MOVE_HIST_WORDS;
static constexpr int LEDGER_HIST = 2 * NCLASS + EIG_PHASES;  // first word of the move histogram
// Moves whose tensor capacity reaches this many elements count as large, and
// so does every move of a circuit above BIG_CIRCUIT_QUBITS qubits (d >= 5).
static constexpr int64_t BIG_MOVE = (int64_t)1 << 17;
static constexpr int BIG_CIRCUIT_QUBITS = 32;
template <typename R>
constexpr int tri_smem_bytes() {
  return 512 * (5 * 2 * (int)sizeof(R) + 3 * (int)sizeof(R)) + 2 * TRI_NB * 512 * 2 * (int)sizeof(R);
}
// without the back-transformation's blocks (MIXED runs defer it to k_eig_bt)
template <typename R>
constexpr int tri_smem_bytes_nobt() {
  return 512 * (5 * 2 * (int)sizeof(R) + 3 * (int)sizeof(R));
}

template <typename R>
__device__ __forceinline__ cx<R>* node_ptr(const Dev<R>& d, int b, int v) {
  return d.T + (int64_t)b * d.tstride + d.off[v];
}

// Algorithmic work of one launch, added once per trajectory by its first block.
__device__ __forceinline__ void ledger_add(unsigned long long* L, int cls, double flops, double bytes) {
  if (!L) return;
  atomicAdd(&L[2 * cls], (unsigned long long)flops);
  atomicAdd(&L[2 * cls + 1], (unsigned long long)bytes);
}

// ------------------------------------------------------------------ init
template <typename R>
__global__ void k_init(Dev<R> d, const int32_t* leafdim, int B) {
  int b = blockIdx.y;
  if (b >= B) return;
  for (int x = threadIdx.x + blockIdx.x * blockDim.x; x < d.ds; x += blockDim.x * gridDim.x) {
    int val = 1;
    if (x >= d.L) val = leafdim[x - d.L];
    d.dims[b * d.ds + x] = val;
  }
  for (int v = 1 + threadIdx.x + blockIdx.x * blockDim.x; v < d.L; v += blockDim.x * gridDim.x) {
    cx<R>* t = node_ptr(d, b, v);
    int dl = (2 * v >= d.L) ? leafdim[2 * v - d.L] : 1;
    int dr = (2 * v + 1 >= d.L) ? leafdim[2 * v + 1 - d.L] : 1;
    for (int i = 0; i < dl * dr; ++i) t[i] = {R(i == 0), R(0)};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.logp[b] = 0.0;
    d.disc[b] = 0.0;
    d.ties[b] = 0;
    d.err[b] = 0;
    d.err_step[2 * b] = -1;
    d.err_step[2 * b + 1] = -1;
  }
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < d.N; i += blockDim.x * gridDim.x)
    d.last[(int64_t)b * d.N + i] = 0;
}

// ------------------------------------------------------------------ SVD move
// Centre move v -> w (neighbour) across their bond.  M = T_v with the bond as
// column index (m x n).  One-sided Jacobi (Hestenes) orthogonalises the
// columns of M V; s_j = |(M V)_j|; keep k singular triplets (s > eps s_max,
// at most kcap); T_v <- U_k, R = S_k V_k^dag (renormalised after a
// truncation) is left in d.Rm for the neighbour.
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__global__ void __launch_bounds__(256) k_svd_move(Dev<R> d, int v, int w, int kcap) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  const int n = leg == 0 ? dl : (leg == 1 ? dr : du);
  const int m = dl * dr * du / n;
  cx<R>* T = node_ptr(d, b, v);
  cx<R>* W = d.W + (int64_t)b * d.wstride;
  cx<R>* V = d.V + (int64_t)b * d.vstride;
  double* sv = d.sv + (int64_t)b * d.nmax;
  int32_t* perm = d.perm + (int64_t)b * d.nmax;
  __shared__ int s_k;
  __shared__ double s_scale;
  if ((int64_t)m * n > d.wstride || n > d.nmax || (int64_t)n * n > d.vstride) {
    if (tid == 0) {
      flag_err(d, b, ERR_CAPACITY);
      d.knew[b] = 0;
    }
    return;
  }

  if (tid == 0)
    ledger_add(d.ledger, KC_SVD, 24.0 * m * (double)n * n + 44.0 * (double)n * n * n,
               2.0 * sizeof(cx<R>) * m * (double)n);
  // gather M (column-major, m x n) and its squared Frobenius norm
  __shared__ double s_part[32];
  double fro_part = 0.0;
  for (int idx = tid; idx < m * n; idx += blockDim.x) {
    int j = idx / m, i = idx - j * m;
    int src;
    if (leg == 2) src = i * du + j;
    else if (leg == 0) src = j * m + i;
    else {
      int l = i / du, u = i - l * du;
      src = (l * dr + j) * du + u;
    }
    cx<R> val = T[src];
    W[idx] = val;
    fro_part += (double)cabs2(val);
  }
  fro_part = warp_sum(fro_part);
  if (lane == 0) s_part[warp] = fro_part;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    int j = idx / n, x = idx - j * n;
    V[idx] = {R(j == x), R(0)};
  }
  __syncthreads();

  double fro2 = 0.0;
  for (int i = 0; i < nwarps; ++i) fro2 += s_part[i];
  if (n > 1) {
    const int ne = n + (n & 1);
    const int M1 = ne - 1;
    const double tolm = d.tol * sqrt((double)(m > 1 ? m : 1));
    // a column below eps |M|_F / sqrt(n) is always dropped (s_max^2 >=
    // |M|_F^2 / n): it takes no part in rotations
    const double skip2 = d.eps * d.eps * fro2 / (double)n;
    int sweep = 0;
    for (; sweep < d.max_sweeps; ++sweep) {
      int rotated = 0;
      for (int s = 0; s < M1; ++s) {
        for (int pr = warp; pr < ne / 2; pr += nwarps) {
          int p, q;
          if (pr == 0) {
            p = 0;
            q = (s % M1) + 1;
          } else {
            p = ((pr + s) % M1) + 1;
            q = ((M1 - pr + s) % M1) + 1;
          }
          if (p >= n || q >= n) continue;
          cx<R>* wp = W + (int64_t)p * m;
          cx<R>* wq = W + (int64_t)q * m;
          // inner products accumulated in double (products of floats are
          // exact in double; this path only sees bonds up to 64)
          double a = 0, bb = 0, gr = 0, gi = 0;
          for (int i = lane; i < m; i += 32) {
            const cx<R> x = wp[i], y = wq[i];
            const double xr = x.x, xi = x.y, yr = y.x, yi = y.y;
            a += xr * xr + xi * xi;
            bb += yr * yr + yi * yi;
            gr += xr * yr + xi * yi;
            gi += xr * yi - xi * yr;
          }
          a = warp_sum(a);
          bb = warp_sum(bb);
          gr = warp_sum(gr);
          gi = warp_sum(gi);
          if (!(a > skip2) || !(bb > skip2)) continue;
          // |g| and its phase without squaring tiny numbers
          const double gm = fmax(fabs(gr), fabs(gi));
          if (gm == 0.0) continue;
          const double grs = gr / gm, gis = gi / gm;
          const double hs = sqrt(grs * grs + gis * gis);
          const double g = gm * hs;
          if (!(g > tolm * sqrt(a) * sqrt(bb))) continue;
          rotated = 1;
          const double zeta = (bb - a) / (2.0 * g);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cd = 1.0 / sqrt(1.0 + t * t);
          const R c = (R)cd, sn = (R)(cd * t);
          const cx<R> ec = {(R)(grs / hs), (R)(-gis / hs)};  // conj(g / |g|), unit modulus
          for (int i = lane; i < m; i += 32) {
            cx<R> x = wp[i], y = cmul(ec, wq[i]);
            wp[i] = {c * x.x - sn * y.x, c * x.y - sn * y.y};
            wq[i] = {sn * x.x + c * y.x, sn * x.y + c * y.y};
          }
          cx<R>* vp = V + (int64_t)p * n;
          cx<R>* vq = V + (int64_t)q * n;
          for (int i = lane; i < n; i += 32) {
            cx<R> x = vp[i], y = cmul(ec, vq[i]);
            vp[i] = {c * x.x - sn * y.x, c * x.y - sn * y.y};
            vq[i] = {sn * x.x + c * y.x, sn * x.y + c * y.y};
          }
        }
        __syncthreads();
      }
      // every thread takes the same decision (a block-wide OR at one barrier)
      if (!__syncthreads_or(rotated)) break;
    }
    if (sweep == d.max_sweeps && tid == 0) flag_err(d, b, ERR_NO_CONVERGE);
  }

  // singular values (double), sort descending, rank
  for (int j = warp; j < n; j += nwarps) {
    double acc = 0.0;
    const cx<R>* wj = W + (int64_t)j * m;
    for (int i = lane; i < m; i += 32) acc += (double)cabs2(wj[i]);
    acc = warp_sum(acc);
    if (lane == 0) {
      double sj = sqrt(acc);
      if (!(sj >= 0.0 && sj < 1e300)) {  // NaN / inf: flag, rank it last
        flag_err(d, b, ERR_NAN);
        sj = 0.0;
      }
      sv[j] = sj;
    }
  }
  __syncthreads();
  for (int j = tid; j < n; j += blockDim.x) {
    double sj = sv[j];
    int r = 0;
    for (int i = 0; i < n; ++i) {
      double si = sv[i];
      r += (si > sj) || (si == sj && i < j);
    }
    perm[r] = j;
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < n; ++i)
      if (perm[i] < 0 || perm[i] >= n) flag_err(d, b, ERR_NAN);
    double smax = sv[perm[0]];
    int k = 0;
    double tot = 0.0;
    for (int i = 0; i < n; ++i) {
      double s = sv[perm[i]];
      tot += s * s;
      if (s > d.eps * smax) ++k;
    }
    if (k < 1) k = 1;
    double scale = 1.0;
    if (smax == 0.0) flag_err(d, b, ERR_ZERO_NORM);
    if (k > kcap) {
      double dsc = 0.0;
      for (int i = kcap; i < n; ++i) dsc += sv[perm[i]] * sv[perm[i]];
      dsc = tot > 0.0 ? dsc / tot : 0.0;
      d.disc[b] += dsc;
      scale = dsc < 1.0 ? 1.0 / sqrt(1.0 - dsc) : 1.0;
      k = kcap;
    }
    s_k = k;
    s_scale = scale;
    const int bond = (w == v / 2) ? v : w;
    D[bond] = k;
    d.knew[b] = k;
    d.nold[b] = n;
  }
  __syncthreads();
  const int k = s_k;
  const R scale = (R)s_scale;
  // T_v <- U_k with the bond dimension k
  for (int idx = tid; idx < m * k; idx += blockDim.x) {
    int c = idx / m, i = idx - c * m;
    int j = perm[c];
    if (j < 0 || j >= n) continue;
    double s = sv[j];
    R inv = s > 0.0 ? (R)(1.0 / s) : R(0);
    cx<R> val = cscale(W[(int64_t)j * m + i], inv);
    int dst;
    if (leg == 2) dst = i * k + c;
    else if (leg == 0) dst = c * m + i;
    else {
      int l = i / du, u = i - l * du;
      dst = (l * k + c) * du + u;
    }
    T[dst] = val;
  }
  // R = S_k V_k^dag (k x n, row-major)
  cx<R>* Rm = d.Rm + (int64_t)b * d.vstride;
  for (int idx = tid; idx < k * n; idx += blockDim.x) {
    int c = idx / n, x = idx - c * n;
    int j = perm[c];
    if (j < 0 || j >= n) continue;
    cx<R> vv = V[(int64_t)j * n + x];
    R s = (R)sv[j] * scale;
    Rm[idx] = {s * vv.x, -s * vv.y};
  }
}

// Copy the workspace back into node v (count from its current dims).
template <typename R>
__global__ void k_copy_back(Dev<R> d, int v) {
  const int b = blockIdx.y;
  const int* D = d.dims + b * d.ds;
  const int64_t cnt = (int64_t)D[2 * v] * D[2 * v + 1] * D[v];
  if (cnt > d.wstride || cnt > d.ncap[v]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag_err(d, b, ERR_CAPACITY);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ledger_add(d.ledger, KC_COPY, 0.0, 2.0 * sizeof(cx<R>) * cnt);
  cx<R>* T = node_ptr(d, b, v);
  const cx<R>* W = d.W + (int64_t)b * d.wstride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    T[i] = W[i];
}

// ------------------------------------------------------------------ Gram-path move
// For large matrices the move factorises M through its Gram matrix:
// G = M^H M (tiled GEMM), G = V L V^H by cyclic two-sided Jacobi (one CTA per
// trajectory, the same rotation as the one-sided kernel), Y = M V_k (tiled
// GEMM), s_c = |Y_c| exactly, U = Y S^-1, R = S V_k^H.  The reconstruction
// M V_k V_k^H and the discarded weight are exact; the Gram matrix only limits
// the orthogonality of U (to about eps s_max / s_c) and the choice of the kept
// space among directions with eigenvalues below eps_gram^2 lambda_max.
template <typename R>
__device__ __forceinline__ int m_addr(int leg, int i, int j, int m, int dr, int du) {
  if (leg == 2) return i * du + j;
  if (leg == 0) return j * m + i;
  int l = i / du, u = i - l * du;
  return (l * dr + j) * du + u;
}

// 64 x 64 output tile of C = A B (complex), K-loop in chunks of 16.
// fa(i, k), fb(k, j) load operands; fc(i, j, v) stores.  A_KFAST: the A
// loader walks k fastest (contiguous when A is row-major).
template <typename R, bool A_KFAST, typename FA, typename FB, typename FC>
__device__ __forceinline__ void tile_gemm64(int Mr, int Nc, int K, int i0, int j0, FA fa, FB fb,
                                            FC fc) {
  __shared__ cx<R> As[16][64];
  __shared__ cx<R> Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = {R(0), R(0)};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      int kk, ii;
      if (A_KFAST) {
        kk = e & 15;
        ii = e >> 4;
      } else {
        kk = e >> 6;
        ii = e & 63;
      }
      const int i = i0 + ii, k = k0 + kk;
      As[kk][ii] = (i < Mr && k < K) ? fa(i, k) : cx<R>{R(0), R(0)};
      const int kb = e >> 6, jb = e & 63;
      const int j = j0 + jb, k2 = k0 + kb;
      Bs[kb][jb] = (j < Nc && k2 < K) ? fb(k2, j) : cx<R>{R(0), R(0)};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      cx<R> av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = cadd(acc[a][c], cmul(av[a], bv[c]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
    if (i >= Mr) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j < Nc) fc(i, j, acc[a][c]);
    }
  }
}

// ------------------------------------------------------------------ tensor-core tile
// 64 x 64 output tile of C = A B (complex FP32) on the tensor cores:
// mma.sync m16n8k8 with TF32 operands and FP32 accumulation, each FP32
// operand split as x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and the
// product formed as hi*hi + hi*lo + lo*hi ("3xTF32"), which keeps FP32-level
// accuracy.  The complex product takes four real products (Ar Br - Ai Bi,
// Ar Bi + Ai Br).  Same operand / output functors as tile_gemm64; the next
// K-chunk's global loads are issued before the current chunk's MMAs.
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32_16x8x8(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                                uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

static constexpr int TC_KT = 16;          // K per shared-memory chunk
static constexpr int TC_AST = TC_KT + 4;  // A row stride (words): conflict-free fragment loads
static constexpr int TC_BST = 64 + 8;     // B row stride (words)

template <bool A_KFAST, typename FA, typename FB, typename FC>
__device__ __forceinline__ void tc_tile_gemm64(int Mr, int Nc, int K, int i0, int j0, FA fa, FB fb,
                                               FC fc) {
  // planes: 0 re-hi, 1 re-lo, 2 im-hi, 3 im-lo
  __shared__ uint32_t As[4][64 * TC_AST];
  __shared__ uint32_t Bs[4][TC_KT * TC_BST];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 1, wn = warp >> 1;  // warp tile: rows wm*32.., cols wn*16..
  float accr[2][2][4], acci[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) accr[a][b][e] = acci[a][b][e] = 0.f;
  cx<float> ra[4], rb[4];  // this thread's elements of the next chunk
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      int kk, ii;
      if (A_KFAST) {
        kk = e & 15;
        ii = e >> 4;
      } else {
        kk = e >> 6;
        ii = e & 63;
      }
      const int i = i0 + ii, k = k0 + kk;
      ra[q] = (i < Mr && k < K) ? fa(i, k) : cx<float>{0.f, 0.f};
      const int kb = e >> 6, jb = e & 63;
      const int j = j0 + jb, k2 = k0 + kb;
      rb[q] = (j < Nc && k2 < K) ? fb(k2, j) : cx<float>{0.f, 0.f};
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      int kk, ii;
      if (A_KFAST) {
        kk = e & 15;
        ii = e >> 4;
      } else {
        kk = e >> 6;
        ii = e & 63;
      }
      const uint32_t rh = tf32_bits(ra[q].x), ih = tf32_bits(ra[q].y);
      const int ao = ii * TC_AST + kk;
      As[0][ao] = rh;
      As[1][ao] = tf32_bits(ra[q].x - __uint_as_float(rh));
      As[2][ao] = ih;
      As[3][ao] = tf32_bits(ra[q].y - __uint_as_float(ih));
      const int kb = e >> 6, jb = e & 63;
      const uint32_t brh = tf32_bits(rb[q].x), bih = tf32_bits(rb[q].y);
      const int bo = kb * TC_BST + jb;
      Bs[0][bo] = brh;
      Bs[1][bo] = tf32_bits(rb[q].x - __uint_as_float(brh));
      Bs[2][bo] = bih;
      Bs[3][bo] = tf32_bits(rb[q].y - __uint_as_float(bih));
    }
  };
  if (K > 0) fetch(0);
  for (int k0 = 0; k0 < K; k0 += TC_KT) {
    stash();
    __syncthreads();
    if (k0 + TC_KT < K) fetch(k0 + TC_KT);
#pragma unroll
    for (int ks = 0; ks < TC_KT; ks += 8) {
      uint32_t af[2][4][4];  // [m-tile][plane][reg]
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm * 32 + mt * 16 + g;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          af[mt][p][0] = As[p][r * TC_AST + ks + t];
          af[mt][p][1] = As[p][(r + 8) * TC_AST + ks + t];
          af[mt][p][2] = As[p][r * TC_AST + ks + t + 4];
          af[mt][p][3] = As[p][(r + 8) * TC_AST + ks + t + 4];
        }
      }
      uint32_t bf[2][4][2];  // [n-tile][plane][reg]
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int cc = wn * 16 + nt * 8 + g;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          bf[nt][p][0] = Bs[p][(ks + t) * TC_BST + cc];
          bf[nt][p][1] = Bs[p][(ks + t + 4) * TC_BST + cc];
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t nah[4], nal[4];  // -Ai (hi, lo): sign bit flipped
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          nah[e] = af[mt][2][e] ^ 0x80000000u;
          nal[e] = af[mt][3][e] ^ 0x80000000u;
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          float(&cr)[4] = accr[mt][nt];
          float(&ci)[4] = acci[mt][nt];
          // small cross terms first
          mma_tf32_16x8x8(cr, af[mt][1], bf[nt][0][0], bf[nt][0][1]);
          mma_tf32_16x8x8(cr, af[mt][0], bf[nt][1][0], bf[nt][1][1]);
          mma_tf32_16x8x8(cr, nal, bf[nt][2][0], bf[nt][2][1]);
          mma_tf32_16x8x8(cr, nah, bf[nt][3][0], bf[nt][3][1]);
          mma_tf32_16x8x8(cr, af[mt][0], bf[nt][0][0], bf[nt][0][1]);
          mma_tf32_16x8x8(cr, nah, bf[nt][2][0], bf[nt][2][1]);
          mma_tf32_16x8x8(ci, af[mt][1], bf[nt][2][0], bf[nt][2][1]);
          mma_tf32_16x8x8(ci, af[mt][0], bf[nt][3][0], bf[nt][3][1]);
          mma_tf32_16x8x8(ci, af[mt][3], bf[nt][0][0], bf[nt][0][1]);
          mma_tf32_16x8x8(ci, af[mt][2], bf[nt][1][0], bf[nt][1][1]);
          mma_tf32_16x8x8(ci, af[mt][0], bf[nt][2][0], bf[nt][2][1]);
          mma_tf32_16x8x8(ci, af[mt][2], bf[nt][0][0], bf[nt][0][1]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = i0 + wm * 32 + mt * 16 + g + (e >> 1) * 8;
        const int j = j0 + wn * 16 + nt * 8 + 2 * t + (e & 1);
        if (i < Mr && j < Nc) fc(i, j, cx<float>{accr[mt][nt][e], acci[mt][nt][e]});
      }
}

// C = A B tile on the tensor cores (TC, FP32 only) or on the FP32/FP64 FMA units.
template <typename R, bool TC, bool A_KFAST, typename FA, typename FB, typename FC>
__device__ __forceinline__ void gemm_tile64(int Mr, int Nc, int K, int i0, int j0, FA fa, FB fb, FC fc) {
  if constexpr (TC && sizeof(R) == 4) {
    tc_tile_gemm64<A_KFAST>(Mr, Nc, K, i0, j0, fa, fb, fc);
  } else {
    tile_gemm64<R, A_KFAST>(Mr, Nc, K, i0, j0, fa, fb, fc);
  }
}

// Neighbour w absorbs R (k x n) on its leg towards v:
//   out[o][i][u] = sum_x R[i][x] in[o][x][u]   (o, u: the other legs)
// written to the workspace W (then copied back).
template <typename R, bool TC>
__global__ void __launch_bounds__(256) k_absorb(Dev<R> d, int w, int v) {
  const int b = blockIdx.z;
  const int* D = d.dims + b * d.ds;
  const int lw = (v == 2 * w) ? 0 : ((v == 2 * w + 1) ? 1 : 2);
  const int dl = D[2 * w], dr = D[2 * w + 1], du = D[w];
  const int n = d.nold[b], k = d.knew[b];
  int outer, inner;
  if (lw == 0) {
    outer = 1;
    inner = dr * du;
  } else if (lw == 1) {
    outer = dl;
    inner = du;
  } else {
    outer = dl * dr;
    inner = 1;
  }
  const int J = outer * inner;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (k <= 0 || (int64_t)k * J > d.wstride || (int64_t)n * J > d.wstride) return;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    ledger_add(d.ledger, KC_ABSORB, 8.0 * k * (double)n * J,
               sizeof(cx<R>) * ((double)n * J + (double)k * n + (double)k * J));
  if (i0 >= k || j0 >= J) return;
  const cx<R>* Rm = d.Rm + (int64_t)b * d.vstride;
  const cx<R>* in = node_ptr(d, b, w);
  cx<R>* out = d.W + (int64_t)b * d.wstride;
  gemm_tile64<R, TC, true>(
      k, J, n, i0, j0, [&](int i, int x) { return Rm[(int64_t)i * n + x]; },
      [&](int x, int j) {
        const int o = j / inner, u = j - o * inner;
        return in[((int64_t)o * n + x) * inner + u];
      },
      [&](int i, int j, cx<R> val) {
        const int o = j / inner, u = j - o * inner;
        out[((int64_t)o * k + i) * inner + u] = val;
      });
}

// M (m x n, row-major) into the workspace.
template <typename R>
__global__ void k_gather_rows(Dev<R> d, int v, int w) {
  const int b = blockIdx.y;
  const int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  const int n = leg == 0 ? dl : (leg == 1 ? dr : du);
  const int m = dl * dr * du / n;
  if (d.shape && blockIdx.x == 0 && threadIdx.x == 0)
    d.shape[b] = (int64_t)m * n > d.wstride ? make_int2(0, 0) : make_int2(m, n);
  if ((int64_t)m * n > d.wstride) return;
  const cx<R>* T = node_ptr(d, b, v);
  cx<R>* W = d.W + (int64_t)b * d.wstride;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * n; idx += gridDim.x * blockDim.x) {
    int i = idx / n, j = idx - i * n;
    W[idx] = T[m_addr<R>(leg, i, j, m, dr, du)];
  }
}

// G = M^H M (n x n)
template <typename R, bool TC>
__global__ void __launch_bounds__(256) k_gram(Dev<R> d, int v, int w) {
  const int b = blockIdx.z;
  const int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  const int n = leg == 0 ? dl : (leg == 1 ? dr : du);
  const int m = dl * dr * du / n;
  if ((int64_t)n * n > d.vstride || (int64_t)m * n > d.wstride) return;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    ledger_add(d.ledger, KC_GRAM, 8.0 * m * (double)n * n,
               sizeof(cx<R>) * ((double)m * n + (double)n * n));
  if (i0 >= n || j0 >= n) return;
  const cx<R>* Mw = d.W + (int64_t)b * d.wstride;
  cx<R>* G = d.G + (int64_t)b * d.vstride;
  gemm_tile64<R, TC, false>(
      n, n, m, i0, j0,
      [&](int i, int k) {
        cx<R> x = Mw[(int64_t)k * n + i];
        return cx<R>{x.x, -x.y};
      },
      [&](int k, int j) { return Mw[(int64_t)k * n + j]; },
      [&](int i, int j, cx<R> val) { G[(int64_t)i * n + j] = val; });
}

// Selection shared by the Gram eigensolvers: eigenvalues (sv[j], any order)
// -> singular values, perm = descending order, kept rank k (s > eps_keep
// s_max, at most kcap), bond dimension update.  Returns k to every
// thread.
template <typename R>
__device__ int eig_select(Dev<R>& d, int b, int v, int w, int kcap, int n, double trace,
                          double eps_keep, long long clk_start = 0) {
  const int tid = threadIdx.x, nth = blockDim.x;
  int* D = d.dims + b * d.ds;
  double* sv = d.sv + (int64_t)b * d.nmax;
  int32_t* perm = d.perm + (int64_t)b * d.nmax;
  __shared__ int s_kk;
  for (int j = tid; j < n; j += nth) {
    double lam = sv[j];
    double sj = lam > 0.0 ? sqrt(lam) : 0.0;
    if (!(sj < 1e300)) {
      flag_err(d, b, ERR_NAN);
      sj = 0.0;
    }
    sv[j] = sj;
  }
  __syncthreads();
  for (int j = tid; j < n; j += nth) {
    double sj = sv[j];
    int r = 0;
    for (int i = 0; i < n; ++i) {
      double si = sv[i];
      r += (si > sj) || (si == sj && i < j);
    }
    perm[r] = j;
  }
  __syncthreads();
  if (tid == 0) {
    double smax = sv[perm[0]];
    int k = 0;
    for (int i = 0; i < n; ++i)
      if (sv[perm[i]] > eps_keep * smax) ++k;
    if (k < 1) k = 1;
    if (smax == 0.0) flag_err(d, b, ERR_ZERO_NORM);
    int trunc = 0;
    if (k > kcap) {
      k = kcap;
      trunc = 1;
    }
    s_kk = k;
    const int bond = (w == v / 2) ? v : w;
    if (d.ledger) {
      const int64_t mm = (int64_t)D[2 * v] * D[2 * v + 1] * (v == 1 ? 1 : D[v]) / (n > 0 ? n : 1);
      unsigned long long* h = d.ledger + LEDGER_HIST +
                              ((int64_t)(d.cur_trunc ? 1 : 0) * MOVE_HIST_N + min(n, MOVE_HIST_N - 1)) * MOVE_HIST_F;
      atomicAdd(&h[0], 1ull);
      atomicAdd(&h[1], (unsigned long long)mm);
      atomicAdd(&h[2], (unsigned long long)k);
      if (clk_start > 0) atomicAdd(&h[3], (unsigned long long)(clock64() - clk_start));
    }
    D[bond] = k;
    d.knew[b] = k;
    d.nold[b] = n;
    d.frob[b] = trace;
    d.trunc[b] = trunc;
  }
  __syncthreads();
  return s_kk;
}

// Jacobi tail: V (row-major n x n eigenvectors) -> V_k into G.
template <typename R>
__device__ void eig_select_tail(Dev<R>& d, int b, int v, int w, int kcap, int n, const cx<R>* V,
                                cx<R>* Gglob, double trace, long long clk_entry) {
  const int k = eig_select(d, b, v, w, kcap, n, trace, d.eps_gram, clk_entry);
  const int32_t* perm = d.perm + (int64_t)b * d.nmax;
  // V_k (n x k, row-major, columns in descending eigenvalue order) into G
  for (int idx = threadIdx.x; idx < n * k; idx += blockDim.x) {
    const int x = idx / k, c = idx - x * k;
    Gglob[idx] = V[(int64_t)x * n + perm[c]];
  }
}

// Eigen-decomposition of G by cyclic two-sided Jacobi; then the kept rank
// and V_k (into G).  The body of k_eig, and of k_eig_tri for the bonds at or
// below eig_nsplit (MIXED runs: one eigensolver launch per move); smem: the
// launch's dynamic shared memory (d.eig_smem_bytes of it).
template <typename R>
__device__ void eig_jacobi(Dev<R>& d, int v, int w, int kcap, unsigned char* eig_smem, long long clk_entry) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  const int n = leg == 0 ? dl : (leg == 1 ? dr : du);
  cx<R>* Gglob = d.G + (int64_t)b * d.vstride;
  cx<R>* V = d.V + (int64_t)b * d.vstride;
  double* sv = d.sv + (int64_t)b * d.nmax;
  // G lives in shared memory when the launch provides room for n x n
  const bool in_smem = (int64_t)n * n * sizeof(cx<R>) <= (int64_t)d.eig_smem_bytes;
  cx<R>* G = in_smem ? reinterpret_cast<cx<R>*>(eig_smem) : Gglob;
  __shared__ R pc[256], ps[256];
  __shared__ cx<R> pe[256];
  __shared__ int pp[256], pq[256];
  __shared__ double s_tr;
  if ((int64_t)n * n > d.vstride || n > d.nmax || n > 512) {
    if (tid == 0) {
      flag_err(d, b, ERR_CAPACITY);
      d.knew[b] = 0;
    }
    return;
  }
  for (int idx = tid; idx < n * n; idx += nth) {
    int x = idx / n, j = idx - x * n;
    V[idx] = {R(x == j), R(0)};
    if (in_smem) G[idx] = Gglob[idx];
  }
  if (tid == 0) ledger_add(d.ledger, KC_EIG, 36.0 * (double)n * n * n, 3.0 * sizeof(cx<R>) * n * (double)n);
  if (tid == 0) {
    double tr = 0.0;
    for (int j = 0; j < n; ++j) tr += (double)G[(int64_t)j * n + j].x;
    s_tr = tr;
  }
  __syncthreads();
  const R skip2 = (R)(d.eps_gram * d.eps_gram * s_tr / (double)n);
  const R tol = (R)d.tol_gram;
  const R tol_abs = (R)(d.tol_abs_gram * s_tr);  // below rounding of G
  if (n > 1) {
    const int ne = n + (n & 1), M1 = ne - 1, np2 = ne / 2;
    int sweep = 0;
    for (; sweep < d.max_sweeps; ++sweep) {
      int rotated = 0;
      for (int s = 0; s < M1; ++s) {
        for (int pr = tid; pr < np2; pr += nth) {
          int p, q;
          if (pr == 0) {
            p = 0;
            q = (s % M1) + 1;
          } else {
            p = ((pr + s) % M1) + 1;
            q = ((M1 - pr + s) % M1) + 1;
          }
          pp[pr] = -1;
          if (p >= n || q >= n) continue;
          const R a = G[(int64_t)p * n + p].x, bb = G[(int64_t)q * n + q].x;
          const cx<R> g = G[(int64_t)p * n + q];
          if (!(a > skip2) || !(bb > skip2)) continue;
          const R gm = fmax(fabs(g.x), fabs(g.y));
          if (gm == R(0)) continue;
          const R grs = g.x / gm, gis = g.y / gm, hs = sqrt(grs * grs + gis * gis), ga = gm * hs;
          if (!(ga > tol * sqrt(a) * sqrt(bb)) || !(ga > tol_abs)) continue;
          rotated = 1;
          const R zeta = (bb - a) / (R(2) * ga);
          const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          const R c = R(1) / sqrt(R(1) + t * t);
          pp[pr] = p;
          pq[pr] = q;
          pc[pr] = c;
          ps[pr] = c * t;
          pe[pr] = {grs / hs, -gis / hs};
        }
        __syncthreads();
        // rows: G <- J^H G, J = [[c, s], [-s e, c e]], e = pe
        for (int idx = tid; idx < np2 * n; idx += nth) {
          const int pr = idx / n, col = idx - pr * n;
          const int p = pp[pr];
          if (p < 0) continue;
          const int q = pq[pr];
          const R c = pc[pr], sn = ps[pr];
          const cx<R> e = pe[pr];
          const cx<R> gp = G[(int64_t)p * n + col], gq = G[(int64_t)q * n + col];
          // conj(Jqp) = -s conj(e), conj(Jqq) = c conj(e)
          const cx<R> ceq = cmulc(e, gq);  // conj(e) * gq
          G[(int64_t)p * n + col] = {c * gp.x - sn * ceq.x, c * gp.y - sn * ceq.y};
          G[(int64_t)q * n + col] = {sn * gp.x + c * ceq.x, sn * gp.y + c * ceq.y};
        }
        __syncthreads();
        // columns: G <- G J, V <- V J
        for (int idx = tid; idx < np2 * n; idx += nth) {
          const int pr = idx / n, row = idx - pr * n;
          const int p = pp[pr];
          if (p < 0) continue;
          const int q = pq[pr];
          const R c = pc[pr], sn = ps[pr];
          const cx<R> e = pe[pr];
          {
            const cx<R> gp = G[(int64_t)row * n + p], gq = cmul(e, G[(int64_t)row * n + q]);
            G[(int64_t)row * n + p] = {c * gp.x - sn * gq.x, c * gp.y - sn * gq.y};
            G[(int64_t)row * n + q] = {sn * gp.x + c * gq.x, sn * gp.y + c * gq.y};
          }
          {
            const cx<R> vp = V[(int64_t)row * n + p], vq = cmul(e, V[(int64_t)row * n + q]);
            V[(int64_t)row * n + p] = {c * vp.x - sn * vq.x, c * vp.y - sn * vq.y};
            V[(int64_t)row * n + q] = {sn * vp.x + c * vq.x, sn * vp.y + c * vq.y};
          }
        }
        __syncthreads();
      }
      if (!__syncthreads_or(rotated)) break;
    }
    if (sweep == d.max_sweeps && tid == 0) flag_err(d, b, ERR_NO_CONVERGE);
  }
  for (int j = tid; j < n; j += nth) sv[j] = (double)G[(int64_t)j * n + j].x;  // eigenvalues
  __syncthreads();
  eig_select_tail(d, b, v, w, kcap, n, V, Gglob, s_tr, clk_entry);
}

template <typename R>
__global__ void __launch_bounds__(512) k_eig(Dev<R> d, int v, int w, int kcap) {
  const long long clk_entry = clock64();
  extern __shared__ __align__(16) unsigned char eig_smem[];
  const int* D = d.dims + blockIdx.x * d.ds;
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  const int n = leg == 0 ? D[2 * v] : (leg == 1 ? D[2 * v + 1] : D[v]);
  if (d.eig_nsplit > 0 && n > d.eig_nsplit) return;  // the tridiagonal solver's share
  eig_jacobi(d, v, w, kcap, eig_smem, clk_entry);
}

// Block-wide sums (blockDim.x a multiple of 32); red holds 64 doubles.
__device__ __forceinline__ double2 block_sum2(double a, double c, double* red) {
  a = warp_sum(a);
  c = warp_sum(c);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[warp] = a;
    red[32 + warp] = c;
  }
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  for (int i = 0; i < nw; ++i) {
    t.x += red[i];
    t.y += red[32 + i];
  }
  return t;
}

__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_zero_bits(float x) { return (__float_as_int(x) << 1) == 0; }
__device__ __forceinline__ int sign_differs(double a, double b) {
  return (int)(((unsigned long long)(__double_as_longlong(a) ^ __double_as_longlong(b))) >> 63);
}
__device__ __forceinline__ int sign_differs(float a, float b) {
  return (int)(((unsigned)(__float_as_int(a) ^ __float_as_int(b))) >> 31);
}

template <typename R>
__device__ __forceinline__ R fast_div(R a, R b) {
  return a / b;
}
template <>
__device__ __forceinline__ float fast_div<float>(float a, float b) {
  return __fdividef(a, b);
}

// Householder vector of column c of A (rows c+1..n-1, already updated):
// H = I - tau v v^H with H x = alpha e_1; v scaled so that |v_0| = 1.
// Writes v into vout[0..m) and into A's column c below the diagonal.
template <typename R>
__device__ void tri_reflector(cx<R>* A, int n, int c, cx<R>* vout, R* tau, cx<R>* ek, double* red) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int m = n - c - 1;
  double x2 = 0.0, t2 = 0.0;
  for (int r = tid; r < m; r += nth) {
    const cx<R> x = A[(int64_t)(c + 1 + r) * n + c];
    const double a2 = (double)x.x * x.x + (double)x.y * x.y;
    x2 += a2;
    if (r > 0) t2 += a2;
  }
  const double2 sums = block_sum2(x2, t2, red);
  const cx<R> x0 = A[(int64_t)(c + 1) * n + c];
  if (sums.y == 0.0) {  // already reduced: H = I
    for (int r = tid; r < m; r += nth) vout[r] = {R(0), R(0)};
    if (tid == 0) {
      tau[c] = R(0);
      ek[c] = x0;
    }
    __syncthreads();
    return;
  }
  const double xn = sqrt(sums.x);
  const double ax0 = sqrt((double)x0.x * x0.x + (double)x0.y * x0.y);
  const double phr = ax0 > 0.0 ? x0.x / ax0 : 1.0, phi = ax0 > 0.0 ? x0.y / ax0 : 0.0;
  const double den = ax0 + xn;  // |x_0 - alpha|
  __syncthreads();               // every thread has read x0
  for (int r = tid; r < m; r += nth) {
    cx<R> vr;
    if (r == 0) {
      vr = {(R)phr, (R)phi};
    } else {
      const cx<R> x = A[(int64_t)(c + 1 + r) * n + c];
      vr = {(R)(x.x / den), (R)(x.y / den)};
    }
    vout[r] = vr;
    A[(int64_t)(c + 1 + r) * n + c] = vr;
  }
  if (tid == 0) {
    tau[c] = (R)(2.0 / (1.0 + sums.y / (den * den)));
    ek[c] = {(R)(-phr * xn), (R)(-phi * xn)};  // alpha = -phase(x_0) |x|
  }
  __syncthreads();
}

// Hermitian eigensolver for Gram matrices too large for shared memory
// (n <= 512), one CTA per trajectory, G resident in L2:
//  1. Householder reduction G = Q T Q^H to Hermitian tridiagonal form, the
//     rank-2 update of step j fused with the matrix-vector product of step
//     j+1 (one read-modify-write pass over the trailing block per step);
//  2. a diagonal phase matrix makes T real symmetric; couplings below
//     2 eps |T| are dropped, splitting T into unreduced blocks;
//  3. eigenvalues by bisection on Sturm counts (thread per eigenvalue);
//  4. eigenvectors of the kept eigenvalues by inverse iteration on the
//     pivoted LU factors of T - lambda I restricted to the eigenvalue's block
//     (thread per vector), alternating with classical Gram-Schmidt applied
//     twice (as LAPACK's stein re-orthogonalises clusters), then a
//     Rayleigh-Ritz step on the kept subspace;
//  5. back-transformation by the stored reflectors.
// (Golub & Van Loan, Matrix Computations, Ch. 8.)  Selection and output as in
// k_eig: V_k (n x k, row-major) into G.
template <typename R>
__global__ void __launch_bounds__(512) k_eig_tri(Dev<R> d, int v, int w, int kcap) {
  const long long clk_entry = clock64();
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int* D = d.dims + b * d.ds;
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  const int n = leg == 0 ? D[2 * v] : (leg == 1 ? D[2 * v + 1] : D[v]);
  extern __shared__ __align__(16) unsigned char tri_smem[];
  if (d.eig_nsplit > 0 && n <= d.eig_nsplit) {  // the Jacobi solver's share
    if (d.eig_smem_bytes > 0) eig_jacobi(d, v, w, kcap, tri_smem, clk_entry);
    return;
  }
  if ((int64_t)n * n > d.vstride || 2 * n > d.vstride || n > d.nmax || n > nth || nth > 512) {
    if (tid == 0) {
      flag_err(d, b, ERR_CAPACITY);
      d.knew[b] = 0;
    }
    return;
  }
  cx<R>* A = d.G + (int64_t)b * d.vstride;
  cx<R>* Vk = d.V + (int64_t)b * d.vstride;
  // real scratch (4 n^2, column-major): eigenvectors Z of T and the LU
  // factors U0, U1, U2
  R* Z = reinterpret_cast<R*>(d.Ts + (int64_t)b * 2 * d.vstride);
  R* U0 = Z + (int64_t)n * n;
  R* U1 = U0 + (int64_t)n * n;
  R* U2 = U1 + (int64_t)n * n;
  double* sv = d.sv + (int64_t)b * d.nmax;
  const int32_t* perm = d.perm + (int64_t)b * d.nmax;
  cx<R>* vk = reinterpret_cast<cx<R>*>(tri_smem);  // reflector of the current step
  cx<R>* wk = vk + 512;                             // w = p - K v; later the phases D
  cx<R>* vn = wk + 512;                             // next reflector; later b^2, lambda
  cx<R>* pp = vn + 512;                             // matvec partials / p
  cx<R>* ek = pp + 512;                             // sub-diagonal of T
  R* dg = reinterpret_cast<R*>(ek + 512);          // diagonal of T
  R* bt = dg + 512;                                 // |sub-diagonal|
  R* tau = bt + 512;                                // reflector scalars
  __shared__ double red[64];
  __shared__ double wx2[32], wt2[32], wvp[32];  // per-warp partial sums
  __shared__ double s_sc;
  __shared__ int bstart[512], bend[512];  // unreduced block [bstart, bend) of each row
  __shared__ short cst[512], cen[512];     // cluster [cst, cen) of each kept column

  double trp = 0.0;
  for (int j = tid; j < n; j += nth) trp += (double)A[(int64_t)j * n + j].x;
  const double trace = block_sum2(trp, 0.0, red).x;
  long long clk0 = clock64();
  auto phase_mark = [&](int ph) {  // cycles of the phase that just ended
    if (tid == 0 && d.ledger) {
      const long long c1 = clock64();
      atomicAdd(&d.ledger[2 * NCLASS + ph], (unsigned long long)(c1 - clk0));
      clk0 = c1;
    }
  };

  // ---- 1. tridiagonalisation
  if (tid == 0) dg[0] = A[0].x;
  if (n == 2 && tid == 0) {
    ek[0] = A[2];
    dg[1] = A[3].x;
  }
  if (n >= 3) {
    // Six barriers per step: reductions (|x|^2 of the next reflector's
    // column, v^H p) are per-warp partials written during the preceding
    // pass and summed in warp order after its barrier (deterministic).
    // Only the lower triangle of the trailing block is kept current.
    const int wid = tid >> 5, lid = tid & 31, nw = nth >> 5;
    tri_reflector(A, n, 0, vk, tau, ek, red);
    {  // p_0 = tau_0 A[1:, 1:] v_0 and v_0^H p_0
      const int m = n - 1, G = nth / m, col = tid % m, g = tid / m;
      if (g < G) {
        cx<R> acc = {R(0), R(0)};
        for (int j = g; j < m; j += G)
          acc = cadd(acc, cmulc(A[(int64_t)(1 + j) * n + 1 + col], vk[j]));
        pp[g * m + col] = acc;
      }
      __syncthreads();
      double vp = 0.0;
      if (tid < m) {
        cx<R> acc = pp[tid];
        for (int gg = 1; gg < G; ++gg) acc = cadd(acc, pp[gg * m + tid]);
        acc = cscale(acc, tau[0]);
        pp[tid] = acc;
        vp = (double)vk[tid].x * acc.x + (double)vk[tid].y * acc.y;
      }
      vp = warp_sum(vp);
      if (lid == 0) wvp[wid] = vp;
      __syncthreads();
    }
    for (int k = 0; k + 3 <= n; ++k) {
      const int o = k + 1, m = n - o;  // trailing block rows/cols o..n-1
      // (a) K = tau/2 v^H p (real), w = p - K v
      double vpsum = 0.0;
      for (int i = 0; i < nw; ++i) vpsum += wvp[i];
      const R K = (R)(0.5 * (double)tau[k] * vpsum);
      for (int r = tid; r < m; r += nth) wk[r] = {pp[r].x - K * vk[r].x, pp[r].y - K * vk[r].y};
      __syncthreads();  // B1
      // (b) column o of the trailing block; partial norms of its rows o+1..
      // (the next reflector's x) and of rows o+2.. (its tail)
      const cx<R> cw0 = {wk[0].x, -wk[0].y}, cv0 = {vk[0].x, -vk[0].y};
      double x2 = 0.0, t2 = 0.0;
      for (int r = tid; r < m; r += nth) {
        cx<R> a = A[(int64_t)(o + r) * n + o];
        const cx<R> t1 = cmul(vk[r], cw0), tt = cmul(wk[r], cv0);
        a = {a.x - t1.x - tt.x, a.y - t1.y - tt.y};
        A[(int64_t)(o + r) * n + o] = a;
        if (r == 0) dg[o] = a.x;
        const double a2 = (double)a.x * a.x + (double)a.y * a.y;
        if (r >= 1) x2 += a2;
        if (r >= 2) t2 += a2;
      }
      x2 = warp_sum(x2);
      t2 = warp_sum(t2);
      if (lid == 0) {
        wx2[wid] = x2;
        wt2[wid] = t2;
      }
      __syncthreads();  // B2
      // (c) next reflector of column o: H = I - tau v v^H, |v_0| = 1
      const bool has_next = (o + 3 <= n);
      if (has_next) {
        double X2 = 0.0, T2 = 0.0;
        for (int i = 0; i < nw; ++i) {
          X2 += wx2[i];
          T2 += wt2[i];
        }
        const int mn = m - 1;  // length of the next reflector
        const cx<R> x0 = A[(int64_t)(o + 1) * n + o];
        if (T2 == 0.0) {  // already reduced: H = I
          for (int r = tid; r < mn; r += nth) vn[r] = {R(0), R(0)};
          if (tid == 0) {
            tau[o] = R(0);
            ek[o] = x0;
          }
        } else {
          const double xn = sqrt(X2);
          const double ax0 = sqrt((double)x0.x * x0.x + (double)x0.y * x0.y);
          const double phr = ax0 > 0.0 ? x0.x / ax0 : 1.0, phi = ax0 > 0.0 ? x0.y / ax0 : 0.0;
          const double den = ax0 + xn;  // |x_0 - alpha|
          for (int r = tid; r < mn; r += nth) {
            cx<R> vr;
            if (r == 0) {
              vr = {(R)phr, (R)phi};
            } else {
              const cx<R> x = A[(int64_t)(o + 1 + r) * n + o];
              vr = {(R)(x.x / den), (R)(x.y / den)};
            }
            vn[r] = vr;
          }
          if (tid == 0) {
            tau[o] = (R)(2.0 / (1.0 + T2 / (den * den)));
            ek[o] = {(R)(-phr * xn), (R)(-phi * xn)};  // alpha = -phase(x_0) |x|
          }
        }
      } else if (tid == 0) {
        ek[o] = A[(int64_t)(n - 1) * n + o];
      }
      __syncthreads();  // B3: vn, tau[o] visible; x0 read by everyone
      if (has_next)  // v stored below the diagonal of column o
        for (int r = tid; r < m - 1; r += nth) A[(int64_t)(o + 1 + r) * n + o] = vn[r];
      // (d) rank-2 update of the lower triangle of rows/cols o+1.. (the
      // upper one is never read again: FP64 is the binding unit, so the
      // Hermitian half is not recomputed), then p_next = A' v_next from the
      // lower triangle read by columns (j >= col) and by rows (j < col)
      const int mp = m - 1;
      if (mp > 0) {
        const int G = nth / mp, col = tid % mp, g = tid / mp;
        cx<R>* colp = A + (int64_t)(o + 1) * n + o + 1 + col;
        if (g < G) {
          const cx<R> cvi = {vk[1 + col].x, -vk[1 + col].y}, cwi = {wk[1 + col].x, -wk[1 + col].y};
          // TRI_UNROLL rows per batch: all loads issued before any store
          for (int j0 = col + g; j0 < mp; j0 += G * TRI_UNROLL) {
            cx<R> a[TRI_UNROLL];
#pragma unroll
            for (int u = 0; u < TRI_UNROLL; ++u) {
              const int j = j0 + u * G;
              if (j < mp) a[u] = colp[(int64_t)j * n];
            }
#pragma unroll
            for (int u = 0; u < TRI_UNROLL; ++u) {
              const int j = j0 + u * G;
              if (j < mp) {
                // a -= v_j conj(w_col) + w_j conj(v_col): eight FMAs, the
                // FP64 minimum for the two complex products
                const cx<R> vj = vk[1 + j], wj = wk[1 + j];
                R ax = a[u].x, ay = a[u].y;
                ax = fma(-vj.x, cwi.x, ax);
                ax = fma(vj.y, cwi.y, ax);
                ay = fma(-vj.x, cwi.y, ay);
                ay = fma(-vj.y, cwi.x, ay);
                ax = fma(-wj.x, cvi.x, ax);
                ax = fma(wj.y, cvi.y, ax);
                ay = fma(-wj.x, cvi.y, ay);
                ay = fma(-wj.y, cvi.x, ay);
                a[u] = {ax, ay};
                colp[(int64_t)j * n] = a[u];
              }
            }
          }
        }
        if (has_next) {
          __syncthreads();  // B4a: the updated lower triangle is visible
          if (g < G) {
            const cx<R>* rowp = A + (int64_t)(o + 1 + col) * n + o + 1;  // row col, entries j < col
            cx<R> acc = {R(0), R(0)};
            for (int j0 = g; j0 < mp; j0 += G * TRI_UNROLL) {
              cx<R> a[TRI_UNROLL];
#pragma unroll
              for (int u = 0; u < TRI_UNROLL; ++u) {
                const int j = j0 + u * G;
                if (j < mp) a[u] = j >= col ? colp[(int64_t)j * n] : rowp[j];
              }
#pragma unroll
              for (int u = 0; u < TRI_UNROLL; ++u) {
                const int j = j0 + u * G;
                // A'[col][j] = conj(A'[j][col]) from the column, itself from the row
                if (j < mp) {
                  // acc += conj(a) v (column entries) or a v (row entries):
                  // four FMAs, the conjugation a sign on a.y
                  const cx<R> vv = vn[j];
                  const R ay = j >= col ? -a[u].y : a[u].y;
                  acc.x = fma(a[u].x, vv.x, acc.x);
                  acc.x = fma(-ay, vv.y, acc.x);
                  acc.y = fma(a[u].x, vv.y, acc.y);
                  acc.y = fma(ay, vv.x, acc.y);
                }
              }
            }
            pp[g * mp + col] = acc;
          }
        }
        __syncthreads();  // B4
        if (has_next) {
          double vp = 0.0;
          if (tid < mp) {
            cx<R> acc = pp[tid];
            for (int gg = 1; gg < G; ++gg) acc = cadd(acc, pp[gg * mp + tid]);
            acc = cscale(acc, tau[o]);
            pp[tid] = acc;
            vp = (double)vn[tid].x * acc.x + (double)vn[tid].y * acc.y;
          }
          vp = warp_sum(vp);
          if (lid == 0) wvp[wid] = vp;
          for (int r = tid; r < mp; r += nth) vk[r] = vn[r];
          __syncthreads();  // B5
        }
      }
    }
    if (tid == 0) dg[n - 1] = A[(int64_t)(n - 1) * n + n - 1].x;
  }
  __syncthreads();
  phase_mark(0);

  // ---- 2. phases D (T = D T_real D^H), scale to |T| <= 1, split
  R* b2 = reinterpret_cast<R*>(vn);
  R* lam = b2 + 512;
  if (tid == 0) {
    cx<R> ph = {R(1), R(0)};
    double dmax = 0.0, bmax = 0.0;
    for (int j = 0; j < n; ++j) {
      wk[j] = ph;
      dmax = fmax(dmax, fabs((double)dg[j]));
      if (j + 1 < n) {
        const cx<R> e = ek[j];
        const double ae = sqrt((double)e.x * e.x + (double)e.y * e.y);
        bt[j] = (R)ae;
        bmax = fmax(bmax, ae);
        if (ae > 0.0) ph = cmul(ph, cx<R>{(R)(e.x / ae), (R)(e.y / ae)});
      }
    }
    double sc = dmax + 2.0 * bmax;
    if (!(sc > 0.0) || !(sc < 1e300)) sc = 1.0;
    s_sc = sc;
  }
  __syncthreads();
  const double sc = s_sc;
  const R epsR = sizeof(R) == 8 ? R(2.220446049250313e-16) : R(1.1920929e-07);
  const R pivmin = sizeof(R) == 8 ? R(1e-280) : R(1e-30);
  // rescaling window of the Sturm minors (exact powers of two)
  const R sturm_hi = sizeof(R) == 8 ? R(0x1p400) : R(0x1p50);   // far from overflow after 8 rows
  const R sturm_lo = sizeof(R) == 8 ? R(0x1p-400) : R(0x1p-50);
  const R sturm_down = sizeof(R) == 8 ? R(0x1p-400) : R(0x1p-50);
  const R sturm_up = sizeof(R) == 8 ? R(0x1p400) : R(0x1p50);
  const R sturm_tiny = sizeof(R) == 8 ? R(0x1p-1000) : R(0x1p-120);
  // rows between range checks: a minor shrinks by at most b^2 >= 4 eps^2 per
  // two rows, so eight rows stay inside FP64's range (2^-408 below the
  // window) but not FP32's (2^-176 below it): FP32 checks every row
  constexpr int sturm_every = sizeof(R) == 8 ? 8 : 1;
  for (int j = tid; j < n; j += nth) {
    dg[j] = (R)(dg[j] / sc);
    if (j + 1 < n) {
      R bj = (R)(bt[j] / sc);
      if (bj <= 2 * epsR) bj = R(0);
      bt[j] = bj;
      b2[j] = bj * bj;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int st = 0;
    for (int i = 0; i < n; ++i) {
      bstart[i] = st;
      if (i == n - 1 || bt[i] == R(0)) {
        for (int r = st; r <= i; ++r) bend[r] = i + 1;
        st = i + 1;
      }
    }
  }
  __syncthreads();

  phase_mark(1);
  // ---- 3. bisection: thread j finds eigenvalue number j - s (ascending) of
  // the block [s, e) that holds row j
  if (tid < n) {
    const int j = tid, s0 = bstart[j], e0 = bend[j];
    R lo = R(-1) - 4 * epsR, hi = R(1) + 4 * epsR;
    for (int it = 0; it < 128; ++it) {
      const R mid = R(0.5) * (lo + hi);
      if (!(hi - lo > fmax(2 * epsR * fmax(fabs(lo), fabs(hi)), R(0.125) * epsR)) || mid == lo || mid == hi)
        break;
      // Sturm count without divisions: the leading principal minors
      // p_i = (d_i - mid) p_{i-1} - b_{i-1}^2 p_{i-2} (p_0 = 1) change sign
      // once per eigenvalue below mid (q_i = p_{i+1} / p_i is the pivot of
      // T - mid I); a zero minor counts as a tiny negative pivot, and the
      // pair is rescaled by exact powers of two to stay in range
      // (sign and zero tests on the bit patterns keep the FP64 pipe to the
      // three operations of the recurrence; |T| <= 1 bounds the growth of a
      // minor to 3x per row, so FP64 checks the range every 8 rows)
      R pm2 = R(1), pm1 = dg[s0] - mid;
      if (fabs(pm1) < pivmin) pm1 = -pivmin;
      int cnt = pm1 < R(0);
      for (int i = s0 + 1; i < e0; ++i) {
        R pc = (dg[i] - mid) * pm1 - b2[i - 1] * pm2;
        if (is_zero_bits(pc)) pc = -copysign(sturm_tiny, pm1);
        cnt += sign_differs(pc, pm1);
        pm2 = pm1;
        pm1 = pc;
        if (((i - s0) & (sturm_every - 1)) == 0) {
          const R big = fmax(fabs(pm1), fabs(pm2));
          if (big > sturm_hi) {
            pm1 *= sturm_down;
            pm2 *= sturm_down;
          } else if (big < sturm_lo) {
            pm1 *= sturm_up;
            pm2 *= sturm_up;
          }
        }
      }
      if (cnt <= j - s0) lo = mid;
      else hi = mid;
    }
    const R l = R(0.5) * (lo + hi);
    lam[j] = l;
    sv[j] = (double)l * sc;
  }
  __syncthreads();
  phase_mark(2);
  // singular values below sqrt(eps) s_max are not resolved by a Gram matrix
  // in this precision
  const double eps_keep = fmax(d.eps_gram, sqrt((double)epsR));
  const int k = eig_select(d, b, v, w, kcap, n, trace, eps_keep, clk_entry);
  if (tid == 0)
    ledger_add(d.ledger, KC_EIG, 16.0 / 3.0 * (double)n * n * n + 8.0 * (double)n * n * k,
               (double)sizeof(cx<R>) * ((double)n * n + (double)n * k));

  // ---- 4. eigenvectors of the kept eigenvalues.  Inverse iteration (thread c
  // for kept column c, shift = its own eigenvalue perm[c], on that
  // eigenvalue's block) alternates with classical Gram-Schmidt applied twice
  // in column order; a column that loses almost all of its norm there
  // restarts from a fresh vector.  Eigenvalues closer than the arithmetic
  // resolves (flat spectra of stabiliser-like states) thus still get
  // independent vectors spanning their invariant subspace, and a
  // Rayleigh-Ritz step on the kept subspace (H = Z^T T Z = Q L Q^T by cyclic
  // Jacobi, Z <- Z Q) diagonalises it.
  // fills column c from thread t0 with stride st (the block: tid, nth; a warp: lane, 32)
  auto start_vec_by = [&](int c, int salt, int s0, int e0, int t0, int st) {
    for (int i = t0; i < n; i += st) {
      uint32_t h = (uint32_t)(i + 7919 * salt) * 0x9E3779B1u ^ ((uint32_t)c + 0x7F4A7C15u) * 0x85EBCA77u;
      h ^= h >> 15;
      h *= 0x2C1B3C6Du;
      h ^= h >> 12;
      const R x = (R)((double)(h >> 8) * (2.0 / 16777216.0) - 1.0 + 1.0 / 16777216.0);
      Z[(int64_t)c * n + i] = (i >= s0 && i < e0) ? x : R(0);
    }
  };
  auto start_vec = [&](int c, int salt, int s0, int e0) { start_vec_by(c, salt, s0, e0, tid, nth); };
  for (int c = 0; c < k; ++c) {
    const int jj = perm[c];
    start_vec(c, 0, bstart[jj], bend[jj]);
  }
  // clusters of kept eigenvalues (descending order): neighbours closer than
  // TRI_CLUSTER_TOL |T| (TRI_CLUSTER_TOL_C64 when V_k is rounded to
  // complex64) share one.  Inverse-iteration vectors of eigenvalues further
  // apart are orthogonal to about eps |T| / gap already, so Gram-Schmidt and
  // the Rayleigh-Ritz rotation act within clusters only (the cluster rule of
  // LAPACK's stein); their cost grows with the square of a cluster's size.
  // (FP32 vectors are orthogonal across clusters only to eps_32 / 1e-3, too
  // coarse: FP32 takes all kept columns as one cluster)
  if (tid == 0) {
    const double crel = d.defer_bt ? TRI_CLUSTER_TOL_C64 : TRI_CLUSTER_TOL;
    const R tolc = sizeof(R) == 8 ? (R)crel * fmax(fabs(lam[perm[0]]), fabs(lam[perm[k - 1]])) : R(4);
    cst[0] = 0;
    for (int a = 1; a < k; ++a) cst[a] = (lam[perm[a - 1]] - lam[perm[a]] <= tolc) ? cst[a - 1] : (short)a;
    cen[k - 1] = (short)k;
    for (int a = k - 2; a >= 0; --a) cen[a] = (cst[a + 1] == cst[a]) ? cen[a + 1] : (short)(a + 1);
  }
  __syncthreads();
  R* cf = reinterpret_cast<R*>(pp);  // Gram-Schmidt coefficients (k <= 512)
  R* shift = reinterpret_cast<R*>(ek);  // inverse-iteration shifts (the sub-diagonal is no longer needed)
  const int warp_id = tid >> 5, lane_id = tid & 31, nwarp = nth >> 5;
  // Shifts: in descending order, a kept column's shift stays at least
  // 10 eps |T| below the previous shift of its unreduced block, so columns
  // of one block never share a shift (LAPACK's stein perturbs close
  // eigenvalues the same way); the vectors of a cluster then start from
  // distinct solves and Gram-Schmidt with Rayleigh-Ritz settles its subspace.
  {
    R* last = cf + 512;  // last shift of each block, by its first row
    for (int i = tid; i < n; i += nth) last[i] = R(4);
    __syncthreads();
    if (tid == 0)
      for (int c = 0; c < k; ++c) {
        const int jj = perm[c], blk = bstart[jj];
        const R sh = fmin(lam[jj], last[blk] - R(10) * epsR);
        shift[c] = sh;
        last[blk] = sh;
      }
    __syncthreads();
  }
  int iters = TRI_INV_ITERS;
  for (int iter = 0; iter < iters; ++iter) {
    if (tid < k) {
      const int c = tid, jj = perm[c], s0 = bstart[jj], e0 = bend[jj];
      const R l = shift[c];
      // forward elimination with partial pivoting, right-hand side carried along
      R* zc = Z + (int64_t)c * n;  // this thread's column (column-major)
      R* u0 = U0 + (int64_t)c * n;
      R* u1 = U1 + (int64_t)c * n;
      R* u2 = U2 + (int64_t)c * n;
      R cd = dg[s0] - l, cu = s0 + 1 < e0 ? bt[s0] : R(0), cr = zc[s0];
      for (int i = s0; i + 1 < e0; ++i) {
        const R lo_ = bt[i], dn = dg[i + 1] - l, un = (i + 2 < e0) ? bt[i + 1] : R(0);
        const R rn = zc[i + 1];
        const int at = i;
        if (fabs(cd) >= fabs(lo_)) {
          const R piv = cd == R(0) ? epsR : cd;
          const R mlt = lo_ / piv;
          u0[at] = piv;
          u1[at] = cu;
          u2[at] = R(0);
          zc[at] = cr;
          cd = dn - mlt * cu;
          cu = un;
          cr = rn - mlt * cr;
        } else {
          const R mlt = cd / lo_;
          u0[at] = lo_;
          u1[at] = dn;
          u2[at] = un;
          zc[at] = rn;
          cd = cu - mlt * dn;
          cu = -mlt * un;
          cr = cr - mlt * rn;
        }
      }
      u0[e0 - 1] = cd;
      zc[e0 - 1] = cr;
      // back substitution; pivots below eps |T| are replaced by eps |T|.
      // The solution grows by up to 1/eps per small pivot: whenever it
      // passes BIG, the solved part and the remaining right-hand side are
      // scaled down together (the system is linear).
      const R BIG = sizeof(R) == 8 ? R(1e150) : R(1e15);
      R y1 = R(0), y2 = R(0), ymax = R(0);
      for (int i = e0 - 1; i >= s0; --i) {
        const int at = i;
        R u = u0[at];
        if (fabs(u) < epsR) u = u < R(0) ? -epsR : epsR;
        R y = zc[at];
        if (i + 1 < e0) y -= u1[at] * y1;
        if (i + 2 < e0) y -= u2[at] * y2;
        y = y / u;
        if (!(fabs(y) <= BIG)) {
          const R f = fabs(y) > R(0) && fabs(y) <= BIG * BIG ? R(1) / fabs(y) : R(0);
          for (int t = s0; t < e0; ++t)
            if (t != i) zc[t] *= f;
          y = f > R(0) ? y * f : (y > R(0) ? R(1) : R(-1));
          y1 *= f;
          y2 *= f;
          ymax *= f;
        }
        zc[at] = y;
        y2 = y1;
        y1 = y;
        ymax = fmax(ymax, fabs(y));
      }
      const R inv = ymax > R(0) && ymax < R(1e30) ? R(1) / ymax : R(1);
      for (int i = s0; i < e0; ++i) zc[i] *= inv;
    }
    __syncthreads();
    // a column alone in its cluster is only normalised (one warp per column,
    // all at once; a zero vector restarts)
    int zero_col = 0;
    for (int a = warp_id; a < k; a += nwarp) {
      if (cen[a] - cst[a] != 1) continue;
      R* za = Z + (int64_t)a * n;
      double nn = 0.0;
      for (int i = lane_id; i < n; i += 32) nn += (double)za[i] * za[i];
      nn = warp_sum(nn);
      if (nn > 0.0) {
        const R sc1 = (R)(1.0 / sqrt(nn));
        for (int i = lane_id; i < n; i += 32) za[i] *= sc1;
      } else {
        const int jj = perm[a];
        start_vec_by(a, 1 + iter * 4, bstart[jj], bend[jj], lane_id, 32);
        zero_col = 1;
      }
    }
    // classical Gram-Schmidt, twice, columns of the larger clusters in order
    bool restarted = __syncthreads_or(zero_col) != 0;  // uniform: every thread sees the same sums
    for (int a = 0; a < k; ++a) {
      if (cen[a] - cst[a] == 1) continue;  // uniform
      const int jj = perm[a];
      for (int rep = 0; rep < 2; ++rep) {
        for (int attempt = 0; attempt < 2; ++attempt) {
          // coefficients <z_b, z_a>: one warp per b, lanes over rows
          for (int bb = cst[a] + warp_id; bb < a; bb += nwarp) {
            R acc = R(0);
            const R* zb = Z + (int64_t)bb * n;
            const R* za = Z + (int64_t)a * n;
            for (int i = lane_id; i < n; i += 32) acc += zb[i] * za[i];
            acc = warp_sum(acc);
            if (lane_id == 0) cf[bb] = acc;
          }
          __syncthreads();
          double n0 = 0.0, n1 = 0.0;
          for (int i = tid; i < n; i += nth) {
            R z = Z[(int64_t)a * n + i];
            n0 += (double)z * z;
            for (int bb = cst[a]; bb < a; ++bb) z -= cf[bb] * Z[(int64_t)bb * n + i];
            Z[(int64_t)a * n + i] = z;
            n1 += (double)z * z;
          }
          const double2 nn = block_sum2(n0, n1, red);
          if (nn.y > 1e-6 * nn.x && nn.y > 0.0) {
            const R sc1 = (R)(1.0 / sqrt(nn.y));
            for (int i = tid; i < n; i += nth) Z[(int64_t)a * n + i] *= sc1;
            __syncthreads();
            break;
          }
          // dependent on the previous columns: restart from a fresh vector
          start_vec(a, 1 + iter * 4 + rep * 2 + attempt, bstart[jj], bend[jj]);
          restarted = true;
          __syncthreads();
        }
      }
    }
    // a restarted column holds a random vector until inverse iterations
    // have acted on it: two more rounds follow every restart
    if (restarted) iters = min(max(iters, iter + 3), TRI_INV_ITERS + TRI_INV_EXTRA);
  }
  phase_mark(3);
  // Rayleigh-Ritz within the clusters of more than one column: TZ into U0
  // (column-major), H = Z^T (TZ) into U1 (k x k), Q into U2.  With every
  // cluster a single column, H is diagonal and Z stays as it is.
  int multi = 0;
  for (int a = tid; a < k; a += nth) multi |= cen[a] - cst[a] > 1;
  if (__syncthreads_or(multi)) {
  R* TZ = U0;
  R* H = U1;
  R* Q = U2;
  for (int idx = tid; idx < n * k; idx += nth) {
    const int c = idx / n, i = idx - c * n;
    const R* zc = Z + (int64_t)c * n;
    R t = dg[i] * zc[i];
    if (i > 0) t += bt[i - 1] * zc[i - 1];
    if (i + 1 < n) t += bt[i] * zc[i + 1];
    TZ[idx] = t;
  }
  for (int idx = tid; idx < k * k; idx += nth) {
    Q[idx] = R((idx / k) == (idx % k));
    H[idx] = R(0);
  }
  __syncthreads();
  for (int e = warp_id; e < k * k; e += nwarp) {  // one warp per entry, lanes over rows
    const int a = e / k, c = e - a * k;
    if (c < a || c >= cen[a]) continue;  // within a's cluster only
    R acc = R(0);
    const R* za = Z + (int64_t)a * n;
    const R* tc = TZ + (int64_t)c * n;
    for (int i = lane_id; i < n; i += 32) acc += za[i] * tc[i];
    acc = warp_sum(acc);
    if (lane_id == 0) {
      H[a * k + c] = acc;
      H[c * k + a] = acc;
    }
  }
  __syncthreads();
  if (k > 1) {
    __shared__ R rc[256], rs[256];
    __shared__ int rp[256], rq[256];
    const int ke = k + (k & 1), M1 = ke - 1, np2 = ke / 2;
    const R rtol = 8 * epsR;  // rotations below rounding are not needed
    for (int sweep = 0; sweep < 12; ++sweep) {
      int rotated = 0;
      for (int st = 0; st < M1; ++st) {
        for (int pr = tid; pr < np2; pr += nth) {
          int p, q;
          if (pr == 0) {
            p = 0;
            q = (st % M1) + 1;
          } else {
            p = ((pr + st) % M1) + 1;
            q = ((M1 - pr + st) % M1) + 1;
          }
          rp[pr] = -1;
          if (p >= k || q >= k) continue;
          const R hpp = H[p * k + p], hqq = H[q * k + q], hpq = H[p * k + q];
          if (!(fabs(hpq) > rtol * (fabs(hpp) + fabs(hqq))) || hpq == R(0)) continue;
          rotated = 1;
          const R zeta = (hqq - hpp) / (R(2) * hpq);
          const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
          const R c = R(1) / sqrt(R(1) + t * t);
          rp[pr] = p;
          rq[pr] = q;
          rc[pr] = c;
          rs[pr] = c * t;
        }
        __syncthreads();
        for (int idx = tid; idx < np2 * k; idx += nth) {  // rows of H
          const int pr = idx / k, col = idx - pr * k;
          const int p = rp[pr];
          if (p < 0) continue;
          const int q = rq[pr];
          const R c = rc[pr], sn = rs[pr];
          const R hp = H[p * k + col], hq = H[q * k + col];
          H[p * k + col] = c * hp - sn * hq;
          H[q * k + col] = sn * hp + c * hq;
        }
        __syncthreads();
        for (int idx = tid; idx < np2 * k; idx += nth) {  // columns of H and Q
          const int pr = idx / k, row = idx - pr * k;
          const int p = rp[pr];
          if (p < 0) continue;
          const int q = rq[pr];
          const R c = rc[pr], sn = rs[pr];
          const R hp = H[row * k + p], hq = H[row * k + q];
          H[row * k + p] = c * hp - sn * hq;
          H[row * k + q] = sn * hp + c * hq;
          const R qp = Q[row * k + p], qq = Q[row * k + q];
          Q[row * k + p] = c * qp - sn * qq;
          Q[row * k + q] = sn * qp + c * qq;
        }
        __syncthreads();
      }
      if (!__syncthreads_or(rotated)) break;
    }
  }
  // Z_k Q into TZ (column-major n x k), then back into Z's first k columns
  for (int idx = tid; idx < n * k; idx += nth) {
    const int c = idx / n, i = idx - c * n;
    R acc = R(0);
    for (int a = cst[c]; a < cen[c]; ++a) acc += Z[(int64_t)a * n + i] * Q[a * k + c];
    TZ[idx] = acc;
  }
  __syncthreads();
  for (int idx = tid; idx < n * k; idx += nth) Z[idx] = TZ[idx];
  __syncthreads();
  }
  // residual |T z - (z^T T z) z| of every kept vector (one warp per column):
  // above 16 sqrt(eps) |T| the vectors did not converge (reported, not fatal)
  for (int c = warp_id; c < k; c += nwarp) {
    const R* zc = Z + (int64_t)c * n;
    auto tz = [&](int i) {
      R t = dg[i] * zc[i];
      if (i > 0) t += bt[i - 1] * zc[i - 1];
      if (i + 1 < n) t += bt[i] * zc[i + 1];
      return t;
    };
    R zz = R(0), ztz = R(0);
    for (int i = lane_id; i < n; i += 32) {
      zz += zc[i] * zc[i];
      ztz += zc[i] * tz(i);
    }
    zz = warp_sum(zz);
    ztz = warp_sum(ztz);
    const R mu = zz > R(0) ? ztz / zz : R(0);
    R r2 = R(0);
    for (int i = lane_id; i < n; i += 32) {
      const R e = tz(i) - mu * zc[i];
      r2 += e * e;
    }
    r2 = warp_sum(r2);
    if (lane_id == 0 && (!(fabs(zz - R(1)) <= R(1e-3)) || !(r2 <= R(256) * epsR))) flag_err(d, b, ERR_NO_CONVERGE);
  }

  phase_mark(4);
  if (d.defer_bt) {
    // phases D and reflector scalars for k_eig_bt; Z and the reflectors stay put
    for (int x = tid; x < n; x += nth) {
      Vk[x] = wk[x];
      Vk[n + x] = {x < n - 2 ? tau[x] : R(0), R(0)};
    }
    return;
  }
  // ---- 5. back-transformation V_k = H_0 ... H_{n-3} D Z_k (n x k in Vk),
  // TRI_NB reflectors at a time in compact WY form (Schreiber & Van Loan):
  // H_j0 ... H_j1 = I - Vb Tb Vb^H, so Vk <- Vk - Vb (Tb (Vb^H Vk)).
  for (int idx = tid; idx < n * k; idx += nth) {
    const int x = idx / k, c = idx - x * k;
    const R z = Z[(int64_t)c * n + x];
    Vk[idx] = {wk[x].x * z, wk[x].y * z};
  }
  cx<R>* Vb = reinterpret_cast<cx<R>*>(tau + 512);  // [TRI_NB][512] reflectors, by row
  cx<R>* Wp = Vb + TRI_NB * 512;                      // [512 * TRI_NB] partial products
  __shared__ cx<R> Tb[TRI_NB][TRI_NB], Sb[TRI_NB][TRI_NB];
  __syncthreads();
  for (int jhi = n - 3; jhi >= 0; jhi -= TRI_NB) {
    const int j0 = jhi - TRI_NB + 1 > 0 ? jhi - TRI_NB + 1 : 0, nbk = jhi - j0 + 1;
    for (int idx = tid; idx < nbk * n; idx += nth) {
      const int i = idx / n, r = idx - i * n, j = j0 + i;
      Vb[i * 512 + r] = (r > j && tau[j] != R(0)) ? A[(int64_t)r * n + j] : cx<R>{R(0), R(0)};
    }
    __syncthreads();
    if (tid < nbk * nbk) {  // Sb = Vb^H Vb (upper part)
      const int l = tid / nbk, i = tid - l * nbk;
      if (l < i) {
        cx<R> acc = {R(0), R(0)};
        for (int r = j0 + i + 1; r < n; ++r) acc = cadd(acc, cmulc(Vb[l * 512 + r], Vb[i * 512 + r]));
        Sb[l][i] = acc;
      }
    }
    __syncthreads();
    if (tid == 0) {  // forward recurrence for the triangular factor
      for (int i = 0; i < nbk; ++i) {
        const R ti = tau[j0 + i];
        for (int l = 0; l < i; ++l) {
          cx<R> acc = {R(0), R(0)};
          for (int m2 = l; m2 < i; ++m2) acc = cadd(acc, cmul(Tb[l][m2], Sb[m2][i]));
          Tb[l][i] = cscale(acc, -ti);
        }
        Tb[i][i] = {ti, R(0)};
        for (int l = i + 1; l < nbk; ++l) Tb[l][i] = {R(0), R(0)};
      }
    }
    __syncthreads();
    {  // Wp = Vb^H Vk, partial sums over row groups
      const int G = nth / k, c = tid % k, g = tid / k;
      if (g < G) {
        cx<R> acc[TRI_NB];
#pragma unroll
        for (int i = 0; i < TRI_NB; ++i) acc[i] = {R(0), R(0)};
        for (int r = j0 + 1 + g; r < n; r += G) {
          const cx<R> x = Vk[(int64_t)r * k + c];
#pragma unroll
          for (int i = 0; i < TRI_NB; ++i)
            if (i < nbk) acc[i] = cadd(acc[i], cmulc(Vb[i * 512 + r], x));
        }
#pragma unroll
        for (int i = 0; i < TRI_NB; ++i) Wp[(g * TRI_NB + i) * k + c] = acc[i];
      }
      __syncthreads();
      if (tid < k) {  // reduce, then apply Tb
        cx<R> wv[TRI_NB];
#pragma unroll
        for (int i = 0; i < TRI_NB; ++i) {
          cx<R> acc = Wp[i * k + tid];
          for (int gg = 1; gg < G; ++gg) acc = cadd(acc, Wp[(gg * TRI_NB + i) * k + tid]);
          wv[i] = acc;
        }
#pragma unroll
        for (int l = 0; l < TRI_NB; ++l) {
          cx<R> acc = {R(0), R(0)};
#pragma unroll
          for (int i = 0; i < TRI_NB; ++i)
            if (i >= l && i < nbk) acc = cadd(acc, cmul(Tb[l][i], wv[i]));
          Wp[l * k + tid] = acc;
        }
      }
      __syncthreads();
    }
    // Vk -= Vb Wp on rows j0+1..n-1 (loads of a batch issued before its stores)
    const int rows = n - j0 - 1, tot = rows * k;
    for (int base = tid; base < tot; base += nth * TRI_UNROLL) {
      cx<R> x[TRI_UNROLL];
#pragma unroll
      for (int u = 0; u < TRI_UNROLL; ++u) {
        const int idx = base + u * nth;
        if (idx < tot) x[u] = Vk[(int64_t)(j0 + 1) * k + idx];
      }
#pragma unroll
      for (int u = 0; u < TRI_UNROLL; ++u) {
        const int idx = base + u * nth;
        if (idx < tot) {
          const int r = j0 + 1 + idx / k, c = idx % k;
          cx<R> acc = x[u];
#pragma unroll
          for (int i = 0; i < TRI_NB; ++i)
            if (i < nbk) {
              const cx<R> t = cmul(Vb[i * 512 + r], Wp[i * k + c]);
              acc = {acc.x - t.x, acc.y - t.y};
            }
          Vk[(int64_t)(j0 + 1) * k + idx] = acc;
        }
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < n * k; idx += nth) A[idx] = Vk[idx];
  phase_mark(5);
}

// Exact singular values of the kept columns: Y = M V_k was written into T_v;
// s_c = |Y_c|, U_c = Y_c / s_c, R_c = s_c V_c^H (renormalised after a
// truncation, the discarded weight 1 - sum s_c^2 / |M|_F^2 recorded), spread
// over the whole grid: k_unorm_sums accumulates s_c^2 per column
// (shared-memory partials, one atomic per column and block), k_unorm_scale
// decides the renormalisation, k_unorm_apply scales U and forms R.  The column of element a of T_v in its
// storage order: leg 2 (i, c): a % k; leg 0 (c, i): a / m; leg 1 (l, c, u):
// (a / du) % k.
template <typename R>
__device__ __forceinline__ void unorm_dims(const Dev<R>& d, int b, int v, int w, int& leg, int& n, int& k,
                                           int& m, int& du) {
  const int* D = d.dims + b * d.ds;
  leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  n = d.nold[b];
  k = d.knew[b];
  const int dl0 = D[2 * v], dr0 = D[2 * v + 1], du0 = D[v];
  const int dl = leg == 0 ? n : dl0, dr = leg == 1 ? n : dr0;
  du = leg == 2 ? n : du0;
  m = k > 0 ? dl * dr * du / n : 0;
}

template <typename R>
__global__ void __launch_bounds__(256) k_unorm_sums(Dev<R> d, int v, int w) {
  const int b = blockIdx.y;
  int leg, n, k, m, du;
  unorm_dims(d, b, v, w, leg, n, k, m, du);
  if (k <= 0 || k > 512) return;
  __shared__ double part[512];
  for (int c = threadIdx.x; c < k; c += blockDim.x) part[c] = 0.0;
  __syncthreads();
  const cx<R>* T = node_ptr(d, b, v);
  const int64_t tot = (int64_t)m * k;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < tot; a += (int64_t)gridDim.x * blockDim.x) {
    const int c = leg == 2 ? (int)(a % k) : (leg == 0 ? (int)(a / m) : (int)((a / du) % k));
    atomicAdd(&part[c], (double)cabs2(T[a]));
  }
  __syncthreads();
  double* acc = d.sv + (int64_t)b * d.nmax;
  for (int c = threadIdx.x; c < k; c += blockDim.x)
    if (part[c] != 0.0) atomicAdd(&acc[c], part[c]);
}

template <typename R>
__global__ void k_unorm_zero(Dev<R> d, int B) {
  const int b = blockIdx.x;
  if (b >= B) return;
  for (int c = threadIdx.x; c < d.nmax; c += blockDim.x) d.sv[(int64_t)b * d.nmax + c] = 0.0;
}

template <typename R>
__global__ void k_unorm_scale(Dev<R> d, int v, int w, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int leg, n, k, m, du;
  unorm_dims(d, b, v, w, leg, n, k, m, du);
  if (k <= 0) return;
  double* sv = d.sv + (int64_t)b * d.nmax;
  double kept = 0.0;
  for (int c = 0; c < k; ++c) {
    kept += sv[c];
    sv[c] = sqrt(sv[c]);
  }
  const double fro2 = d.frob[b];
  double scale = 1.0;
  if (d.trunc[b] && fro2 > 0.0 && kept > 0.0) {
    d.disc[b] += fmax(0.0, 1.0 - kept / fro2);
    scale = sqrt(fro2 / kept);
  }
  if (!(kept > 0.0)) flag_err(d, b, ERR_ZERO_NORM);
  d.frob[b] = scale;  // consumed by k_unorm_apply
}

template <typename R>
__global__ void __launch_bounds__(256) k_unorm_apply(Dev<R> d, int v, int w) {
  const int b = blockIdx.y;
  int leg, n, k, m, du;
  unorm_dims(d, b, v, w, leg, n, k, m, du);
  if (k <= 0) return;
  const double* sv = d.sv + (int64_t)b * d.nmax;
  cx<R>* T = node_ptr(d, b, v);
  const int64_t tot = (int64_t)m * k;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < tot; a += stride) {
    const int c = leg == 2 ? (int)(a % k) : (leg == 0 ? (int)(a / m) : (int)((a / du) % k));
    const double sc = sv[c];
    T[a] = cscale(T[a], sc > 0.0 ? (R)(1.0 / sc) : R(0));
  }
  const cx<R>* Vk = d.G + (int64_t)b * d.vstride;
  cx<R>* Rm = d.Rm + (int64_t)b * d.vstride;
  const R scale = (R)d.frob[b];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)k * n; idx += stride) {
    const int c = (int)(idx / n), x = (int)(idx - (int64_t)c * n);
    const cx<R> vv = Vk[(int64_t)x * k + c];
    const R sc = (R)sv[c] * scale;
    Rm[idx] = {sc * vv.x, -sc * vv.y};
  }
}

// Back-transformation of the tridiagonal solver's eigenvectors, spread over
// CTAs (MIXED runs): V_k = H_0 ... H_{n-3} D Z_k with H_j = I - tau_j v_j
// v_j^H (v_j below the diagonal of column j of the reduced matrix), each CTA
// applying all reflectors to BT_COLS kept columns in FP64 in shared memory,
// then rounding V_k to complex64 (row-major n x k) for Y = M V_k.  The single
// CTA of k_eig_tri would apply them to all k columns itself; here the k
// columns take k / BT_COLS SMs at once.
static constexpr int BT_COLS = 16;
// dynamic shared memory of k_eig_bt for bonds up to nm (the launch's capacity)
__host__ __device__ constexpr int bt_smem_bytes(int nm = 512) {
  return (nm * BT_COLS + nm + 16 * BT_COLS) * (int)sizeof(cx<double>);
}
__global__ void __launch_bounds__(256) k_eig_bt(Dev<float> df, Dev<double> dv) {
  const int b = blockIdx.y;
  const int n = dv.nold[b], k = dv.knew[b];
  if (n <= dv.eig_nsplit || k <= 0 || n > 512 || (int64_t)n * k > dv.vstride) return;
  unsigned dyn = 0;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  if ((int64_t)bt_smem_bytes(n) > (int64_t)dyn) {  // launched for smaller bonds
    if (threadIdx.x == 0 && blockIdx.x == 0) flag_err(dv, b, ERR_CAPACITY);
    return;
  }
  const int c0 = blockIdx.x * BT_COLS;
  if (c0 >= k) return;
  const int nc = min(BT_COLS, k - c0);
  const int tid = threadIdx.x, col = tid & (BT_COLS - 1), part = tid >> 4;  // 16 columns x 16 row parts
  extern __shared__ __align__(16) unsigned char bt_smem[];
  cx<double>* X = reinterpret_cast<cx<double>*>(bt_smem);   // [n][BT_COLS]
  cx<double>* vj = X + (int64_t)n * BT_COLS;                 // [n] current reflector
  cx<double>* red = vj + n;                                  // [16][BT_COLS] partial dots
  const cx<double>* A = dv.G + (int64_t)b * dv.vstride;
  const double* Z = reinterpret_cast<const double*>(dv.Ts + (int64_t)b * 2 * dv.vstride);
  const cx<double>* D = dv.V + (int64_t)b * dv.vstride;
  const cx<double>* tau = D + n;
  for (int idx = tid; idx < n * BT_COLS; idx += blockDim.x) {
    const int x = idx / BT_COLS, c = idx - x * BT_COLS;
    const double z = c < nc ? Z[(int64_t)(c0 + c) * n + x] : 0.0;
    X[idx] = {D[x].x * z, D[x].y * z};
  }
  for (int j = n - 3; j >= 0; --j) {
    const double tj = tau[j].x;
    if (tj == 0.0) continue;  // uniform: every thread reads the same tau
    __syncthreads();
    for (int r = j + 1 + tid; r < n; r += blockDim.x) vj[r] = A[(int64_t)r * n + j];
    __syncthreads();
    cx<double> acc = {0.0, 0.0};
    for (int r = j + 1 + part; r < n; r += 16) acc = cadd(acc, cmulc(vj[r], X[r * BT_COLS + col]));
    red[part * BT_COLS + col] = acc;
    __syncthreads();
    cx<double> w = {0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 16; ++q) w = cadd(w, red[q * BT_COLS + col]);
    w = cscale(w, tj);
    for (int r = j + 1 + part; r < n; r += 16) {
      const cx<double> t = cmul(vj[r], w);
      cx<double>& xr = X[r * BT_COLS + col];
      xr = {xr.x - t.x, xr.y - t.y};
    }
  }
  __syncthreads();
  cx<float>* out = df.G + (int64_t)b * df.vstride;
  for (int idx = tid; idx < n * BT_COLS; idx += blockDim.x) {
    const int x = idx / BT_COLS, c = idx - x * BT_COLS;
    if (c < nc) out[(int64_t)x * k + c0 + c] = {(float)X[idx].x, (float)X[idx].y};
  }
}


// MIXED runs: the FP64 eigensolver leaves V_k (n x k, row-major, complex128)
// in its Gram buffer; the tensor-core contraction Y = M V_k takes it in
// complex64.
__global__ void k_vk_to_float(Dev<float> d, const cx<double>* G64, int nmax_here) {
  const int b = blockIdx.x;
  const int n = d.nold[b], k = d.knew[b];
  if (k <= 0 || n > nmax_here || (int64_t)n * k > d.vstride) return;  // larger: k_eig_bt's output
  const cx<double>* src = G64 + (int64_t)b * d.vstride;
  cx<float>* dst = d.G + (int64_t)b * d.vstride;
  for (int i = threadIdx.x; i < n * k; i += blockDim.x) dst[i] = {(float)src[i].x, (float)src[i].y};
}

// Y = M V_k: m x k, written into T_v with bond dimension k.
template <typename R, bool TC>
__global__ void __launch_bounds__(256) k_form_u(Dev<R> d, int v, int w) {
  const int b = blockIdx.z;
  const int* D = d.dims + b * d.ds;
  const int leg = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
  // dims already hold k on the bond; n is the previous dimension
  const int n = d.nold[b], k = d.knew[b];
  if (k <= 0) return;
  const int dl0 = D[2 * v], dr0 = D[2 * v + 1], du0 = D[v];
  const int dl = leg == 0 ? n : dl0, dr = leg == 1 ? n : dr0, du = leg == 2 ? n : du0;
  const int m = dl * dr * du / n;
  if ((int64_t)m * n > d.wstride) return;
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    ledger_add(d.ledger, KC_FORMU, 8.0 * m * (double)n * k,
               sizeof(cx<R>) * ((double)m * n + (double)n * k + (double)m * k));
  if (i0 >= m || j0 >= k) return;
  const cx<R>* Mw = d.W + (int64_t)b * d.wstride;
  const cx<R>* Vs = d.G + (int64_t)b * d.vstride;  // V_k
  cx<R>* T = node_ptr(d, b, v);
  gemm_tile64<R, TC, true>(
      m, k, n, i0, j0, [&](int i, int kk) { return Mw[(int64_t)i * n + kk]; },
      [&](int kk, int j) { return Vs[(int64_t)kk * k + j]; },
      [&](int i, int c, cx<R> val) {
        int dst;
        if (leg == 2) dst = i * k + c;
        else if (leg == 0) dst = c * m + i;
        else {
          int l = i / du, u = i - l * du;
          dst = (l * k + c) * du + u;
        }
        T[dst] = val;
      });
}

// ------------------------------------------------------------------ MPO threading
// Operator-Schmidt factors of CNOT: control side {|0><0|, |1><1|}, target side
// {I, X}.  A factor F_k applied on a leaf leg of node v; the up bond becomes
// (k, u) with index k * du + u.
template <typename R>
__global__ void k_thread_leaf(Dev<R> d, int v, int leg, int side) {
  const int b = blockIdx.y;
  int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  const int cnt = dl * dr * 2 * du;
  if (cnt > d.wstride) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag_err(d, b, ERR_CAPACITY);
    return;
  }
  const cx<R>* T = node_ptr(d, b, v);
  cx<R>* out = d.W + (int64_t)b * d.wstride;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cnt; idx += gridDim.x * blockDim.x) {
    int u2 = idx % (2 * du);
    int rest = idx / (2 * du);
    int y = rest % dr, x = rest / dr;
    int kk = u2 / du, u = u2 - kk * du;
    int xo = leg == 0 ? x : y;   // output physical index on the gate leg
    cx<R> val;
    if (side == 0) {              // |k><k| on the control
      val = (xo == kk) ? T[(x * dr + y) * du + u] : cx<R>{R(0), R(0)};
    } else {                      // I (k=0) or X (k=1) on the target
      int xi = kk ? 1 - xo : xo;
      int xs = leg == 0 ? xi : x, ys = leg == 0 ? y : xi;
      val = T[(xs * dr + ys) * du + u];
    }
    out[idx] = val;
  }
}

template <typename R>
__global__ void k_thread_dims_leaf(Dev<R> d, int v, int B) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) d.dims[b * d.ds + v] *= 2;
}

// Internal path node: its path-child leg and its up leg both carry k (block
// diagonal).  The child leg's dimension in dims is already doubled.
template <typename R>
__global__ void k_thread_node(Dev<R> d, int v, int leg) {
  const int b = blockIdx.y;
  const int* D = d.dims + b * d.ds;
  const int dl0 = D[2 * v], dr0 = D[2 * v + 1], du = D[v];
  const int dl = leg == 0 ? dl0 / 2 : dl0, dr = leg == 1 ? dr0 / 2 : dr0;  // input dims
  const int ol = leg == 0 ? 2 * dl : dl, orr = leg == 1 ? 2 * dr : dr, ou = 2 * du;
  const int cnt = ol * orr * ou;
  if (cnt > d.wstride) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag_err(d, b, ERR_CAPACITY);
    return;
  }
  const cx<R>* T = node_ptr(d, b, v);
  cx<R>* out = d.W + (int64_t)b * d.wstride;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cnt; idx += gridDim.x * blockDim.x) {
    int u2 = idx % ou, rest = idx / ou;
    int y2 = rest % orr, x2 = rest / orr;
    int ku = u2 / du, u = u2 - ku * du;
    int kc, x = x2, y = y2;
    if (leg == 0) {
      kc = x2 / dl;
      x = x2 - kc * dl;
    } else {
      kc = y2 / dr;
      y = y2 - kc * dr;
    }
    out[idx] = (kc == ku) ? T[(x * dr + y) * du + u] : cx<R>{R(0), R(0)};
  }
}

// Lowest common ancestor: both child legs carry the same k.
template <typename R>
__global__ void k_thread_lca(Dev<R> d, int v) {
  const int b = blockIdx.y;
  const int* D = d.dims + b * d.ds;
  const int ol = D[2 * v], orr = D[2 * v + 1], du = D[v];
  const int dl = ol / 2, dr = orr / 2;
  const int cnt = ol * orr * du;
  if (cnt > d.wstride) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flag_err(d, b, ERR_CAPACITY);
    return;
  }
  const cx<R>* T = node_ptr(d, b, v);
  cx<R>* out = d.W + (int64_t)b * d.wstride;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < cnt; idx += gridDim.x * blockDim.x) {
    int u = idx % du, rest = idx / du;
    int y2 = rest % orr, x2 = rest / orr;
    int k1 = x2 / dl, x = x2 - k1 * dl, k2 = y2 / dr, y = y2 - k2 * dr;
    out[idx] = (k1 == k2) ? T[(x * dr + y) * du + u] : cx<R>{R(0), R(0)};
  }
}

// Both qubits in one node: CNOT permutes the leaf indices in place.
template <typename R>
__global__ void k_gate_node(Dev<R> d, int v, int orient, int B) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = idx / 64, u = idx % 64;
  if (b >= B) return;
  const int* D = d.dims + b * d.ds;
  const int du = D[v];
  if (u >= du) return;
  cx<R>* T = node_ptr(d, b, v);
  // element (x, y, u) at (x * 2 + y) * du + u, both legs of dimension 2
  int i1, i2;
  if (orient == 0) {  // control on l: swap (1,0) <-> (1,1)
    i1 = 2 * du + u;
    i2 = 3 * du + u;
  } else {            // control on r: swap (0,1) <-> (1,1)
    i1 = du + u;
    i2 = 3 * du + u;
  }
  cx<R> t = T[i1];
  T[i1] = T[i2];
  T[i2] = t;
}

// ------------------------------------------------------------------ single-qubit layer
// One thread per (trajectory, level-1 node): applies the node's ops of this
// layer in program order to every column u of T[x][y][u].
template <typename R>
__device__ void apply2x2(cx<R>* T, int dl, int dr, int du, int leg, const cx<R> U[4]) {
  for (int u = 0; u < du; ++u) {
    if (leg == 0) {
      for (int y = 0; y < dr; ++y) {
        cx<R> a0 = T[(0 * dr + y) * du + u], a1 = T[(1 * dr + y) * du + u];
        T[(0 * dr + y) * du + u] = cadd(cmul(U[0], a0), cmul(U[1], a1));
        T[(1 * dr + y) * du + u] = cadd(cmul(U[2], a0), cmul(U[3], a1));
      }
    } else {
      for (int x = 0; x < dl; ++x) {
        cx<R> a0 = T[(x * dr + 0) * du + u], a1 = T[(x * dr + 1) * du + u];
        T[(x * dr + 0) * du + u] = cadd(cmul(U[0], a0), cmul(U[1], a1));
        T[(x * dr + 1) * du + u] = cadd(cmul(U[2], a0), cmul(U[3], a1));
      }
    }
  }
}

template <typename R>
__global__ void k_layer1q(Dev<R> d, const Op1* ops, const Group1* groups, int g0, int ng, int B) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int b = idx / ng, g = idx % ng;
  if (b >= B) return;
  const Group1 G = groups[g0 + g];
  const int v = G.node;
  const int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  cx<R>* T = node_ptr(d, b, v);
  const R rs2 = (R)0.70710678118654752440;
  for (int e = G.begin; e < G.end; ++e) {
    const Op1 o = ops[e];
    cx<R> U[4];
    if (o.kind == O1_RESET_Z || o.kind == O1_RESET_X) {
      uint8_t* lq = d.last + (int64_t)b * d.N + o.qubit;
      if (*lq) {
        U[0] = {0, 0}; U[1] = {1, 0}; U[2] = {1, 0}; U[3] = {0, 0};
        apply2x2(T, dl, dr, du, o.leg, U);
        *lq = 0;
      }
      if (o.kind == O1_RESET_X) {
        U[0] = {rs2, 0}; U[1] = {rs2, 0}; U[2] = {rs2, 0}; U[3] = {-rs2, 0};
        apply2x2(T, dl, dr, du, o.leg, U);
      }
    } else if (o.kind == O1_SRX) {
      double th = d.theta[b];
      R c = (R)cos(th), s = (R)sin(th);
      U[0] = {c, 0}; U[1] = {0, -s}; U[2] = {0, -s}; U[3] = {c, 0};
      apply2x2(T, dl, dr, du, o.leg, U);
    } else if (o.kind == O1_PTA) {
      double p[4];
      if (d.noise == TTN_NOISE_SRX_PTA) {
        double c = cos(d.theta[b]), s = sin(d.theta[b]);
        p[0] = c * c; p[1] = s * s; p[2] = 0.0; p[3] = 0.0;
      } else if (d.noise == TTN_NOISE_DEPOL) {
        const double g = d.gamma[b];
        p[0] = 1.0 - g; p[1] = g / 3; p[2] = g / 3; p[3] = g / 3;
      } else {
        double g = d.gamma[b], r = sqrt(1.0 - g);
        p[0] = (1 + r) * (1 + r) / 4; p[1] = g / 4; p[2] = g / 4; p[3] = (1 - r) * (1 - r) / 4;
      }
      double uu = draw_uniform(d.seed, d.traj[b], (uint32_t)o.event);
      double cum = 0.0;
      int kk = 3;
      double margin = 1e300;
      for (int i = 0; i < 3; ++i) {
        cum += p[i];
        margin = fmin(margin, fabs(uu - cum));
        if (kk == 3 && uu < cum) kk = i;
      }
      uint8_t* ch = d.choice + (int64_t)b * d.n_events + o.event;
      if (d.forced) {
        kk = *ch;
      } else {
        *ch = (uint8_t)kk;
        if (margin < d.tie_eps) atomicAdd(&d.ties[b], 1);
      }
      atomicAdd(&d.logp[b], log(p[kk]));
      if (kk == 1) { U[0] = {0, 0}; U[1] = {1, 0}; U[2] = {1, 0}; U[3] = {0, 0}; }
      if (kk == 2) { U[0] = {0, 0}; U[1] = {0, -1}; U[2] = {0, 1}; U[3] = {0, 0}; }
      if (kk == 3) { U[0] = {1, 0}; U[1] = {0, 0}; U[2] = {0, 0}; U[3] = {-1, 0}; }
      if (kk > 0) apply2x2(T, dl, dr, du, o.leg, U);
    }
  }
}

// ------------------------------------------------------------------ centre sampling
// One warp per trajectory; the centre is at the level-1 node of the qubit.
template <typename R>
__global__ void k_measure(Dev<R> d, int q, int event, int recbit, int xbasis, int pos, int B) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  const int v = pos >> 1, leg = pos & 1;
  const int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  cx<R>* T = node_ptr(d, b, v);
  const int cnt = dl * dr * du;
  const R rs2 = (R)0.70710678118654752440;
  if (xbasis) {  // H on the qubit's leg, then Z measurement
    const int half = cnt / 2;
    for (int e = lane; e < half; e += 32) {
      int i0, i1;
      if (leg == 0) { i0 = e; i1 = e + dr * du; }
      else { int x = e / du, u = e % du; i0 = (x * dr) * du + u; i1 = (x * dr + 1) * du + u; }
      cx<R> a0 = T[i0], a1 = T[i1];
      T[i0] = {rs2 * (a0.x + a1.x), rs2 * (a0.y + a1.y)};
      T[i1] = {rs2 * (a0.x - a1.x), rs2 * (a0.y - a1.y)};
    }
    __syncwarp();
  }
  double n0 = 0.0, n1 = 0.0;
  for (int e = lane; e < cnt; e += 32) {
    int x = e / (dr * du), y = (e / du) % dr;
    int bit = leg == 0 ? x : y;
    double a = (double)cabs2(T[e]);
    if (bit) n1 += a; else n0 += a;
  }
  n0 = warp_sum(n0);
  n1 = warp_sum(n1);
  double tot = n0 + n1;
  double p1 = n1 / tot, p0 = 1.0 - p1;
  double uu = draw_uniform(d.seed, d.traj[b], (uint32_t)event);
  uint8_t* ch = d.choice + (int64_t)b * d.n_events + event;
  int mres = d.forced ? (int)*ch : (uu >= p0 ? 1 : 0);
  double pm = mres ? p1 : p0;
  const double nm = mres ? n1 : n0;
  R sc = nm > 0.0 ? (R)(1.0 / sqrt(nm)) : R(0);
  for (int e = lane; e < cnt; e += 32) {
    int x = e / (dr * du), y = (e / du) % dr;
    int bit = leg == 0 ? x : y;
    T[e] = bit == mres ? cscale(T[e], sc) : cx<R>{R(0), R(0)};
  }
  if (lane == 0) {
    d.logp[b] += log(pm);
    if (!d.forced) {
      *ch = (uint8_t)mres;
      if (fabs(uu - p0) < d.tie_eps) d.ties[b] += 1;
    }
    d.rec[(int64_t)b * d.n_rec + recbit] = (uint8_t)mres;
    d.last[(int64_t)b * d.N + q] = (uint8_t)mres;
    if (!(tot > 0.0)) flag_err(d, b, ERR_ZERO_NORM);
  }
}

// Amplitude damping at one location (Eqs. 2-3), exact Kraus unravelling:
// jump with probability gamma * P(1).
template <typename R>
__global__ void k_ad(Dev<R> d, int q, int event, int pos, int B) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  const int v = pos >> 1, leg = pos & 1;
  const int* D = d.dims + b * d.ds;
  const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
  cx<R>* T = node_ptr(d, b, v);
  const int cnt = dl * dr * du;
  double n0 = 0.0, n1 = 0.0;
  for (int e = lane; e < cnt; e += 32) {
    int x = e / (dr * du), y = (e / du) % dr;
    int bit = leg == 0 ? x : y;
    double a = (double)cabs2(T[e]);
    if (bit) n1 += a; else n0 += a;
  }
  n0 = warp_sum(n0);
  n1 = warp_sum(n1);
  const double g = d.gamma[b];
  const double tot = n0 + n1;
  const double P1 = n1 / tot;
  const double p1 = g * P1;
  const double uu = draw_uniform(d.seed, d.traj[b], (uint32_t)event);
  uint8_t* ch = d.choice + (int64_t)b * d.n_events + event;
  const bool jump = d.forced ? (*ch != 0) : (uu < p1);
  __syncwarp();
  if (jump) {
    // K1 = sqrt(g)|0><1|: the |1> slice moves to |0>, normalised by sqrt(n1)
    R sc = n1 > 0.0 ? (R)(1.0 / sqrt(n1)) : R(0);
    const int half = cnt / 2;
    for (int e = lane; e < half; e += 32) {
      int i0, i1;
      if (leg == 0) { i0 = e; i1 = e + dr * du; }
      else { int x = e / du, u = e % du; i0 = (x * dr) * du + u; i1 = (x * dr + 1) * du + u; }
      T[i0] = cscale(T[i1], sc);
      T[i1] = {R(0), R(0)};
    }
  } else {
    R s0 = (R)(1.0 / sqrt(n0 + (1.0 - g) * n1));
    R s1 = (R)(sqrt(1.0 - g) / sqrt(n0 + (1.0 - g) * n1));
    for (int e = lane; e < cnt; e += 32) {
      int x = e / (dr * du), y = (e / du) % dr;
      int bit = leg == 0 ? x : y;
      T[e] = cscale(T[e], bit ? s1 : s0);
    }
  }
  if (lane == 0) {
    d.logp[b] += jump ? log(p1) : log1p(-p1);
    if (!d.forced) {
      *ch = (uint8_t)jump;
      if (fabs(uu - p1) < d.tie_eps) d.ties[b] += 1;
    }
  }
}

// ------------------------------------------------------------------ debug amplitudes
// Contract the whole tree of trajectory b for every basis state (N <= 24,
// bonds <= 64, leaves <= 16): one thread per amplitude, bottom-up.
template <typename R>
__global__ void k_amplitudes(Dev<R> d, int b, const int32_t* qubit_of_leaf, int nq,
                             double* out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= ((int64_t)1 << nq)) return;
  const int L = d.L;
  const int* D = d.dims + b * d.ds;
  cx<double> vec[16][64];  // per node (v < L <= 16), bonds <= 64
  for (int v = L - 1; v >= 1; --v) {
    const int dl = D[2 * v], dr = D[2 * v + 1], du = D[v];
    const cx<R>* T = node_ptr(d, b, v);
    cx<double> acc[64];
    for (int u = 0; u < du; ++u) acc[u] = {0.0, 0.0};
    if (2 * v >= L) {
      int ql = qubit_of_leaf[2 * v - L], qr = qubit_of_leaf[2 * v + 1 - L];
      int x = ql >= 0 ? (int)((idx >> ql) & 1) : 0;
      int y = qr >= 0 ? (int)((idx >> qr) & 1) : 0;
      for (int u = 0; u < du; ++u) {
        cx<R> t = T[(x * dr + y) * du + u];
        acc[u] = {(double)t.x, (double)t.y};
      }
    } else {
      for (int x = 0; x < dl; ++x)
        for (int y = 0; y < dr; ++y) {
          cx<double> a = vec[2 * v][x], bb = vec[2 * v + 1][y];
          cx<double> ab = {a.x * bb.x - a.y * bb.y, a.x * bb.y + a.y * bb.x};
          for (int u = 0; u < du; ++u) {
            cx<R> t = T[(x * dr + y) * du + u];
            acc[u].x += ab.x * (double)t.x - ab.y * (double)t.y;
            acc[u].y += ab.x * (double)t.y + ab.y * (double)t.x;
          }
        }
    }
    for (int u = 0; u < du; ++u) vec[v][u] = acc[u];
  }
  out[2 * idx] = vec[1][0].x;
  out[2 * idx + 1] = vec[1][0].y;
}

// ------------------------------------------------------------------ host driver
#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error(std::string("CUDA: ") + cudaGetErrorString(e_) + " at " #call);    \
      return TTN_ECUDA;                                                            \
    }                                                                              \
  } while (0)

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

Profile& profile() {
  static Profile p;
  return p;
}

ttn_status philox_uniforms_device(uint64_t seed, const uint64_t* trajs, uint64_t n_traj,
                                  const int32_t* events, int32_t n_events, double* out) {
  uint64_t* dt = nullptr;
  int32_t* de = nullptr;
  double* dout = nullptr;
  const size_t cnt = (size_t)n_traj * n_events;
  CK(cudaMalloc(&dt, n_traj * sizeof(uint64_t)));
  CK(cudaMalloc(&de, n_events * sizeof(int32_t)));
  CK(cudaMalloc(&dout, cnt * sizeof(double)));
  CK(cudaMemcpy(dt, trajs, n_traj * sizeof(uint64_t), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(de, events, n_events * sizeof(int32_t), cudaMemcpyHostToDevice));
  k_philox_uniforms<<<ceil_div(cnt, 256), 256>>>(seed, dt, (int)n_traj, de, n_events, dout);
  CK(cudaGetLastError());
  CK(cudaMemcpy(out, dout, cnt * sizeof(double), cudaMemcpyDeviceToHost));
  cudaFree(dt);
  cudaFree(de);
  cudaFree(dout);
  return TTN_OK;
}

// Bond capacity of bond (x, parent(x)) outside gates.
static std::vector<int> bond_caps(const ttn_circuit& c, int chi) {
  const int L = c.L;
  std::vector<int> nq(2 * L, 0);
  for (int q = 0; q < c.N; ++q) nq[L + c.leaf_of_qubit[q]] = 1;
  for (int x = L - 1; x >= 1; --x) nq[x] = nq[2 * x] + nq[2 * x + 1];
  std::vector<int> cap(2 * L, 1);
  for (int x = 2; x < 2 * L; ++x) {
    if (x >= L) {
      cap[x] = nq[x] ? 2 : 1;
      continue;
    }
    int a = nq[x], bq = c.N - nq[x];
    int e = std::min(a, bq);
    int64_t v = e >= 30 ? (int64_t)1 << 30 : ((int64_t)1 << e);
    cap[x] = (int)std::min<int64_t>(v, chi);
  }
  return cap;
}

template <typename R>
struct Engine {
  const ttn_circuit& c;
  const Program& prog;
  int chi, noise, B;
  int gemm_mode = 0;               // 0 auto, 1 FMA units, 2 tensor cores (FP32)
  bool mixed = false;              // MIXED: exact Gram matrix + FP64 eigensolver on every move
  cudaStream_t st;
  std::vector<int> bcap;           // bond caps (outside gates)
  std::vector<int64_t> ncap;       // node slot capacity (elements)
  std::vector<int64_t> off;
  int64_t tstride = 0, wstride = 0, vstride = 0;
  int nmax = 0;
  // device buffers
  cx<R>* dT = nullptr;
  cx<R>* dW = nullptr;
  cx<R>* dV = nullptr;
  cx<R>* dR = nullptr;
  cx<R>* dG = nullptr;
  cx<R>* dTs = nullptr;
  int64_t* dOff = nullptr;
  int32_t* dDims = nullptr;
  double* dSv = nullptr;
  int32_t* dPerm = nullptr;
  int32_t* dK = nullptr;
  int32_t* dN = nullptr;
  double* dLogp = nullptr;
  double* dDisc = nullptr;
  int32_t* dTies = nullptr;
  uint8_t* dRec = nullptr;
  uint8_t* dLast = nullptr;
  double* dTheta = nullptr;
  double* dGamma = nullptr;
  uint64_t* dTraj = nullptr;
  int32_t* dErr = nullptr;
  int32_t* dErrStep = nullptr;
  double* dFrob = nullptr;
  int32_t* dTrunc = nullptr;
  uint8_t* dChoice = nullptr;
  int32_t* dLeafdim = nullptr;
  Op1* dOp1 = nullptr;
  Group1* dGroups = nullptr;
  unsigned long long* dLedger = nullptr;
  // MIXED runs: exact Gram matrix workspaces and the FP64 eigensolver's buffers
  int2* dShape = nullptr;
  unsigned int* dAmax = nullptr;
  int* dExpo = nullptr;
  uint16_t* dSlices = nullptr;
  unsigned long long* dGfix = nullptr;
  cx<double>* dG64 = nullptr;
  cx<double>* dV64 = nullptr;
  cx<double>* dTs64 = nullptr;
  int* dCExpo = nullptr;           // row exponents of the exact contractions
  int64_t sstride = 0;             // bf16 digit tiles per trajectory (largest move)
  int crows = 0;                   // row exponents per trajectory
  GramArgs gargs, gbase;
  Dev<R> base{};                   // the whole batch (dev = a group of it, see select_group)
  int64_t b0 = 0;                  // first trajectory of the selected group
  double eps_mixed = 1e-6;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  std::vector<int> event_class;
  uint64_t class_launches[NCLASS] = {0};
  Dev<R> dev{};

  // Launch wrapper: counts launches per class and, when profiling that
  // class, brackets the launch with events on the launch stream.
  uint64_t kernel_launches = 0;    // kernels launched since the last collect_profile

  template <typename F>
  void timed(int cls, F&& fn) {
    timed(cls, 1, fn);
  }
  // nk: kernels fn launches
  template <typename F>
  void timed(int cls, int nk, F&& fn) {
    Profile& pf = profile();
    class_launches[cls]++;
    kernel_launches += (uint64_t)nk;
    if (pf.active && (pf.timed_class == cls || pf.timed_class == NCLASS)) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, st);
      fn();
      cudaEventRecord(b, st);
      events.push_back({a, b});
      event_class.push_back(cls);
    } else {
      fn();
    }
  }

  void collect_profile() {
    Profile& pf = profile();
    if (!pf.active) {
      if (dLedger) cudaMemset(dLedger, 0, sizeof(unsigned long long) * LEDGER_WORDS);
      for (int c = 0; c < NCLASS; ++c) class_launches[c] = 0;
      kernel_launches = 0;
      return;
    }
    for (size_t i = 0; i < events.size(); ++i) {
      auto& e = events[i];
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
        pf.ms += ms;
        pf.class_ms[event_class[i]] += ms;
      }
      pf.launches++;
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    events.clear();
    event_class.clear();
    unsigned long long h[LEDGER_WORDS] = {0};
    if (dLedger && cudaMemcpy(h, dLedger, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess) {
      for (int c = 0; c < NCLASS; ++c) {
        pf.flops[c] += (double)h[2 * c];
        pf.bytes[c] += (double)h[2 * c + 1];
      }
      for (int ph = 0; ph < EIG_PHASES; ++ph) pf.eig_phase_cycles[ph] += (double)h[2 * NCLASS + ph];
      for (int i = 0; i < MOVE_HIST_WORDS; ++i) pf.move_hist[i] += (double)h[LEDGER_HIST + i];
    }
    for (int c = 0; c < NCLASS; ++c) {
      pf.class_launches[c] += class_launches[c];
      class_launches[c] = 0;
    }
    pf.kernels += kernel_launches;
    kernel_launches = 0;
    if (dLedger) cudaMemset(dLedger, 0, sizeof(h));
  }

  Engine(const ttn_circuit& cc, const Program& p, int chi_, int noise_, cudaStream_t s)
      : c(cc), prog(p), chi(chi_), noise(noise_), B(0), st(s) {
    bcap = bond_caps(c, chi);
    const int L = c.L;
    ncap.assign(L, 0);
    off.assign(L, 0);
    int64_t acc = 0;
    int maxb = 2;
    for (int v = 1; v < L; ++v) {
      int64_t cl = bcap[2 * v], cr = bcap[2 * v + 1], cu = v == 1 ? 1 : bcap[v];
      ncap[v] = 4 * cl * cr * cu;
      off[v] = acc;
      acc += (ncap[v] + 31) / 32 * 32;
      maxb = std::max<int>(maxb, (int)std::max(cl, std::max(cr, cu)));
    }
    tstride = acc;
    int64_t wmax = 0;
    for (int v = 1; v < L; ++v) wmax = std::max(wmax, ncap[v]);
    wstride = (wmax + 31) / 32 * 32;
    nmax = 2 * maxb;
    vstride = (int64_t)nmax * nmax;
    // digit tiles of the exact Gram matrix: the largest bond matrix any move
    // of the program can form (capacities, legs doubled inside a gate)
    for (const Step& st : prog.steps) {
      if (st.kind != S_MOVE) continue;
      const int v = st.a, w = st.b;
      const int bond = (w == v / 2) ? v : w;
      const int lv = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
      const int64_t c3[3] = {2 * (int64_t)bcap[2 * v], 2 * (int64_t)bcap[2 * v + 1],
                             v == 1 ? 1 : 2 * (int64_t)bcap[v]};
      int64_t mm = 1;
      for (int t = 0; t < 3; ++t)
        if (t != lv) mm *= c3[t];
      mm = std::min<int64_t>(mm, ncap[v]);
      const int nb2 = (int)(2 * bcap[bond]);
      sstride = std::max<int64_t>(sstride, gram_slice_elems(mm, nb2));
      // the exact contractions Y = M V_k (m x n times n x k) and R T_w
      // (k x n times n x J, J the product of w's other two legs)
      const int kc = std::min<int>(nb2, st.c ? bcap[bond] : 2 * bcap[bond]);
      const int lw = (v == 2 * w) ? 0 : ((v == 2 * w + 1) ? 1 : 2);
      const int64_t w3[3] = {2 * (int64_t)bcap[2 * w], 2 * (int64_t)bcap[2 * w + 1],
                             w == 1 ? 1 : 2 * (int64_t)bcap[w]};
      int64_t J = 1;
      for (int t = 0; t < 3; ++t)
        if (t != lw) J *= w3[t];
      J = std::min<int64_t>(J, ncap[w]);
      sstride = std::max<int64_t>(sstride, contract_form_elems(mm, nb2, kc));
      sstride = std::max<int64_t>(sstride, contract_absorb_elems(nb2, kc, J));
      crows = (int)std::max<int64_t>(crows, std::max<int64_t>(mm, J) + 512);
    }
    sstride = (sstride + 63) / 64 * 64;  // 128-byte aligned digit tiles
  }

  size_t bytes_per_traj() const {
    size_t b = sizeof(cx<R>) * (size_t)(tstride + wstride + 5 * vstride) +  // V, Rm, G, Ts (2)
               sizeof(int32_t) * (2 * c.L + 2 * nmax + 4) + sizeof(double) * (nmax + 5) + c.n_rec + c.N +
               c.n_events + 64;
    if (mixed)
      b += sizeof(uint16_t) * (size_t)sstride + sizeof(unsigned long long) * (size_t)(2 * nmax) * (2 * nmax) +
           sizeof(cx<double>) * (size_t)(4 * vstride) + (sizeof(unsigned) + sizeof(int)) * 2 * nmax +
           sizeof(int) * (size_t)crows + 64;
    return b;
  }

  ttn_status alloc(int Bmax) {
    B = Bmax;
    CK(cudaMalloc(&dT, sizeof(cx<R>) * (size_t)tstride * B));
    CK(cudaMalloc(&dW, sizeof(cx<R>) * (size_t)wstride * B));
    CK(cudaMalloc(&dV, sizeof(cx<R>) * (size_t)vstride * B));
    CK(cudaMalloc(&dR, sizeof(cx<R>) * (size_t)vstride * B));
    CK(cudaMalloc(&dG, sizeof(cx<R>) * (size_t)vstride * B));
    CK(cudaMalloc(&dTs, sizeof(cx<R>) * (size_t)vstride * 2 * B));
    CK(cudaMalloc(&dOff, sizeof(int64_t) * 2 * c.L));  // off, then ncap
    CK(cudaMalloc(&dDims, sizeof(int32_t) * 2 * c.L * B));
    CK(cudaMalloc(&dSv, sizeof(double) * nmax * B));
    CK(cudaMalloc(&dPerm, sizeof(int32_t) * nmax * B));
    CK(cudaMalloc(&dK, sizeof(int32_t) * B));
    CK(cudaMalloc(&dN, sizeof(int32_t) * B));
    CK(cudaMalloc(&dLogp, sizeof(double) * B));
    CK(cudaMalloc(&dDisc, sizeof(double) * B));
    CK(cudaMalloc(&dTies, sizeof(int32_t) * B));
    CK(cudaMalloc(&dRec, (size_t)c.n_rec * B));
    CK(cudaMalloc(&dLast, (size_t)c.N * B));
    CK(cudaMalloc(&dTheta, sizeof(double) * B));
    CK(cudaMalloc(&dGamma, sizeof(double) * B));
    CK(cudaMalloc(&dTraj, sizeof(uint64_t) * B));
    CK(cudaMalloc(&dErr, sizeof(int32_t) * B));
    CK(cudaMalloc(&dErrStep, sizeof(int32_t) * 2 * B));
    CK(cudaMalloc(&dFrob, sizeof(double) * B));
    CK(cudaMalloc(&dTrunc, sizeof(int32_t) * B));
    CK(cudaMalloc(&dChoice, (size_t)std::max(1, c.n_events) * B));
    // the ledger is always kept (one atomic add per kernel and trajectory);
    // collect_profile hands it to an active profile and clears it
    CK(cudaMalloc(&dLedger, sizeof(unsigned long long) * LEDGER_WORDS));
    CK(cudaMemset(dLedger, 0, sizeof(unsigned long long) * LEDGER_WORDS));
    CK(cudaMalloc(&dLeafdim, sizeof(int32_t) * c.L));
    CK(cudaMalloc(&dOp1, sizeof(Op1) * std::max<size_t>(1, prog.op1.size())));
    CK(cudaMalloc(&dGroups, sizeof(Group1) * std::max<size_t>(1, prog.groups.size())));
    CK(cudaMemcpy(dOff, off.data(), sizeof(int64_t) * c.L, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dOff + c.L, ncap.data(), sizeof(int64_t) * c.L, cudaMemcpyHostToDevice));
    std::vector<int32_t> leafdim(c.L, 1);
    for (int q = 0; q < c.N; ++q) leafdim[c.leaf_of_qubit[q]] = 2;
    CK(cudaMemcpy(dLeafdim, leafdim.data(), sizeof(int32_t) * c.L, cudaMemcpyHostToDevice));
    if (!prog.op1.empty())
      CK(cudaMemcpy(dOp1, prog.op1.data(), sizeof(Op1) * prog.op1.size(), cudaMemcpyHostToDevice));
    if (!prog.groups.empty())
      CK(cudaMemcpy(dGroups, prog.groups.data(), sizeof(Group1) * prog.groups.size(),
                    cudaMemcpyHostToDevice));
    dev.T = dT;
    dev.off = dOff;
    dev.ncap = dOff + c.L;
    dev.tstride = tstride;
    dev.dims = dDims;
    dev.ds = 2 * c.L;
    dev.W = dW;
    dev.wstride = wstride;
    dev.V = dV;
    dev.Rm = dR;
    dev.G = dG;
    dev.Ts = dTs;
    dev.vstride = vstride;
    dev.sv = dSv;
    dev.perm = dPerm;
    dev.nmax = nmax;
    dev.knew = dK;
    dev.nold = dN;
    dev.logp = dLogp;
    dev.disc = dDisc;
    dev.ties = dTies;
    dev.rec = dRec;
    dev.n_rec = c.n_rec;
    dev.last = dLast;
    dev.N = c.N;
    dev.theta = dTheta;
    dev.gamma = dGamma;
    dev.traj = dTraj;
    dev.L = c.L;
    dev.chi = chi;
    dev.noise = noise;
    dev.err = dErr;
    dev.err_step = dErrStep;
    dev.frob = dFrob;
    dev.trunc = dTrunc;
    dev.ledger = dLedger;
    dev.choice = dChoice;
    dev.n_events = std::max(1, c.n_events);
    dev.forced = 0;
    dev.shape = nullptr;
    dev.eig_nsplit = 0;
    if (mixed) {
      const size_t cs = 2 * (size_t)nmax;
      CK(cudaMalloc(&dShape, sizeof(int2) * B));
      CK(cudaMalloc(&dAmax, sizeof(unsigned) * cs * B));
      CK(cudaMalloc(&dExpo, sizeof(int) * cs * B));
      CK(cudaMalloc(&dSlices, sizeof(uint16_t) * (size_t)sstride * B));
      CK(cudaMalloc(&dCExpo, sizeof(int) * (size_t)crows * B));
      CK(cudaMalloc(&dGfix, sizeof(unsigned long long) * cs * cs * B));
      CK(cudaMalloc(&dG64, sizeof(cx<double>) * (size_t)vstride * B));
      CK(cudaMalloc(&dV64, sizeof(cx<double>) * (size_t)vstride * B));
      CK(cudaMalloc(&dTs64, sizeof(cx<double>) * (size_t)vstride * 2 * B));
      // the Gram kernels leave these zero after every matrix
      CK(cudaMemset(dAmax, 0, sizeof(unsigned) * cs * B));
      CK(cudaMemset(dGfix, 0, sizeof(unsigned long long) * cs * cs * B));
      dev.shape = dShape;
      gargs.M = reinterpret_cast<const float2*>(dW);
      gargs.mstride = wstride;
      gargs.shape = dShape;
      gargs.amax = dAmax;
      gargs.expo = dExpo;
      gargs.cstride = (int)cs;
      gargs.slices = dSlices;
      gargs.sstride = sstride;
      gargs.gfix = dGfix;
      gargs.gld = (int)cs;
      gargs.G = reinterpret_cast<double2*>(dG64);
      gargs.g64stride = vstride;
      gargs.err = dErr;
      gargs.ledger = dLedger;
      gargs.ledger_class = KC_GRAM;
    }
    base = dev;
    gbase = gargs;
    b0 = 0;
    return TTN_OK;
  }

  // The FP64 eigensolvers' view of the batch (MIXED runs): the exact Gram
  // matrices and FP64 scratch in place of the FP32 ones; bond dimensions,
  // singular values, kept ranks and flags shared with the FP32 state.
  Dev<double> view64() const {
    Dev<double> v{};
    v.off = dev.off;
    v.ncap = dev.ncap;
    v.tstride = dev.tstride;
    v.dims = dev.dims;
    v.ds = dev.ds;
    v.wstride = dev.wstride;
    v.G = dG64 + b0 * vstride;
    v.V = dV64 + b0 * vstride;
    v.Ts = dTs64 + b0 * 2 * vstride;
    v.vstride = dev.vstride;
    v.sv = dev.sv;
    v.perm = dev.perm;
    v.nmax = dev.nmax;
    v.knew = dev.knew;
    v.nold = dev.nold;
    v.logp = dev.logp;
    v.disc = dev.disc;
    v.ties = dev.ties;
    v.n_rec = dev.n_rec;
    v.N = dev.N;
    v.L = dev.L;
    v.chi = dev.chi;
    v.noise = dev.noise;
    v.eps_gram = eps_mixed;
    v.tol_gram = 1e-13;
    v.tol_abs_gram = 1e-15;
    v.max_sweeps = 40;
    v.ledger = dev.ledger;
    v.frob = dev.frob;
    v.trunc = dev.trunc;
    v.err = dev.err;
    v.err_step = dev.err_step;
    v.cur_step = dev.cur_step;
    v.cur_trunc = dev.cur_trunc;
    v.svd_mode = 2;
    return v;
  }

  void release() {
    void* ptrs[] = {dT, dW, dV, dR, dG, dTs, dOff, dDims, dSv, dPerm, dK, dN, dLogp, dDisc, dTies, dRec,
                    dLast, dTheta, dGamma, dTraj, dErr, dErrStep, dFrob, dTrunc, dLeafdim, dOp1, dGroups,
                    dLedger, dChoice, dShape, dAmax, dExpo, dSlices, dGfix, dG64, dV64, dTs64, dCExpo};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }

  // Launch the step program for trajectories [0, nb) of the batch.
  ttn_status launch(int nb, int stop_step) {
    return launch_range(nb, 0, stop_step < 0 ? (int)prog.steps.size() : stop_step);
  }

  // Trajectories [b0, b0 + nb) of the batch on stream s: every later launch
  // sees only that group (per-trajectory pointers shifted by b0).
  void select_group(int64_t b0_, cudaStream_t s) {
    b0 = b0_;
    st = s;
    dev = base;
    Dev<R>& x = dev;
    x.T += b0 * tstride;
    x.dims += b0 * x.ds;
    x.W += b0 * wstride;
    x.V += b0 * vstride;
    x.Rm += b0 * vstride;
    x.G += b0 * vstride;
    x.Ts += b0 * 2 * vstride;
    x.sv += b0 * nmax;
    x.perm += b0 * nmax;
    x.knew += b0;
    x.nold += b0;
    x.logp += b0;
    x.disc += b0;
    x.ties += b0;
    x.rec += b0 * c.n_rec;
    x.last += b0 * c.N;
    x.theta += b0;
    x.gamma += b0;
    x.traj += b0;
    x.choice += b0 * x.n_events;
    x.frob += b0;
    x.trunc += b0;
    x.err += b0;
    x.err_step += 2 * b0;
    if (x.shape) x.shape += b0;
    if (mixed) {
      gargs = gbase;
      gargs.M += b0 * gbase.mstride;
      gargs.shape += b0;
      gargs.amax += b0 * gbase.cstride;
      gargs.expo += b0 * gbase.cstride;
      gargs.slices += b0 * gbase.sstride;
      gargs.gfix += b0 * (int64_t)gbase.gld * gbase.gld;
      gargs.G += b0 * gbase.g64stride;
      gargs.err += b0;
    }
  }

  // Operands of the exact tensor-core contractions of the move v -> w for
  // the selected group (MIXED runs).
  ContractArgs contract_args(int v, int w) const {
    ContractArgs a{};
    a.dims = dev.dims;
    a.ds = dev.ds;
    a.v = v;
    a.w = w;
    a.leg_v = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
    a.leg_w = (v == 2 * w) ? 0 : ((v == 2 * w + 1) ? 1 : 2);
    a.nold = dev.nold;
    a.knew = dev.knew;
    a.M = reinterpret_cast<const float2*>(dev.W);
    a.mstride = dev.wstride;
    a.V = reinterpret_cast<const float2*>(dev.G);
    a.Rm = reinterpret_cast<const float2*>(dev.Rm);
    a.vstride = dev.vstride;
    a.T = reinterpret_cast<float2*>(dev.T);
    a.tstride = dev.tstride;
    a.off_v = off[v];
    a.off_w = off[w];
    a.W = reinterpret_cast<float2*>(dev.W);
    a.wstride = dev.wstride;
    a.slices = dSlices + b0 * sstride;
    a.sstride = sstride;
    a.expo = dCExpo + b0 * crows;
    a.rows_cap = crows;
    a.err = dev.err;
    a.ledger = dev.ledger;
    a.ledger_form = KC_FORMU;
    a.ledger_absorb = KC_ABSORB;
    return a;
  }

  // Steps [s0, s1) of the program for the selected group's first nb
  // trajectories; s0 == 0 starts them from |0...0>.
  ttn_status launch_range(int nb, int s0, int s1) {
    const int L = c.L;
    if (s0 == 0) {
      dev.cur_step = -1;
      k_init<R><<<dim3(std::max(1, ceil_div(2 * L, 256)), nb), 256, 0, st>>>(dev, dLeafdim, nb);
      CK(cudaGetLastError());
      kernel_launches += 1;
    }
    const int nsteps = std::min<int>(s1, (int)prog.steps.size());
    for (int si = s0; si < nsteps; ++si) {
      const Step& s = prog.steps[si];
      dev.cur_step = si;
      dev.cur_trunc = s.kind == S_MOVE ? s.c : 0;
      switch (s.kind) {
        case S_MOVE: {
          const int v = s.a, w = s.b;
          const int bond = (w == v / 2) ? v : w;
          const int64_t nmv = 2 * (int64_t)bcap[bond];
          // largest rank this move may keep: the bond's structural cap
          // (min(chi, 2^{qubits on the smaller side})) on truncating moves,
          // twice that while a gate's operator index rides on the bond.  In
          // FP32 the Gram matrix's rounding puts spurious singular values
          // near 1e-3 s_max, above the kept-rank floor; without this cap they
          // would keep small bonds above their structural rank and the next
          // gate would grow the node past its slot.
          const int kcap = s.c ? bcap[bond] : 2 * bcap[bond];
          // FP32 auto: the Gram path for bonds above 64 and for every move of a
          // large tensor (there the one-sided Jacobi's FP32 orthogonality test
          // is not reachable and its iteration stalls); FP64 auto: Jacobi.
          const int lv0 = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
          const int64_t cc3[3] = {2 * (int64_t)bcap[2 * v], 2 * (int64_t)bcap[2 * v + 1],
                                  v == 1 ? 1 : 2 * (int64_t)bcap[v]};
          int64_t mcap = 1;
          for (int t = 0; t < 3; ++t)
            if (t != lv0) mcap *= cc3[t];
          const bool big = c.N > BIG_CIRCUIT_QUBITS || mcap * nmv >= BIG_MOVE;
          const bool gram = mixed || dev.svd_mode >= 2 || (dev.svd_mode == 0 && sizeof(R) == 4 && (nmv > 64 || big));
          // contractions of this move on the tensor cores (FP32 only).
          // MIXED: the FMA units by default (0, 1); gemm_mode 3 the digit
          // products on tcgen05 (contract.cu), 2 the mma.sync 3xTF32 tile
          // (whose truncating FP32 accumulation costs ~1e-5 of amplitude
          // accuracy over a syndrome round).  In the pipelined d=7 batch the
          // tcgen05 route runs 3 % slower than the FMA kernels and is not
          // more accurate (its inputs are rounded relative to row maxima).
          const bool exact_c = mixed && gemm_mode == 3;
          const bool tc = sizeof(R) == 4 && (gemm_mode == 2 || (gemm_mode == 0 && gram && !mixed));
          if (gram) {
            const int lv = (w == 2 * v) ? 0 : ((w == 2 * v + 1) ? 1 : 2);
            int64_t c3[3] = {2 * (int64_t)bcap[2 * v], 2 * (int64_t)bcap[2 * v + 1],
                             v == 1 ? 1 : 2 * (int64_t)bcap[v]};
            int64_t mmax = 1;
            for (int t = 0; t < 3; ++t)
              if (t != lv) mmax *= c3[t];
            timed(KC_COPY, [&] { k_gather_rows<R><<<dim3(std::max(1, ceil_div(ncap[v], 1024)), nb), 256, 0, st>>>(dev, v, w); });
            const int tn = std::max(1, ceil_div(nmv, 64));
            if (mixed) {
              // exact Gram matrix on the tensor cores, FP64 eigensolver
              timed(KC_GRAM, 5, [&] { (void)gram_exact_launch(gargs, nb, (int)nmv, std::min<int64_t>(mmax, ncap[v]), st); });
              // the solver is chosen per trajectory by its bond's actual
              // dimension: cyclic Jacobi in shared memory up to EIG_JACOBI_N,
              // the tridiagonal solver above (each kernel skips the others)
              const bool both = nmv > EIG_JACOBI_N;
              timed(KC_EIG, (sizeof(R) == 4 ? 1 : 0) + (both ? 2 : 1), [&] {
                Dev<double> dv = view64();
                dv.eig_nsplit = EIG_JACOBI_N;
                dv.eig_smem_bytes = EIG_JACOBI_N * EIG_JACOBI_N * (int)sizeof(cx<double>);
                dv.defer_bt = sizeof(R) == 4 ? 1 : 0;
                if (!both) {
                  k_eig<double><<<nb, 512, dv.eig_smem_bytes, st>>>(dv, v, w, kcap);
                } else {
                  // one launch per move: the tridiagonal kernel runs the
                  // Jacobi body itself for the trajectories whose bond is at
                  // most EIG_JACOBI_N (an idle second launch would still wait
                  // for a slot on a busy SM).  A bond up to 256 fits 256
                  // threads (one per eigenvalue), leaving room for a second
                  // CTA on the SM.
                  const int smem = std::max(dv.eig_smem_bytes, dv.defer_bt ? tri_smem_bytes_nobt<double>()
                                                                             : tri_smem_bytes<double>());
                  k_eig_tri<double><<<nb, nmv <= 256 ? 256 : 512, smem, st>>>(dv, v, w, kcap);
                }
                if constexpr (sizeof(R) == 4) {
                  k_vk_to_float<<<nb, 256, 0, st>>>(dev, dG64 + b0 * vstride, EIG_JACOBI_N);
                  if (both)
                    k_eig_bt<<<dim3((unsigned)ceil_div(std::min<int64_t>(kcap, nmv), BT_COLS), nb), 256,
                               bt_smem_bytes((int)std::min<int64_t>(nmv, 512)), st>>>(dev, dv);
                }
              });
            } else {
            timed(KC_GRAM, [&] {
              if (tc) k_gram<R, true><<<dim3(tn, tn, nb), 256, 0, st>>>(dev, v, w);
              else k_gram<R, false><<<dim3(tn, tn, nb), 256, 0, st>>>(dev, v, w);
            });
            }
            if (mixed) {
              // eigendecomposition done above
            } else if (dev.svd_mode != 3 && !(dev.svd_mode == 0 && big) &&
                nmv * nmv * (int64_t)sizeof(cx<R>) <= EIG_SMEM_MAX) {
              dev.eig_smem_bytes = (int)(nmv * nmv * (int64_t)sizeof(cx<R>));
              timed(KC_EIG, [&] { k_eig<R><<<nb, 512, dev.eig_smem_bytes, st>>>(dev, v, w, kcap); });
            } else {
              timed(KC_EIG, [&] { k_eig_tri<R><<<nb, 512, tri_smem_bytes<R>(), st>>>(dev, v, w, kcap); });
            }
            if (exact_c) {
              timed(KC_FORMU, 3, [&] {
                (void)contract_form_launch(contract_args(v, w), nb, mmax, (int)nmv,
                                           (int)std::min<int64_t>(kcap, nmv), st);
              });
            } else {
            timed(KC_FORMU, [&] {
              const dim3 gf(std::max(1, ceil_div(mmax, 64)), tn, nb);
              if (tc) k_form_u<R, true><<<gf, 256, 0, st>>>(dev, v, w);
              else k_form_u<R, false><<<gf, 256, 0, st>>>(dev, v, w);
            });
            }
            timed(KC_OTHER, 4, [&] {
              const int gx = (int)std::min<int64_t>(std::max<int64_t>(1, mmax * nmv / 4096), 512);
              k_unorm_zero<R><<<nb, 256, 0, st>>>(dev, nb);
              k_unorm_sums<R><<<dim3(gx, nb), 256, 0, st>>>(dev, v, w);
              k_unorm_scale<R><<<ceil_div(nb, 128), 128, 0, st>>>(dev, v, w, nb);
              k_unorm_apply<R><<<dim3(gx, nb), 256, 0, st>>>(dev, v, w);
            });
          } else {
            timed(KC_SVD, [&] { k_svd_move<R><<<nb, 256, 0, st>>>(dev, v, w, kcap); });
          }
          // neighbour absorbs R: grid from capacities
          const int lw = (v == 2 * w) ? 0 : ((v == 2 * w + 1) ? 1 : 2);
          int64_t cl = 2 * (int64_t)bcap[2 * w], cr = 2 * (int64_t)bcap[2 * w + 1],
                  cu = w == 1 ? 1 : 2 * (int64_t)bcap[w];
          int64_t kmax = lw == 0 ? cl : (lw == 1 ? cr : cu);
          int64_t Jmax = ncap[w] * 2 / std::max<int64_t>(1, kmax);
          Jmax = std::min<int64_t>(Jmax, (lw == 0 ? cr * cu : (lw == 1 ? cl * cu : cl * cr)));
          dim3 ga(std::max(1, ceil_div(Jmax, 64)), std::max(1, ceil_div(kmax, 64)), nb);
          if (exact_c && gram) {
            timed(KC_ABSORB, 3, [&] {
              (void)contract_absorb_launch(contract_args(v, w), nb, (int)nmv, (int)std::min<int64_t>(kcap, nmv),
                                           Jmax, st);
            });
          } else {
          timed(KC_ABSORB, [&] {
            if (tc) k_absorb<R, true><<<ga, 256, 0, st>>>(dev, w, v);
            else k_absorb<R, false><<<ga, 256, 0, st>>>(dev, w, v);
          });
          }
          timed(KC_COPY, [&] { k_copy_back<R><<<dim3(std::max(1, ceil_div(ncap[w], 256 * 4)), nb), 256, 0, st>>>(dev, w); });
          break;
        }
        case S_THREAD_LEAF: {
          timed(KC_LOCAL, 2, [&] {
            k_thread_leaf<R><<<dim3(std::max(1, ceil_div(ncap[s.a], 256)), nb), 256, 0, st>>>(
                dev, s.a, s.b, s.c);
            k_thread_dims_leaf<R><<<ceil_div(nb, 128), 128, 0, st>>>(dev, s.a, nb);
          });
          timed(KC_COPY, [&] {
            k_copy_back<R><<<dim3(std::max(1, ceil_div(ncap[s.a], 256 * 4)), nb), 256, 0, st>>>(dev, s.a);
          });
          break;
        }
        case S_THREAD_NODE: {
          timed(KC_LOCAL, 2, [&] {
            k_thread_node<R><<<dim3(std::max(1, ceil_div(ncap[s.a], 256)), nb), 256, 0, st>>>(
                dev, s.a, s.b);
            // same dims update as the leaf step: only the node's up bond
            // doubles here (its child bond doubled when the child was threaded)
            k_thread_dims_leaf<R><<<ceil_div(nb, 128), 128, 0, st>>>(dev, s.a, nb);
          });
          timed(KC_COPY, [&] {
            k_copy_back<R><<<dim3(std::max(1, ceil_div(ncap[s.a], 256 * 4)), nb), 256, 0, st>>>(dev, s.a);
          });
          break;
        }
        case S_THREAD_LCA: {
          timed(KC_LOCAL, [&] {
            k_thread_lca<R><<<dim3(std::max(1, ceil_div(ncap[s.a], 256)), nb), 256, 0, st>>>(dev, s.a);
          });
          timed(KC_COPY, [&] {
            k_copy_back<R><<<dim3(std::max(1, ceil_div(ncap[s.a], 256 * 4)), nb), 256, 0, st>>>(dev, s.a);
          });
          break;
        }
        case S_GATE_NODE:
          timed(KC_LOCAL, [&] {
            k_gate_node<R><<<ceil_div((int64_t)nb * 64, 256), 256, 0, st>>>(dev, s.a, s.b, nb);
          });
          break;
        case S_LAYER1Q: {
          const int ng = s.d - s.c;
          timed(KC_LOCAL, [&] {
            k_layer1q<R><<<ceil_div((int64_t)nb * ng, 128), 128, 0, st>>>(dev, dOp1, dGroups, s.c, ng, nb);
          });
          break;
        }
        case S_MEASURE:
          timed(KC_LOCAL, [&] {
            k_measure<R><<<ceil_div(nb, 4), 128, 0, st>>>(dev, s.a, s.b, s.c, s.d,
                                                          L + c.leaf_of_qubit[s.a], nb);
          });
          break;
        case S_AD:
          timed(KC_LOCAL, [&] {
            k_ad<R><<<ceil_div(nb, 4), 128, 0, st>>>(dev, s.a, s.b, L + c.leaf_of_qubit[s.a], nb);
          });
          break;
      }
    }
    CK(cudaGetLastError());
    return TTN_OK;
  }
};

// Numerical settings of an engine from a request (precision-dependent
// tolerances, eigensolver shared-memory limits).
template <typename R>
static ttn_status configure(Engine<R>& eng, const RunRequest& rq) {
  eng.dev.seed = rq.seed;
  eng.dev.eps = rq.svd_eps;
  eng.dev.tie_eps = sizeof(R) == 8 ? 1e-9 : 1e-5;
  eng.dev.tol = sizeof(R) == 8 ? 1e-15 : 1e-7;
  eng.dev.max_sweeps = sizeof(R) == 8 ? 40 : 30;
  eng.dev.svd_mode = rq.svd_mode;
  eng.gemm_mode = rq.gemm_mode;
  eng.dev.eig_smem_bytes = 0;
  eng.mixed = rq.precision == TTN_PREC_MIXED;
  eng.eps_mixed = rq.svd_eps > 0 ? rq.svd_eps : 1e-6;
  CK(cudaFuncSetAttribute(k_eig<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, EIG_SMEM_MAX));
  CK(cudaFuncSetAttribute(k_eig_tri<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, tri_smem_bytes<R>()));
  if (eng.mixed) {
    CK(cudaFuncSetAttribute(k_eig_bt, cudaFuncAttributeMaxDynamicSharedMemorySize, bt_smem_bytes()));
    CK(cudaFuncSetAttribute(k_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, EIG_SMEM_MAX));
    CK(cudaFuncSetAttribute(k_eig_tri<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            tri_smem_bytes<double>()));
  }
  eng.dev.eps_gram = sizeof(R) == 8 ? 1e-7 : 1e-4;
  eng.dev.tol_gram = sizeof(R) == 8 ? 1e-13 : 3e-6;
  eng.dev.tol_abs_gram = sizeof(R) == 8 ? 1e-15 : 2e-7;
  return TTN_OK;
}

template <typename R>
static ttn_status run_impl(const ttn_circuit& c, const RunRequest& rq, RunOutputs& out) {
  Program prog = compile_program(c, rq.noise, -1);
  cudaStream_t st = (cudaStream_t)rq.stream;
  Engine<R> eng(c, prog, rq.chi, rq.noise, st);
  ttn_status cs = configure(eng, rq);
  if (cs != TTN_OK) return cs;
  size_t freeb = 0, totb = 0;
  CK(cudaMemGetInfo(&freeb, &totb));
  const size_t per = eng.bytes_per_traj();
  size_t budget = (size_t)((double)freeb * 0.80);
  if (rq.max_device_bytes > 0) budget = std::min(budget, rq.max_device_bytes);
  int64_t Bmax = (int64_t)(budget / per);
  if (Bmax < 1) {
    set_error("one trajectory needs " + std::to_string(per) + " device bytes; " +
              std::to_string(budget) + " available");
    return TTN_ENOMEM;
  }
  Bmax = std::min<int64_t>(Bmax, (int64_t)rq.n_traj);
  if (rq.max_batch > 0) Bmax = std::min<int64_t>(Bmax, rq.max_batch);
  Bmax = std::min<int64_t>(Bmax, 32768);
  ttn_status stt = eng.alloc((int)Bmax);
  if (stt != TTN_OK) {
    eng.release();
    return stt;
  }
  out.batch = (int)Bmax;
  out.bytes_per_traj = per;
  std::vector<double> th(Bmax), ga(Bmax);
  std::vector<uint64_t> tj(Bmax);
  std::vector<int32_t> err(Bmax);
  int stop = -1;
  if (rq.debug_amps) stop = rq.last_layer < 0 ? 0 : prog.stop_step_of_layer[rq.last_layer];
  for (uint64_t t0 = 0; t0 < rq.n_traj; t0 += Bmax) {
    const int nb = (int)std::min<uint64_t>(Bmax, rq.n_traj - t0);
    for (int i = 0; i < nb; ++i) {
      th[i] = rq.theta_per_traj ? rq.theta_per_traj[t0 + i] : rq.theta;
      ga[i] = rq.gamma_per_traj ? rq.gamma_per_traj[t0 + i] : rq.gamma;
      tj[i] = rq.first_traj + t0 + i;
    }
    CK(cudaMemcpyAsync(eng.dTheta, th.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(eng.dGamma, ga.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(eng.dTraj, tj.data(), sizeof(uint64_t) * nb, cudaMemcpyHostToDevice, st));
    ttn_status s2 = eng.launch(nb, stop);
    if (s2 != TTN_OK) {
      eng.release();
      return s2;
    }
    // decode on the device (full circuits only)
    if (!rq.debug_amps && out.fail) {
      s2 = decode_device(c, nb, eng.dRec, out.fail + t0, nullptr, nullptr, st, out.on_device);
      if (s2 == TTN_EOVERFLOW) {
        out.decode_overflow += 1;
      } else if (s2 != TTN_OK) {
        eng.release();
        return s2;
      }
    }
    auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
      return cudaMemcpyAsync(dst, src, bytes,
                             out.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    };
    if (out.records) CK(cp(out.records + t0 * c.n_rec, eng.dRec, (size_t)nb * c.n_rec));
    if (out.log_prob) CK(cp(out.log_prob + t0, eng.dLogp, sizeof(double) * nb));
    if (out.discarded) CK(cp(out.discarded + t0, eng.dDisc, sizeof(double) * nb));
    if (out.near_ties) CK(cp(out.near_ties + t0, eng.dTies, sizeof(int32_t) * nb));
    CK(cudaMemcpyAsync(err.data(), eng.dErr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> err_step(2 * nb, -1);
    CK(cudaMemcpyAsync(err_step.data(), eng.dErrStep, sizeof(int32_t) * 2 * nb, cudaMemcpyDeviceToHost, st));
    // score of each trajectory: replay its choices at strength +- h
    if (rq.grad_wrt >= 0 && !rq.debug_amps) {
      std::vector<double> lp(nb), lm(nb);
      for (int sgn = 0; sgn < 2; ++sgn) {
        const double dh = sgn == 0 ? rq.grad_h : -rq.grad_h;
        for (int i = 0; i < nb; ++i) {
          if (rq.grad_wrt == 0) th[i] += dh;
          else ga[i] += dh;
        }
        CK(cudaMemcpyAsync(eng.dTheta, th.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(eng.dGamma, ga.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st));
        // keep the forward records: the replay writes the same bits
        eng.dev.forced = 1;
        ttn_status s3 = eng.launch(nb, stop);
        eng.dev.forced = 0;
        if (s3 != TTN_OK) {
          eng.release();
          return s3;
        }
        CK(cudaMemcpyAsync(sgn == 0 ? lp.data() : lm.data(), eng.dLogp, sizeof(double) * nb,
                           cudaMemcpyDeviceToHost, st));
        for (int i = 0; i < nb; ++i) {
          if (rq.grad_wrt == 0) th[i] -= dh;
          else ga[i] -= dh;
        }
      }
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i < nb; ++i) out.score[t0 + i] = (lp[i] - lm[i]) / (2.0 * rq.grad_h);
    }
    if (rq.debug_amps) {
      std::vector<int32_t> qol(c.L, -1);
      for (int q = 0; q < c.N; ++q) qol[c.leaf_of_qubit[q]] = q;
      int32_t* dq = nullptr;
      double* da = nullptr;
      const size_t na = (size_t)1 << c.N;
      CK(cudaMalloc(&dq, sizeof(int32_t) * c.L));
      CK(cudaMalloc(&da, sizeof(double) * 2 * na));
      CK(cudaMemcpyAsync(dq, qol.data(), sizeof(int32_t) * c.L, cudaMemcpyHostToDevice, st));
      k_amplitudes<R><<<ceil_div(na, 64), 64, 0, st>>>(eng.dev, 0, dq, c.N, da);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(rq.debug_amps, da, sizeof(double) * 2 * na, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      cudaFree(dq);
      cudaFree(da);
    }
    CK(cudaStreamSynchronize(st));
    eng.collect_profile();
    for (int i = 0; i < nb; ++i) out.err_flags |= err[i];
    // Every error is fatal: a trajectory whose state lost its norm or became
    // non-finite cannot be left out of p_L without biasing it (the loss
    // depends on the state), so the run stops and names it.
    const bool fatal = (out.err_flags & (ERR_CAPACITY | ERR_ZERO_NORM | ERR_NAN | GRAM_ERR_TIMEOUT)) != 0;
    if (fatal) {
      // first failing trajectory: which step of the program raised it
      std::string where;
      for (int i = 0; i < nb; ++i)
        if (err[i] & (ERR_CAPACITY | ERR_ZERO_NORM | ERR_NAN | GRAM_ERR_TIMEOUT)) {
          static const char* kinds[] = {"move", "thread-leaf", "thread-node", "thread-lca",
                                        "gate-node", "single-qubit layer", "measure", "damping"};
          where = " (trajectory " + std::to_string(rq.first_traj + t0 + i) + ", flags " + std::to_string(err[i]);
          for (int which = 0; which < 2; ++which) {
            const int si = err_step[2 * i + which];
            if (si >= 0 && si < (int)prog.steps.size()) {
              const Step& s = prog.steps[si];
              where += std::string(which ? "; first non-convergence" : "") + ", step " + std::to_string(si) +
                       " " + kinds[s.kind] + " a=" + std::to_string(s.a) + " b=" + std::to_string(s.b);
            }
          }
          where += ")";
          break;
        }
      eng.release();
      const int f = out.err_flags;
      set_error(std::string("engine: ") +
                ((f & GRAM_ERR_TIMEOUT) ? "a bounded wait of the tensor-core Gram kernel expired"
                 : (f & ERR_CAPACITY) ? "tensor exceeded its slot capacity"
                 : (f & ERR_NAN) ? "non-finite value in a centre move" : "zero-norm state") + where);
      if (f & GRAM_ERR_TIMEOUT) return TTN_ETIMEOUT;
      if (f & ERR_CAPACITY) return TTN_ECUDA;
      return TTN_ENUMERIC;
    }
  }
  eng.release();
  return TTN_OK;
}

size_t run_bytes_per_traj(const ttn_circuit& c, const RunRequest& rq) {
  Program prog = compile_program(c, rq.noise, -1);
  if (rq.precision == TTN_PREC_FP64) return Engine<double>(c, prog, rq.chi, rq.noise, nullptr).bytes_per_traj();
  Engine<float> e(c, prog, rq.chi, rq.noise, nullptr);
  e.mixed = rq.precision == TTN_PREC_MIXED;
  return e.bytes_per_traj();
}

// Worst case of the node-slot fill over the step program: every move keeps
// the largest rank its kernels allow, min(n, cap) for an m x n matrix (cap =
// the bond's structural cap on truncating moves and twice that otherwise, as
// S_MOVE launches it; rounding can keep more than the exact rank min(m, n):
// an FP32 Gram matrix turns the n - m zero eigenvalues of a wide M into
// values near the kept-rank floor), threading doubles bonds as its kernels
// do, and every node's element count is compared with its slot after each
// step, as are the workspaces each step uses (W, the n x n blocks, the
// n-entry arrays).  fill <= 1 means no trajectory can overflow a slot or a
// workspace, whatever its rounding.  binding counts truncating moves whose structural cap is below
// chi and below n: there a cap at chi alone would keep more.
void slot_check(const ttn_circuit& c, int noise, int chi, double* worst_fill, int* worst_node,
                int* worst_step, int64_t* binding) {
  Program prog = compile_program(c, noise, -1);
  Engine<float> eng(c, prog, chi, noise, nullptr);  // capacities only
  const int L = c.L;
  std::vector<int64_t> D(2 * L, 1);
  for (int q = 0; q < c.N; ++q) D[L + c.leaf_of_qubit[q]] = 2;
  auto size = [&](int v) { return D[2 * v] * D[2 * v + 1] * (v == 1 ? 1 : D[v]); };
  double wf = 0.0;
  int wn = -1, ws = -1;
  int64_t nb = 0;
  auto check = [&](int v, int si) {
    const double f = (double)size(v) / (double)eng.ncap[v];
    if (f > wf) wf = f, wn = v, ws = si;
  };
  // the per-trajectory workspaces a move or a threading step uses: W holds
  // the node or the m x n bond matrix, V / Rm / G an n x n block, sv and perm
  // n entries
  auto check_ws = [&](double f, int v, int si) {
    if (f > wf) wf = f, wn = v, ws = si;
  };
  for (int v = 1; v < L; ++v) check(v, -1);
  for (int si = 0; si < (int)prog.steps.size(); ++si) {
    const Step& s = prog.steps[si];
    switch (s.kind) {
      case S_THREAD_LEAF:
      case S_THREAD_NODE:
        D[s.a] *= 2;
        check(s.a, si);
        check_ws((double)size(s.a) / (double)eng.wstride, s.a, si);
        break;
      case S_THREAD_LCA:
        check(s.a, si);
        check_ws((double)size(s.a) / (double)eng.wstride, s.a, si);
        break;
      case S_MOVE: {
        const int v = s.a, w = s.b;
        const int bond = (w == v / 2) ? v : w;
        const int64_t n = D[bond], m = size(v) / n;  // M is m x n
        const int64_t cap = s.c ? eng.bcap[bond] : 2 * (int64_t)eng.bcap[bond];
        check_ws((double)(m * n) / (double)eng.wstride, v, si);
        check_ws((double)n / (double)eng.nmax, v, si);
        check_ws((double)(n * n) / (double)eng.vstride, v, si);
        if (s.c && eng.bcap[bond] < chi && n > eng.bcap[bond]) ++nb;
        D[bond] = std::min(n, cap);
        check(v, si);
        check(w, si);
        break;
      }
      default:
        break;
    }
  }
  *worst_fill = wf;
  *worst_node = wn;
  *worst_step = ws;
  *binding = nb;
}

ttn_status run_trajectories_device(const ttn_circuit& c, const RunRequest& rq, RunOutputs& out) {
  if (rq.precision == TTN_PREC_FP64) return run_impl<double>(c, rq, out);
  // FP32 and MIXED: complex64 tensors (MIXED adds the FP64 centre)
  return run_impl<float>(c, rq, out);
}

}  // namespace ttn

namespace ttn {

// ------------------------------------------------------------------ pipelined resident batch
// n_resident trajectories live on the device at once, in S groups of
// G = n_resident / S.  The step program is cut into S segments of about
// equal worst-case cost; group g holds trajectories that have run g segments
// when the pipeline starts, and every pipeline step runs one segment of
// every group, each group on its own stream.  The group that runs the last
// segment is decoded and restarts with the next G trajectory indices, so
// every step completes exactly G trajectories and all steps cost the same.
struct PipelineImpl {
  virtual ~PipelineImpl() {}
  virtual ttn_status step(uint8_t* fail, double* log_prob, double* discarded, uint64_t* traj,
                          int32_t* n_done, bool on_device, cudaStream_t caller) = 0;
  virtual int group_size() const = 0;
  virtual int segment_ms(double* ms) const = 0;
};

template <typename R>
struct PipelineT : PipelineImpl {
  const ttn_circuit& c;
  Program prog;
  RunRequest rq;
  Engine<R> eng;
  int B = 0, S = 0, G = 0;
  // program steps each group gets per turn of the interleaved launches
  // (TTN_PIPELINE_CHUNK, default 16)
  int chunk = 16;
  std::vector<int> seg;             // S + 1 step boundaries
  std::vector<int> phase;           // next segment of each group
  std::vector<uint64_t> first;      // first trajectory index of each group's trajectories
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev, ev_a, ev_b;  // ev_a / ev_b bracket each group's segment (timing)
  std::vector<int> timed_seg;               // segment each group ran in the last step
  std::vector<double> seg_ms;               // device time of each segment in the last step
  cudaEvent_t ev_start = nullptr;
  uint64_t next_traj = 0;
  std::vector<double> theta_cycle;
  double* h_theta = nullptr;        // pinned [B]
  double* h_gamma = nullptr;
  uint64_t* h_traj = nullptr;

  PipelineT(const ttn_circuit& cc, const RunRequest& r)
      : c(cc), prog(compile_program(cc, r.noise, -1)), rq(r), eng(cc, prog, r.chi, r.noise, nullptr) {
    if (const char* e = std::getenv("TTN_PIPELINE_CHUNK")) chunk = std::max(1, std::min(1 << 20, std::atoi(e)));
  }

  ~PipelineT() override {
    for (cudaStream_t x : streams) cudaStreamDestroy(x);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_a) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_b) cudaEventDestroy(e);
    if (ev_start) cudaEventDestroy(ev_start);
    if (h_theta) cudaFreeHost(h_theta);
    if (h_gamma) cudaFreeHost(h_gamma);
    if (h_traj) cudaFreeHost(h_traj);
    eng.release();
  }

  int group_size() const override { return G; }
  int segment_ms(double* ms) const override {
    for (int i = 0; i < S; ++i) ms[i] = seg_ms[i];
    return S;
  }

  ttn_status create(int n_resident, int n_segments, const double* cycle, int n_cycle, cudaStream_t caller) {
    S = n_segments;
    B = n_resident;
    G = B / S;
    next_traj = rq.first_traj;
    if (cycle && n_cycle > 0) theta_cycle.assign(cycle, cycle + n_cycle);
    ttn_status s = configure(eng, rq);
    if (s != TTN_OK) return s;
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    size_t budget = (size_t)((double)freeb * 0.85);
    if (rq.max_device_bytes > 0) budget = std::min(budget, rq.max_device_bytes);
    if (eng.bytes_per_traj() * (size_t)B > budget) {
      set_error("pipeline: " + std::to_string(B) + " resident trajectories need " +
                std::to_string(eng.bytes_per_traj() * (size_t)B) + " device bytes; " + std::to_string(budget) +
                " available");
      return TTN_ENOMEM;
    }
    s = eng.alloc(B);
    if (s != TTN_OK) return s;
    // segments of about equal worst-case cost (moves: Gram + eigensolver
    // of the capacity-sized bond matrix; other steps: one pass over a node)
    std::vector<double> cost(prog.steps.size(), 1.0);
    for (size_t i = 0; i < prog.steps.size(); ++i) {
      const Step& st = prog.steps[i];
      if (st.kind == S_MOVE) {
        const int v = st.a, w = st.b;
        const int bond = (w == v / 2) ? v : w;
        const double nmv = 2.0 * eng.bcap[bond];
        const double mm = (double)eng.ncap[v] / std::max(1.0, nmv);
        cost[i] = mm * nmv * nmv + 12.0 * nmv * nmv * nmv;
      } else if (st.kind == S_THREAD_LEAF || st.kind == S_THREAD_NODE || st.kind == S_THREAD_LCA) {
        cost[i] = (double)eng.ncap[st.a];
      }
    }
    double tot = 0.0;
    for (double x : cost) tot += x;
    seg.assign(S + 1, 0);
    double acc = 0.0;
    int k = 1;
    for (size_t i = 0; i < prog.steps.size() && k < S; ++i) {
      acc += cost[i];
      if (acc >= tot * k / S) seg[k++] = (int)i + 1;
    }
    for (; k < S; ++k) seg[k] = (int)prog.steps.size();
    seg[S] = (int)prog.steps.size();
    for (int i = 1; i <= S; ++i) seg[i] = std::max(seg[i], seg[i - 1]);
    streams.resize(S);
    ev.resize(S);
    ev_a.resize(S);
    ev_b.resize(S);
    timed_seg.assign(S, -1);
    seg_ms.assign(S, 0.0);
    for (int g = 0; g < S; ++g) {
      CK(cudaStreamCreateWithFlags(&streams[g], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ev[g], cudaEventDisableTiming));
      CK(cudaEventCreate(&ev_a[g]));
      CK(cudaEventCreate(&ev_b[g]));
    }
    CK(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
    CK(cudaMallocHost(&h_theta, sizeof(double) * B));
    CK(cudaMallocHost(&h_gamma, sizeof(double) * B));
    CK(cudaMallocHost(&h_traj, sizeof(uint64_t) * B));
    phase.assign(S, 0);
    first.assign(S, 0);
    // ramp-up: group g runs segments 0 .. g-1
    CK(cudaEventRecord(ev_start, caller));
    for (int g = 0; g < S; ++g) CK(cudaStreamWaitEvent(streams[g], ev_start, 0));
    for (int r = 0; r + 1 < S; ++r) {
      std::vector<int> gs;
      for (int g = r + 1; g < S; ++g) gs.push_back(g);
      s = run_segments(gs);
      if (s != TTN_OK) return s;
    }
    for (int g = 0; g < S; ++g) CK(cudaStreamSynchronize(streams[g]));
    s = check_errors();
    eng.collect_profile();
    return s;
  }

  ttn_status start_group(int g) {
    first[g] = next_traj;
    next_traj += (uint64_t)G;
    for (int i = 0; i < G; ++i) {
      const uint64_t t = first[g] + (uint64_t)i;
      h_traj[g * G + i] = t;
      h_theta[g * G + i] = theta_cycle.empty() ? rq.theta : theta_cycle[(size_t)(t % theta_cycle.size())];
      h_gamma[g * G + i] = rq.gamma;
    }
    cudaStream_t st = streams[g];
    CK(cudaMemcpyAsync(eng.dTraj + g * G, h_traj + g * G, sizeof(uint64_t) * G, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(eng.dTheta + g * G, h_theta + g * G, sizeof(double) * G, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(eng.dGamma + g * G, h_gamma + g * G, sizeof(double) * G, cudaMemcpyHostToDevice, st));
    return TTN_OK;
  }

  // Next segment of each group in `gs`, each on its own stream.  The groups'
  // launches are interleaved a few program steps at a time: a segment is tens
  // of thousands of launches, and a stream whose launch queue is full blocks
  // the host, so enqueueing one group's segment whole would hold back the
  // others until it had nearly finished.
  ttn_status run_segments(const std::vector<int>& gs) {
    std::vector<int> cur(gs.size()), end(gs.size());
    for (size_t i = 0; i < gs.size(); ++i) {
      const int g = gs[i];
      if (phase[g] == 0) {
        ttn_status s = start_group(g);
        if (s != TTN_OK) return s;
      }
      cur[i] = seg[phase[g]];
      end[i] = seg[phase[g] + 1];
      timed_seg[g] = phase[g];
      CK(cudaEventRecord(ev_a[g], streams[g]));
    }
    const int CHUNK = chunk;  // program steps per group per turn
    for (bool more = true; more;) {
      more = false;
      for (size_t i = 0; i < gs.size(); ++i) {
        if (cur[i] >= end[i]) continue;
        const int hi = std::min(end[i], cur[i] + CHUNK);
        eng.select_group((int64_t)gs[i] * G, streams[gs[i]]);
        ttn_status s = eng.launch_range(G, cur[i], hi);
        if (s != TTN_OK) return s;
        cur[i] = hi;
        more = more || cur[i] < end[i];
      }
    }
    for (int g : gs) {
      CK(cudaEventRecord(ev_b[g], streams[g]));
      phase[g] = (phase[g] + 1) % S;
    }
    return TTN_OK;
  }

  ttn_status run_segment(int g) { return run_segments(std::vector<int>{g}); }

  ttn_status check_errors() {
    std::vector<int32_t> err(B);
    CK(cudaMemcpy(err.data(), eng.dErr, sizeof(int32_t) * B, cudaMemcpyDeviceToHost));
    for (int i = 0; i < B; ++i) {
      const int f = err[i];
      if (!(f & (ERR_CAPACITY | ERR_ZERO_NORM | ERR_NAN | GRAM_ERR_TIMEOUT))) continue;
      const int g = i / G;
      set_error("pipeline: trajectory " + std::to_string(first[g] + (uint64_t)(i - g * G)) + ": " +
                ((f & GRAM_ERR_TIMEOUT) ? "a bounded wait of the tensor-core Gram kernel expired"
                 : (f & ERR_CAPACITY) ? "tensor exceeded its slot capacity"
                 : (f & ERR_NAN) ? "non-finite value in a centre move" : "zero-norm state"));
      if (f & GRAM_ERR_TIMEOUT) return TTN_ETIMEOUT;
      if (f & ERR_CAPACITY) return TTN_ECUDA;
      return TTN_ENUMERIC;
    }
    return TTN_OK;
  }

  ttn_status step(uint8_t* fail, double* log_prob, double* discarded, uint64_t* traj, int32_t* n_done,
                  bool on_device, cudaStream_t caller) override {
    CK(cudaEventRecord(ev_start, caller));
    int done = -1;
    std::vector<int> gs;
    for (int g = 0; g < S; ++g) {
      CK(cudaStreamWaitEvent(streams[g], ev_start, 0));
      if (phase[g] == S - 1) done = g;
      gs.push_back(g);
    }
    ttn_status s = run_segments(gs);
    if (s != TTN_OK) return s;
    cudaStream_t st = streams[done];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (log_prob) CK(cudaMemcpyAsync(log_prob, eng.dLogp + done * G, sizeof(double) * G, kind, st));
    if (discarded) CK(cudaMemcpyAsync(discarded, eng.dDisc + done * G, sizeof(double) * G, kind, st));
    int overflow = 0;
    if (fail) {
      s = decode_device(c, G, eng.dRec + (size_t)done * G * c.n_rec, fail, nullptr, nullptr, st, on_device);
      if (s == TTN_EOVERFLOW) overflow = 1;
      else if (s != TTN_OK) return s;
    }
    for (int g = 0; g < S; ++g) {
      CK(cudaEventRecord(ev[g], streams[g]));
      CK(cudaStreamWaitEvent(caller, ev[g], 0));
    }
    CK(cudaStreamSynchronize(caller));
    for (int g = 0; g < S; ++g) {
      float ms = 0.f;
      if (timed_seg[g] >= 0 && cudaEventElapsedTime(&ms, ev_a[g], ev_b[g]) == cudaSuccess)
        seg_ms[timed_seg[g]] = ms;
    }
    if (traj)
      for (int i = 0; i < G; ++i) traj[i] = first[done] + (uint64_t)i;
    if (n_done) *n_done = G;
    s = check_errors();
    eng.collect_profile();
    if (s != TTN_OK) return s;
    if (overflow) {
      set_error("decoder: shot(s) exceeded the matching bound (fail byte 2)");
      return TTN_EOVERFLOW;
    }
    return TTN_OK;
  }
};

ttn_status pipeline_create(const ttn_circuit& c, const RunRequest& rq, int n_resident, int n_segments,
                           const double* theta_cycle, int n_theta, void* stream, PipelineImpl** out) {
  PipelineImpl* p = nullptr;
  ttn_status s;
  if (rq.precision == TTN_PREC_FP64) {
    auto* q = new PipelineT<double>(c, rq);
    p = q;
    s = q->create(n_resident, n_segments, theta_cycle, n_theta, (cudaStream_t)stream);
  } else {
    auto* q = new PipelineT<float>(c, rq);
    p = q;
    s = q->create(n_resident, n_segments, theta_cycle, n_theta, (cudaStream_t)stream);
  }
  if (s != TTN_OK) {
    delete p;
    return s;
  }
  *out = p;
  return TTN_OK;
}

ttn_status pipeline_step(PipelineImpl* p, uint8_t* fail, double* log_prob, double* discarded, uint64_t* traj,
                         int32_t* n_done, bool on_device, void* stream) {
  return p->step(fail, log_prob, discarded, traj, n_done, on_device, (cudaStream_t)stream);
}

int pipeline_group_size(const PipelineImpl* p) { return p->group_size(); }
int pipeline_segment_ms(const PipelineImpl* p, double* ms) { return p->segment_ms(ms); }

void pipeline_free(PipelineImpl* p) { delete p; }

}  // namespace ttn

// ---------------------------------------------------------------- standalone Gram eigensolver
namespace ttn {

// Kept columns in descending order, zero-padded to kcap, and the descending
// singular values (square roots of the eigenvalues).  V_k is complex128
// (vin64) or complex64 (vin32, the multi-CTA back-transformation's output).
__global__ void k_eig_collect(Dev<double> d, const cx<float>* vin32, cx<double>* Vout, double* s, int32_t* kout,
                              int n, int kcap) {
  const int b = blockIdx.x;
  const int k = d.knew[b];
  const cx<double>* v64 = d.G + (int64_t)b * d.vstride;
  const cx<float>* v32 = vin32 ? vin32 + (int64_t)b * d.vstride : nullptr;
  const double* sv = d.sv + (int64_t)b * d.nmax;
  const int32_t* perm = d.perm + (int64_t)b * d.nmax;
  for (int idx = threadIdx.x; idx < n * kcap; idx += blockDim.x) {
    const int x = idx / kcap, c = idx - x * kcap;
    cx<double> z = {0.0, 0.0};
    if (c < k) {
      if (v32) z = {(double)v32[(int64_t)x * k + c].x, (double)v32[(int64_t)x * k + c].y};
      else z = v64[(int64_t)x * k + c];
    }
    Vout[(int64_t)b * n * kcap + idx] = z;
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) s[(int64_t)b * n + c] = k > 0 ? sv[perm[c]] : 0.0;
  if (threadIdx.x == 0) kout[b] = k;
}

}  // namespace ttn

extern "C" ttn_status ttn_eig_gram(const void* G, int32_t batch, int32_t n, int32_t kcap, int32_t route,
                                   double eps_keep, void* V, double* s, int32_t* k, void* cuda_stream) {
  using namespace ttn;
  const int64_t jac_max = (int64_t)EIG_SMEM_MAX / (int64_t)sizeof(cx<double>);
  if (!G || !V || !s || !k || batch < 1 || n < 1 || n > 512 || kcap < 1 || kcap > n || route < 0 ||
      route > 3 || !(eps_keep >= 0.0 && eps_keep < 1.0) || (route == 0 && (int64_t)n * n > jac_max)) {
    set_error("ttn_eig_gram: need device G [batch][n][n], V [batch][n][kcap], s [batch][n], k [batch]; "
              "1 <= kcap <= n <= 512 (n^2 <= 8192 for route 0), route 0..3, 0 <= eps_keep < 1");
    return TTN_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(G) & 15) || (reinterpret_cast<uintptr_t>(V) & 15)) {
    set_error("ttn_eig_gram: G and V must be 16-byte aligned");
    return TTN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // a slot holds n x n (and the deferred route's 2n phases and reflector scalars)
  const int64_t vs = std::max<int64_t>((int64_t)n * n, 2 * (int64_t)n), B = batch;
  Dev<double> d{};
  Dev<float> df{};
  d.ds = 4;
  d.vstride = vs;
  d.nmax = n;
  d.eps_gram = eps_keep;
  d.tol_gram = 1e-13;
  d.tol_abs_gram = 1e-15;
  d.max_sweeps = 40;
  d.defer_bt = route >= 2 ? 1 : 0;
  // route 3: bonds up to EIG_JACOBI_N by the Jacobi body inside the tridiagonal kernel
  d.eig_nsplit = route == 3 ? EIG_JACOBI_N : 0;
  d.eig_smem_bytes = route == 0   ? (int)(vs * (int64_t)sizeof(cx<double>))
                     : route == 3 ? EIG_JACOBI_N * EIG_JACOBI_N * (int)sizeof(cx<double>)
                                  : 0;
  df.vstride = vs;
  void* pool = nullptr;
  const size_t b_cx = sizeof(cx<double>) * (size_t)(vs * B);
  const size_t b_total = 4 * b_cx + sizeof(cx<float>) * (size_t)(vs * B) + (sizeof(double) + sizeof(int32_t)) * n * B +
                         sizeof(int32_t) * (size_t)B * (d.ds + 6) + sizeof(double) * B + 4096;
  cudaError_t e = cudaMalloc(&pool, b_total);
  if (e == cudaSuccess) {
    unsigned char* p = static_cast<unsigned char*>(pool);
    auto take = [&](size_t bytes) {
      unsigned char* q = p;
      p += (bytes + 255) / 256 * 256;
      return q;
    };
    d.G = reinterpret_cast<cx<double>*>(take(b_cx));
    d.V = reinterpret_cast<cx<double>*>(take(b_cx));
    d.Ts = reinterpret_cast<cx<double>*>(take(2 * b_cx));
    df.G = reinterpret_cast<cx<float>*>(take(sizeof(cx<float>) * (size_t)(vs * B)));
    d.sv = reinterpret_cast<double*>(take(sizeof(double) * n * B));
    d.perm = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * n * B));
    d.dims = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * d.ds * B));
    d.knew = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * B));
    d.nold = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * B));
    d.trunc = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * B));
    d.err = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * B));
    d.err_step = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * 2 * B));
    d.frob = reinterpret_cast<double*>(take(sizeof(double) * B));
    // one move of node 1 towards its left child 2, whose bond has dimension n
    std::vector<int32_t> dims((size_t)d.ds * B, 1);
    for (int64_t b = 0; b < B; ++b) dims[(size_t)b * d.ds + 2] = n;
    e = cudaMemcpyAsync(d.dims, dims.data(), sizeof(int32_t) * dims.size(), cudaMemcpyHostToDevice, st);
    // matrix b at b * n^2 in G, at b * vs in the solver's slots
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(d.G, sizeof(cx<double>) * (size_t)vs, G, sizeof(cx<double>) * (size_t)n * n,
                            sizeof(cx<double>) * (size_t)n * n, (size_t)B, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, sizeof(int32_t) * B, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err_step, 0xFF, sizeof(int32_t) * 2 * B, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.knew, 0, sizeof(int32_t) * B, st);
    if (e == cudaSuccess && route == 0)
      e = cudaFuncSetAttribute(k_eig<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, EIG_SMEM_MAX);
    if (e == cudaSuccess && route > 0)
      e = cudaFuncSetAttribute(k_eig_tri<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               tri_smem_bytes<double>());
    if (e == cudaSuccess && route >= 2)
      e = cudaFuncSetAttribute(k_eig_bt, cudaFuncAttributeMaxDynamicSharedMemorySize, bt_smem_bytes());
    if (e == cudaSuccess) {
      if (route == 0) {
        k_eig<double><<<batch, 512, d.eig_smem_bytes, st>>>(d, 1, 2, kcap);
      } else {
        const int smem = std::max(d.eig_smem_bytes, route >= 2 ? tri_smem_bytes_nobt<double>() : tri_smem_bytes<double>());
        // the MIXED runs' launch shape: 256 threads up to n = 256
        k_eig_tri<double><<<batch, route == 3 && n <= 256 ? 256 : 512, smem, st>>>(d, 1, 2, kcap);
        if (route >= 2)
          k_eig_bt<<<dim3((unsigned)ceil_div(kcap, BT_COLS), batch), 256, bt_smem_bytes(n), st>>>(df, d);
      }
      if (route == 3) {  // the Jacobi share's V_k in complex64, as k_vk_to_float leaves it
        Dev<float> dfv = df;
        dfv.nold = d.nold;
        dfv.knew = d.knew;
        k_vk_to_float<<<batch, 256, 0, st>>>(dfv, d.G, EIG_JACOBI_N);
      }
      k_eig_collect<<<batch, 256, 0, st>>>(d, route >= 2 ? df.G : nullptr, static_cast<cx<double>*>(V), s, k, n,
                                           kcap);
      e = cudaGetLastError();
    }
  }
  std::vector<int32_t> herr(batch, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(herr.data(), d.err, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(pool);
  if (e != cudaSuccess) {
    set_error(std::string("CUDA: ttn_eig_gram: ") + cudaGetErrorString(e));
    return TTN_ECUDA;
  }
  for (int b = 0; b < batch; ++b)
    if (herr[b]) {
      set_error("ttn_eig_gram: matrix " + std::to_string(b) + ": error flags " + std::to_string(herr[b]) +
                " (1 zero matrix, 2 no convergence, 4 capacity, 8 non-finite)");
      return TTN_ENUMERIC;
    }
  return TTN_OK;
}

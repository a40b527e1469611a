// The two contractions of an isometry-centre move on the tcgen05 tensor
// cores, with exact products (digit_gemm.cuh):
//
//   form:    Y = M V_k    (M: the m x n bond matrix, V_k: its n x k kept
//                          right singular vectors; Y -> T_v with bond k)
//   absorb:  T_w <- R T_w on w's leg towards v (R = S V_k^H, k x n)
//
// A complex product becomes one real product of "interleaved" matrices: a
// complex row (a_0 + i b_0, a_1 + i b_1, ...) is the real row (a_0, b_0, a_1,
// b_1, ...), the same memory.  For Y = M V: Y_re = sum a v_re - b v_im,
// Y_im = sum a v_im + b v_re, so with A = M (m x 2n) and B^T (2k x 2n) whose
// row 2c holds (v_re, -v_im) and row 2c+1 (v_im, v_re) of column c of V, the
// real product A B^T has Y_re, Y_im in columns 2c, 2c+1.  For R T: A (2k x
// 2n) has rows (r_re, -r_im) and (r_im, r_re) for row i of R, and B^T (J x
// 2n) holds the J = (outer, inner) fibres of T_w along the leg, so rows 2i,
// 2i+1 of A B^T are the real and imaginary parts of row i of the result.
//
// Every row of A and of B^T is scaled by its own power of two (the scales
// leave the sum), rounded to 23 bits below its largest entry and split into
// bf16 digits; the tensor cores then sum the integer products exactly, and
// one rounding (int64 -> double, then -> float) gives each entry.  So the
// contraction is exact for its rounded inputs and free of the truncating
// accumulation of the legacy 3xTF32 mma.sync tile; entries far below their
// row's maximum keep fewer than FP32's 24 significant bits, so the result is
// not more accurate than FP32 FMA sums in general (both hold the MIXED
// amplitude bars).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "contract.h"
#include "digit_gemm.cuh"

namespace ttn {

__host__ __device__ inline int c_ceil(int64_t a, int b) { return (int)((a + b - 1) / b); }

static __device__ __forceinline__ uint16_t bf16_of(int v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
}

// Shape of a trajectory's move (kept rank k; n the bond before the move; m the
// rows of the bond matrix) and the column of element (i, c) of Y in T_v.
struct MoveShape {
  int leg, n, k, m, du;
};

static __device__ __forceinline__ MoveShape move_shape(const ContractArgs& a, int b) {
  const int* D = a.dims + (int64_t)b * a.ds;
  MoveShape s;
  s.leg = a.leg_v;
  s.n = a.nold[b];
  s.k = a.knew[b];
  const int dl0 = D[2 * a.v], dr0 = D[2 * a.v + 1], du0 = D[a.v];
  const int dl = s.leg == 0 ? s.n : dl0, dr = s.leg == 1 ? s.n : dr0;
  s.du = s.leg == 2 ? s.n : du0;
  s.m = s.k > 0 ? dl * dr * s.du / s.n : 0;
  return s;
}

static __device__ __forceinline__ int64_t y_addr(const MoveShape& s, int i, int c) {
  if (s.leg == 2) return (int64_t)i * s.k + c;
  if (s.leg == 0) return (int64_t)c * s.m + i;
  const int l = i / s.du, u = i - l * s.du;
  return ((int64_t)l * s.k + c) * s.du + u;
}

static __device__ __forceinline__ void c_flag(const ContractArgs& a, int b, int32_t code) {
  if (a.err) atomicOr(&a.err[b], code);
}

// ================================================================== Y = M V_k
// Digit tiles: A (m rows, K = 2n) at [s][mt][kt] * G_TILE, then B^T (2k rows)
// at the end of A's space, [s][nt][kt] * G_TILE / 2.  Row exponents: A's m
// then B's 2k (at offset a.rows_cap - 512).
__global__ void __launch_bounds__(256) k_form_packA(ContractArgs a) {
  const int b = blockIdx.y;
  const MoveShape s = move_shape(a, b);
  if (s.k <= 0) return;
  const int K = 2 * s.n, NMT = c_ceil(s.m, G_TA), NKT = c_ceil(K, G_KT);
  const int mt = blockIdx.x;
  if (mt >= NMT) return;
  if (3LL * NMT * NKT * G_TILE + 3LL * c_ceil(2 * s.k, G_TB) * NKT * (G_TILE / 2) > a.sstride ||
      s.m + 512 > a.rows_cap) {
    if (mt == 0 && threadIdx.x == 0) c_flag(a, b, CONTRACT_ERR_CAPACITY);
    return;
  }
  const float* X = reinterpret_cast<const float*>(a.M + (int64_t)b * a.mstride);
  uint16_t* S = a.slices + (int64_t)b * a.sstride;
  int* E = a.expo + (int64_t)b * a.rows_cap;
  __shared__ float rmax[2][G_TA];
  __shared__ int re[G_TA];
  const int r = threadIdx.x & (G_TA - 1), half = threadIdx.x >> 7;
  const int64_t i = (int64_t)mt * G_TA + r;
  float mx = 0.f;
  if (i < s.m)
    for (int c = half; c < K; c += 2) mx = fmaxf(mx, fabsf(X[i * K + c]));
  rmax[half][r] = mx;
  __syncthreads();
  if (half == 0) {
    int e = 0;
    const float v = fmaxf(rmax[0][r], rmax[1][r]);
    if (v > 0.f) frexpf(v, &e);
    re[r] = e;
    if (i < s.m) E[i] = e;
  }
  __syncthreads();
  for (int kt = 0; kt < NKT; ++kt) {
    uint16_t* t0 = S + ((int64_t)(0 * NMT + mt) * NKT + kt) * G_TILE;
    uint16_t* t1 = S + ((int64_t)(1 * NMT + mt) * NKT + kt) * G_TILE;
    uint16_t* t2 = S + ((int64_t)(2 * NMT + mt) * NKT + kt) * G_TILE;
    for (int e = threadIdx.x; e < G_TA * G_KT; e += 256) {
      const int kk = e & (G_KT - 1), rr = e / G_KT;
      const int64_t ii = (int64_t)mt * G_TA + rr;
      const int c = kt * G_KT + kk;
      int n1 = 0, n2 = 0, n3 = 0;
      if (ii < s.m && c < K) digits3(X[ii * K + c], re[rr], n1, n2, n3);
      const int off = digit_offset(rr, kk);
      t0[off] = bf16_of(n1);
      t1[off] = bf16_of(n2);
      t2[off] = bf16_of(n3);
    }
  }
}

__global__ void __launch_bounds__(256) k_form_packB(ContractArgs a) {
  const int b = blockIdx.y;
  const MoveShape s = move_shape(a, b);
  if (s.k <= 0) return;
  const int K = 2 * s.n, NMT = c_ceil(s.m, G_TA), NKT = c_ceil(K, G_KT), NNT = c_ceil(2 * s.k, G_TB);
  const int nt = blockIdx.x;
  if (nt >= NNT) return;
  if (3LL * NMT * NKT * G_TILE + 3LL * NNT * NKT * (G_TILE / 2) > a.sstride || s.m + 512 > a.rows_cap) return;
  const float2* V = a.V + (int64_t)b * a.vstride;  // n x k row-major
  uint16_t* S = a.slices + (int64_t)b * a.sstride + 3LL * NMT * NKT * G_TILE;
  int* E = a.expo + (int64_t)b * a.rows_cap + (a.rows_cap - 512);
  __shared__ float rmax[4][G_TB];
  __shared__ int re[G_TB];
  const int r = threadIdx.x & (G_TB - 1), part = threadIdx.x >> 6;
  const int j = nt * G_TB + r, c = j >> 1;
  float mx = 0.f;
  if (j < 2 * s.k)
    for (int x = part; x < s.n; x += 4) {
      const float2 v = V[(int64_t)x * s.k + c];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  rmax[part][r] = mx;
  __syncthreads();
  if (part == 0) {
    int e = 0;
    const float v = fmaxf(fmaxf(rmax[0][r], rmax[1][r]), fmaxf(rmax[2][r], rmax[3][r]));
    if (v > 0.f) frexpf(v, &e);
    re[r] = e;
    if (j < 2 * s.k) E[j] = e;
  }
  __syncthreads();
  for (int kt = 0; kt < NKT; ++kt) {
    uint16_t* t0 = S + ((int64_t)(0 * NNT + nt) * NKT + kt) * (G_TILE / 2);
    uint16_t* t1 = S + ((int64_t)(1 * NNT + nt) * NKT + kt) * (G_TILE / 2);
    uint16_t* t2 = S + ((int64_t)(2 * NNT + nt) * NKT + kt) * (G_TILE / 2);
    for (int e = threadIdx.x; e < G_TB * G_KT; e += 256) {
      const int kk = e & (G_KT - 1), rr = e / G_KT;
      const int jj = nt * G_TB + rr, cc = jj >> 1, p = jj & 1;
      const int col = kt * G_KT + kk, x = col >> 1, q = col & 1;
      int n1 = 0, n2 = 0, n3 = 0;
      if (jj < 2 * s.k && col < K) {
        const float2 v = V[(int64_t)x * s.k + cc];
        // row 2c: (v_re, -v_im); row 2c + 1: (v_im, v_re)
        const float val = p == 0 ? (q == 0 ? v.x : -v.y) : (q == 0 ? v.y : v.x);
        digits3(val, re[rr], n1, n2, n3);
      }
      const int off = digit_offset(rr, kk);
      t0[off] = bf16_of(n1);
      t1[off] = bf16_of(n2);
      t2[off] = bf16_of(n3);
    }
  }
}

// The trajectory's G_CTAS CTAs (blockIdx.x) loop over the (mt, nt) tiles of
// its actual shape, with one tensor memory allocation per CTA.
__global__ void __launch_bounds__(128, 1) k_form_mma(ContractArgs a) {
  const int b = blockIdx.y;
  const MoveShape s = move_shape(a, b);
  if (s.k <= 0) return;
  const int K = 2 * s.n, NMT = c_ceil(s.m, G_TA), NKT = c_ceil(K, G_KT), NNT = c_ceil(2 * s.k, G_TB);
  if (3LL * NMT * NKT * G_TILE + 3LL * NNT * NKT * (G_TILE / 2) > a.sstride || s.m + 512 > a.rows_cap) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.ledger && a.ledger_form >= 0) {
    atomicAdd(&a.ledger[2 * a.ledger_form], (unsigned long long)(8.0 * s.m * (double)s.n * s.k));
    atomicAdd(&a.ledger[2 * a.ledger_form + 1],
              (unsigned long long)(8.0 * ((double)s.m * s.n + (double)s.n * s.k + (double)s.m * s.k)));
  }
  if ((int)blockIdx.x >= NMT * NNT) return;
  const uint16_t* SA = a.slices + (int64_t)b * a.sstride;
  const uint16_t* SB = SA + 3LL * NMT * NKT * G_TILE;
  const int* EA = a.expo + (int64_t)b * a.rows_cap;
  const int* EB = EA + (a.rows_cap - 512);
  float2* T = a.T + (int64_t)b * a.tstride + a.off_v;
  __shared__ DigitShared dsh;
  DigitCtx dc;
  digit_begin(dsh, dc);
  for (int t = blockIdx.x; t < NMT * NNT; t += gridDim.x) {
    const int mt = t / NNT, nt = t - mt * NNT;
    auto srcA = [&](int d, int kt) { return SA + ((int64_t)(d * NMT + mt) * NKT + kt) * G_TILE; };
    auto srcB = [&](int d, int kt) { return SB + ((int64_t)(d * NNT + nt) * NKT + kt) * (G_TILE / 2); };
    const int i = mt * G_TA + threadIdx.x;
    const int ei = i < s.m ? EA[i] : 0;
    auto epilogue = [&](int h, const unsigned long long (&v)[32]) {
      if (i >= s.m) return;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = nt * G_TB + h * 32 + 2 * q, c = j >> 1;
        if (c < s.k) {
          const double y_re = ldexp((double)(long long)v[2 * q], ei + EB[j] - 46);
          const double y_im = ldexp((double)(long long)v[2 * q + 1], ei + EB[j + 1] - 46);
          T[y_addr(s, i, c)] = make_float2((float)y_re, (float)y_im);
        }
      }
    };
    if (!digit_tile(dsh, dc, 0, NKT, srcA, srcB, epilogue)) {
      if (threadIdx.x == 0) c_flag(a, b, CONTRACT_ERR_TIMEOUT);
      break;
    }
  }
  digit_end(dsh, dc);
}

// ================================================================== absorb
// T_w (dims dl, dr, du; the leg towards v has the old dimension n) <- R T_w
// on that leg, R: k x n (row-major complex64 in Rm).  Output into W (the
// layout k_absorb writes: out[(o * k + i) * inner + u]).
struct AbsorbShape {
  int lw, n, k, outer, inner, J;
};

static __device__ __forceinline__ AbsorbShape absorb_shape(const ContractArgs& a, int b) {
  const int* D = a.dims + (int64_t)b * a.ds;
  AbsorbShape s;
  s.lw = a.leg_w;
  const int dl = D[2 * a.w], dr = D[2 * a.w + 1], du = D[a.w];
  s.n = a.nold[b];
  s.k = a.knew[b];
  if (s.lw == 0) {
    s.outer = 1;
    s.inner = dr * du;
  } else if (s.lw == 1) {
    s.outer = dl;
    s.inner = du;
  } else {
    s.outer = dl * dr;
    s.inner = 1;
  }
  s.J = s.outer * s.inner;
  return s;
}

// A = rows (r_re, -r_im), (r_im, r_re) of R: 2k rows, K = 2n; B^T = the J
// fibres of T_w.  Digit tiles: A [s][mt][kt], then B^T [s][nt][kt]; row
// exponents: B's J, then A's 2k (at offset rows_cap - 512).
__global__ void __launch_bounds__(256) k_absorb_packA(ContractArgs a) {
  const int b = blockIdx.y;
  const AbsorbShape s = absorb_shape(a, b);
  if (s.k <= 0) return;
  const int K = 2 * s.n, NMT = c_ceil(2 * s.k, G_TA), NKT = c_ceil(K, G_KT), NNT = c_ceil(s.J, G_TB);
  const int mt = blockIdx.x;
  if (mt >= NMT) return;
  if (3LL * NMT * NKT * G_TILE + 3LL * NNT * NKT * (G_TILE / 2) > a.sstride || s.J + 512 > a.rows_cap) {
    if (mt == 0 && threadIdx.x == 0) c_flag(a, b, CONTRACT_ERR_CAPACITY);
    return;
  }
  const float2* R = a.Rm + (int64_t)b * a.vstride;
  uint16_t* S = a.slices + (int64_t)b * a.sstride;
  int* E = a.expo + (int64_t)b * a.rows_cap + (a.rows_cap - 512);
  __shared__ float rmax[2][G_TA];
  __shared__ int re[G_TA];
  const int r = threadIdx.x & (G_TA - 1), half = threadIdx.x >> 7;
  const int row = mt * G_TA + r, i = row >> 1;
  float mx = 0.f;
  if (row < 2 * s.k)
    for (int x = half; x < s.n; x += 2) {
      const float2 v = R[(int64_t)i * s.n + x];
      mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  rmax[half][r] = mx;
  __syncthreads();
  if (half == 0) {
    int e = 0;
    const float v = fmaxf(rmax[0][r], rmax[1][r]);
    if (v > 0.f) frexpf(v, &e);
    re[r] = e;
    if (row < 2 * s.k) E[row] = e;
  }
  __syncthreads();
  for (int kt = 0; kt < NKT; ++kt) {
    uint16_t* t0 = S + ((int64_t)(0 * NMT + mt) * NKT + kt) * G_TILE;
    uint16_t* t1 = S + ((int64_t)(1 * NMT + mt) * NKT + kt) * G_TILE;
    uint16_t* t2 = S + ((int64_t)(2 * NMT + mt) * NKT + kt) * G_TILE;
    for (int e = threadIdx.x; e < G_TA * G_KT; e += 256) {
      const int kk = e & (G_KT - 1), rr = e / G_KT;
      const int rw = mt * G_TA + rr, ii = rw >> 1, p = rw & 1;
      const int col = kt * G_KT + kk, x = col >> 1, q = col & 1;
      int n1 = 0, n2 = 0, n3 = 0;
      if (rw < 2 * s.k && col < K) {
        const float2 v = R[(int64_t)ii * s.n + x];
        const float val = p == 0 ? (q == 0 ? v.x : -v.y) : (q == 0 ? v.y : v.x);
        digits3(val, re[rr], n1, n2, n3);
      }
      const int off = digit_offset(rr, kk);
      t0[off] = bf16_of(n1);
      t1[off] = bf16_of(n2);
      t2[off] = bf16_of(n3);
    }
  }
}

__global__ void __launch_bounds__(256) k_absorb_packB(ContractArgs a) {
  const int b = blockIdx.y;
  const AbsorbShape s = absorb_shape(a, b);
  if (s.k <= 0) return;
  const int K = 2 * s.n, NMT = c_ceil(2 * s.k, G_TA), NKT = c_ceil(K, G_KT), NNT = c_ceil(s.J, G_TB);
  if (3LL * NMT * NKT * G_TILE + 3LL * NNT * NKT * (G_TILE / 2) > a.sstride || s.J + 512 > a.rows_cap) return;
  const float2* in = a.T + (int64_t)b * a.tstride + a.off_w;
  uint16_t* S = a.slices + (int64_t)b * a.sstride + 3LL * NMT * NKT * G_TILE;
  int* E = a.expo + (int64_t)b * a.rows_cap;
  __shared__ float rmax[4][G_TB];
  __shared__ int re[G_TB];
  for (int nt = blockIdx.x; nt < NNT; nt += gridDim.x) {
    const int r = threadIdx.x & (G_TB - 1), part = threadIdx.x >> 6;
    const int j = nt * G_TB + r;
    const int o = j / s.inner, u = j - o * s.inner;
    float mx = 0.f;
    if (j < s.J)
      for (int x = part; x < s.n; x += 4) {
        const float2 v = in[((int64_t)o * s.n + x) * s.inner + u];
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    rmax[part][r] = mx;
    __syncthreads();
    if (part == 0) {
      int e = 0;
      const float v = fmaxf(fmaxf(rmax[0][r], rmax[1][r]), fmaxf(rmax[2][r], rmax[3][r]));
      if (v > 0.f) frexpf(v, &e);
      re[r] = e;
      if (j < s.J) E[j] = e;
    }
    __syncthreads();
    for (int kt = 0; kt < NKT; ++kt) {
      uint16_t* t0 = S + ((int64_t)(0 * NNT + nt) * NKT + kt) * (G_TILE / 2);
      uint16_t* t1 = S + ((int64_t)(1 * NNT + nt) * NKT + kt) * (G_TILE / 2);
      uint16_t* t2 = S + ((int64_t)(2 * NNT + nt) * NKT + kt) * (G_TILE / 2);
      for (int e = threadIdx.x; e < G_TB * G_KT; e += 256) {
        const int kk = e & (G_KT - 1), rr = e / G_KT;
        const int jj = nt * G_TB + rr, oo = jj / s.inner, uu = jj - oo * s.inner;
        const int col = kt * G_KT + kk, x = col >> 1, q = col & 1;
        int n1 = 0, n2 = 0, n3 = 0;
        if (jj < s.J && col < K) {
          const float2 v = in[((int64_t)oo * s.n + x) * s.inner + uu];
          digits3(q == 0 ? v.x : v.y, re[rr], n1, n2, n3);
        }
        const int off = digit_offset(rr, kk);
        t0[off] = bf16_of(n1);
        t1[off] = bf16_of(n2);
        t2[off] = bf16_of(n3);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(128, 1) k_absorb_mma(ContractArgs a) {
  const int b = blockIdx.y;
  const AbsorbShape s = absorb_shape(a, b);
  if (s.k <= 0) return;
  const int K = 2 * s.n, NMT = c_ceil(2 * s.k, G_TA), NKT = c_ceil(K, G_KT), NNT = c_ceil(s.J, G_TB);
  if (3LL * NMT * NKT * G_TILE + 3LL * NNT * NKT * (G_TILE / 2) > a.sstride || s.J + 512 > a.rows_cap) return;
  if ((int64_t)s.k * s.J > a.wstride) return;
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.ledger && a.ledger_absorb >= 0) {
    atomicAdd(&a.ledger[2 * a.ledger_absorb], (unsigned long long)(8.0 * s.k * (double)s.n * s.J));
    atomicAdd(&a.ledger[2 * a.ledger_absorb + 1],
              (unsigned long long)(8.0 * ((double)s.n * s.J + (double)s.k * s.n + (double)s.k * s.J)));
  }
  if ((int)blockIdx.x >= NMT * NNT) return;
  const uint16_t* SA = a.slices + (int64_t)b * a.sstride;
  const uint16_t* SB = SA + 3LL * NMT * NKT * G_TILE;
  const int* EB = a.expo + (int64_t)b * a.rows_cap;
  const int* EA = EB + (a.rows_cap - 512);
  float* out = reinterpret_cast<float*>(a.W + (int64_t)b * a.wstride);
  __shared__ DigitShared dsh;
  DigitCtx dc;
  digit_begin(dsh, dc);
  for (int t = blockIdx.x; t < NMT * NNT; t += gridDim.x) {
    const int nt = t / NMT, mt = t - nt * NMT;
    auto srcA = [&](int d, int kt) { return SA + ((int64_t)(d * NMT + mt) * NKT + kt) * G_TILE; };
    auto srcB = [&](int d, int kt) { return SB + ((int64_t)(d * NNT + nt) * NKT + kt) * (G_TILE / 2); };
    const int row = mt * G_TA + threadIdx.x, i = row >> 1, p = row & 1;
    const int er = row < 2 * s.k ? EA[row] : 0;
    auto epilogue = [&](int h, const unsigned long long (&v)[32]) {
      if (row >= 2 * s.k) return;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = nt * G_TB + h * 32 + q;
        if (j < s.J) {
          const int o = j / s.inner, u = j - o * s.inner;
          out[(((int64_t)o * s.k + i) * s.inner + u) * 2 + p] =
              (float)ldexp((double)(long long)v[q], er + EB[j] - 46);
        }
      }
    };
    if (!digit_tile(dsh, dc, 0, NKT, srcA, srcB, epilogue)) {
      if (threadIdx.x == 0) c_flag(a, b, CONTRACT_ERR_TIMEOUT);
      break;
    }
  }
  digit_end(dsh, dc);
}

// ================================================================== host
int64_t contract_form_elems(int64_t m, int n, int k) {
  const int NKT = c_ceil(2 * n, G_KT);
  return 3LL * c_ceil(m, G_TA) * NKT * G_TILE + 3LL * c_ceil(2 * k, G_TB) * NKT * (G_TILE / 2);
}

int64_t contract_absorb_elems(int n, int k, int64_t J) {
  const int NKT = c_ceil(2 * n, G_KT);
  return 3LL * c_ceil(2 * k, G_TA) * NKT * G_TILE + 3LL * c_ceil(J, G_TB) * NKT * (G_TILE / 2);
}

static bool g_attr_set[64] = {false};

static cudaError_t set_attrs() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && g_attr_set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(k_form_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_absorb_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_attr_set[dev] = true;
  return e;
}

cudaError_t contract_form_launch(const ContractArgs& a, int B, int64_t m_cap, int n_cap, int k_cap,
                                 cudaStream_t st) {
  if (B <= 0 || m_cap <= 0 || n_cap <= 0 || k_cap <= 0) return cudaSuccess;
  cudaError_t e = set_attrs();
  if (e != cudaSuccess) return e;
  const int nmt = c_ceil(m_cap, G_TA), nnt = c_ceil(2 * k_cap, G_TB);
  k_form_packA<<<dim3(nmt, B), 256, 0, st>>>(a);
  k_form_packB<<<dim3(nnt, B), 256, 0, st>>>(a);
  k_form_mma<<<dim3(std::min(nmt * nnt, G_CTAS), B), 128, G_SMEM, st>>>(a);
  return cudaGetLastError();
}

cudaError_t contract_absorb_launch(const ContractArgs& a, int B, int n_cap, int k_cap, int64_t J_cap,
                                   cudaStream_t st) {
  if (B <= 0 || n_cap <= 0 || k_cap <= 0 || J_cap <= 0) return cudaSuccess;
  cudaError_t e = set_attrs();
  if (e != cudaSuccess) return e;
  const int nmt = c_ceil(2 * k_cap, G_TA), nnt = c_ceil(J_cap, G_TB);
  k_absorb_packA<<<dim3(nmt, B), 256, 0, st>>>(a);
  k_absorb_packB<<<dim3(std::min(nnt, 1024), B), 256, 0, st>>>(a);
  k_absorb_mma<<<dim3(std::min(nmt * nnt, G_CTAS), B), 128, G_SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ttn

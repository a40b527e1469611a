// Exact Gram matrix of complex64 bond matrices on the tcgen05 tensor cores.
//
// The isometry-centre move factorises the bond matrix M (m x n, complex64)
// through its Gram matrix G = M^H M and an FP64 eigendecomposition.  A Gram
// matrix formed in FP32 squares M's condition number at FP32 precision: its
// eigenvalues lose every singular value below ~sqrt(eps_fp32) s_max.  Here G
// is formed exactly for the matrix M~ obtained by rounding every column of M
// to 23 bits below that column's largest entry (|M~ - M| <= 2^-24 max|M_c|
// per entry, the precision M is stored with), and rounded once to FP64:
//
//  1. X = M viewed as a real m x 2n matrix (columns Re M_j, Im M_j
//     interleaved, the same memory).  Column c is scaled by 2^(23 - E_c)
//     (max |X_c| < 2^E_c) and rounded to an integer |N| <= 2^23.
//  2. N = n1 2^16 + n2 2^8 + n3 with integer digits |n_s| <= 128, each exact
//     in bf16.  The digit matrices are written as bf16 tiles in the K-major
//     core-matrix layout of tcgen05.mma.
//  3. X^T X = sum over digit pairs (s, t) of 2^(8 (6 - s - t)) D_s^T D_t.
//     The nine products run on the tensor cores (kind::f16, BF16 operands,
//     FP32 accumulators in tensor memory), pairs of equal weight sharing one
//     of five accumulators.  Products of digits are below 2^14 and a weight
//     group holds at most three of them, so a 256-row chunk sums to below
//     2^24 in magnitude: the FP32 accumulation is exact.  After every chunk
//     the five accumulators are converted to integers and combined into one
//     64-bit fixed-point sum per entry (|N_a N_b| <= 2^46, m <= 2^16 rows).
//  4. The integer sums of the row-splits meet in an int64 matrix (atomic
//     adds, exact), which the last kernel converts to double, scales back by
//     2^(E_a + E_b - 46) and combines into the complex G:
//     Re G_ij = X_2i.X_2j + X_2i+1.X_2j+1,  Im G_ij = X_2i.X_2j+1 - X_2i+1.X_2j.
//
// This is the digit-splitting ("Ozaki") scheme for error-free matrix
// products (Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59 (2012)),
// specialised to the Gram matrix of FP32 data with bf16 tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "gram.h"
#include "internal.h"
#include "digit_gemm.cuh"
#include "tc100.cuh"

namespace ttn {

static constexpr int G_SPLIT = 4096 / G_KT;      // K-tiles per CTA (4096 rows)

__host__ __device__ inline int g_nct(int n) { return (2 * n + G_TA - 1) / G_TA; }
__host__ __device__ inline int g_nkt(int64_t m) { return (int)((m + G_KT - 1) / G_KT); }

int64_t gram_slice_elems(int64_t m, int n) { return 3LL * g_nct(n) * g_nkt(m) * G_TILE; }

__device__ __forceinline__ int64_t d_slice_elems(int64_t m, int n) {
  return 3LL * g_nct(n) * g_nkt(m) * G_TILE;
}

__device__ __forceinline__ void g_flag(const GramArgs& a, int b, int32_t code) {
  if (a.err) atomicOr(&a.err[b], code);
}

// ---------------------------------------------------------------- 1. column maxima
__global__ void __launch_bounds__(256) k_gram_amax(GramArgs a) {
  const int b = blockIdx.z;
  const int2 sh = a.shape[b];
  const int64_t m = sh.x;
  const int nc = 2 * sh.y;
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  if (sh.y <= 0 || c >= nc) return;
  const float* X = reinterpret_cast<const float*>(a.M + (int64_t)b * a.mstride);
  float mx = 0.f;
  for (int64_t r = (int64_t)blockIdx.y * 8 + (threadIdx.x >> 5); r < m; r += (int64_t)gridDim.y * 8)
    mx = fmaxf(mx, fabsf(X[r * nc + c]));
  if (mx > 0.f) atomicMax(&a.amax[(int64_t)b * a.cstride + c], __float_as_uint(mx));
}

// ---------------------------------------------------------------- column exponents
__global__ void k_gram_exps(GramArgs a) {
  const int b = blockIdx.y;
  const int n = a.shape[b].y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= 2 * n) return;
  unsigned int* am = a.amax + (int64_t)b * a.cstride + c;
  const float mx = __uint_as_float(*am);
  int e = 0;
  if (mx > 0.f) frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1): max |X_c| < 2^e
  a.expo[(int64_t)b * a.cstride + c] = e;
  *am = 0u;                      // ready for the next matrix
}

// ---------------------------------------------------------------- 2. digit tiles
// Tile (s, ct, kt) of trajectory b: X-columns ct*128.., rows kt*32.., digit
// s, at ((s * NCT + ct) * NKT + kt) * G_TILE.  Inside a tile, element
// (column cc, row rr) at (cc/8)*256 + (rr/8)*64 + (cc%8)*8 + rr%8: core
// matrices of 8 columns x 8 rows (16 bytes per column), K-groups adjacent
// (LBO 128 bytes), 8-column groups G_SBO = 512 bytes apart (SBO).
__global__ void __launch_bounds__(256) k_gram_pack(GramArgs a) {
  const int b = blockIdx.z;
  const int2 sh = a.shape[b];
  const int64_t m = sh.x;
  const int n = sh.y, nc = 2 * n;
  if (n <= 0) return;
  const int NCT = g_nct(n), NKT = g_nkt(m);
  const int ct = blockIdx.x;
  if (ct >= NCT) return;
  if (d_slice_elems(m, n) > a.sstride) {
    if (ct == 0 && blockIdx.y == 0 && threadIdx.x == 0) g_flag(a, b, GRAM_ERR_CAPACITY);
    return;
  }
  const float* X = reinterpret_cast<const float*>(a.M + (int64_t)b * a.mstride);
  const int* E = a.expo + (int64_t)b * a.cstride;
  uint16_t* S = a.slices + (int64_t)b * a.sstride;
  bool bad = false;
  for (int kt = blockIdx.y; kt < NKT; kt += gridDim.y) {
    uint16_t* t0 = S + ((int64_t)(0 * NCT + ct) * NKT + kt) * G_TILE;
    uint16_t* t1 = S + ((int64_t)(1 * NCT + ct) * NKT + kt) * G_TILE;
    uint16_t* t2 = S + ((int64_t)(2 * NCT + ct) * NKT + kt) * G_TILE;
    for (int e = threadIdx.x; e < G_TA * G_KT; e += 256) {
      const int cc = e & (G_TA - 1), rr = e >> 7;
      const int c = ct * G_TA + cc;
      const int64_t r = (int64_t)kt * G_KT + rr;
      int n1 = 0, n2 = 0, n3 = 0;
      if (c < nc && r < m) {
        const float x = X[r * nc + c];
        if (!isfinite(x)) {
          bad = true;
        } else {
          digits3(x, E[c], n1, n2, n3);
        }
      }
      const int off = digit_offset(cc, rr);
      t0[off] = __bfloat16_as_ushort(__float2bfloat16_rn((float)n1));
      t1[off] = __bfloat16_as_ushort(__float2bfloat16_rn((float)n2));
      t2[off] = __bfloat16_as_ushort(__float2bfloat16_rn((float)n3));
    }
  }
  if (bad) g_flag(a, b, 8);  // non-finite entry
}

// ---------------------------------------------------------------- 3. tensor-core products
// CTA = (tile pair, row split, trajectory).  Tile pair: 128 X-columns ta (MMA
// rows) x 64 X-columns tb (MMA columns), tb >= 2 ta (the upper triangle of
// X^T X in 64-column blocks).  The digit products and their exact integer
// sums are digit_gemm's (digit_gemm.cuh); the epilogue adds each row's sums
// into the trajectory's int64 matrix.
// Tiles: (A row tile ta, 64-column B tile tb >= 2 ta) pairs of the upper
// triangle, enumerated row by row, times splits of G_SPLIT K-tiles.  A trajectory's G_CTAS CTAs
// (blockIdx.x) loop over the tiles of its actual shape, with one tensor
// memory allocation per CTA.
__global__ void __launch_bounds__(128, 1) k_gram_mma(GramArgs a) {
  const int b = blockIdx.z;
  const int2 sh2 = a.shape[b];
  const int64_t m = sh2.x;
  const int n = sh2.y, nc = 2 * n;
  if (n <= 0) return;
  const int NCT = g_nct(n), NKT = g_nkt(m);
  if (d_slice_elems(m, n) > a.sstride) return;  // flagged by the packing kernel
  const int npair = NCT * (NCT + 1);  // (ta, tb) with 2 ta <= tb < 2 NCT, row by row
  const int ntile = npair * ((NKT + G_SPLIT - 1) / G_SPLIT);
  if ((int)blockIdx.x >= ntile) return;
  const uint16_t* S = a.slices + (int64_t)b * a.sstride;
  __shared__ DigitShared dsh;
  DigitCtx dc;
  digit_begin(dsh, dc);
  for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
    const int sp = t / npair;
    int p = t - sp * npair, ta = 0;
    while (p >= 2 * NCT - 2 * ta) {
      p -= 2 * NCT - 2 * ta;
      ++ta;
    }
    const int tb = 2 * ta + p;
    if (tb * G_TB >= nc) continue;  // past the last column (2n an odd multiple of 64): uniform
    const int kt0 = sp * G_SPLIT, kt1 = min(NKT, kt0 + G_SPLIT);
    auto srcA = [&](int s, int kt) { return S + ((int64_t)(s * NCT + ta) * NKT + kt) * G_TILE; };
    auto srcB = [&](int s, int kt) {
      return S + ((int64_t)(s * NCT + (tb >> 1)) * NKT + kt) * G_TILE + (tb & 1) * (G_TILE / 2);
    };
    const int arow = ta * G_TA + threadIdx.x;
    unsigned long long* F = a.gfix + (int64_t)b * a.gld * a.gld + (int64_t)arow * a.gld;
    auto epilogue = [&](int h, const unsigned long long (&v)[32]) {
      if (arow >= nc) return;
      for (int j = 0; j < 32; ++j) {
        const int c = tb * G_TB + h * 32 + j;
        if (c >= arow && c < nc && v[j] != 0ull) atomicAdd(&F[c], v[j]);
      }
    };
    if (!digit_tile(dsh, dc, kt0, kt1 - kt0, srcA, srcB, epilogue)) {
      if (threadIdx.x == 0) g_flag(a, b, GRAM_ERR_TIMEOUT);
      break;
    }
  }
  digit_end(dsh, dc);
}

// ---------------------------------------------------------------- 4. complex FP64 Gram
__global__ void k_gram_finalize(GramArgs a) {
  const int b = blockIdx.y;
  const int2 sh = a.shape[b];
  const int n = sh.y;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n <= 0 || idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
  if (i > j) return;
  const int* E = a.expo + (int64_t)b * a.cstride;
  unsigned long long* F = a.gfix + (int64_t)b * a.gld * a.gld;
  auto rd = [&](int p, int q) -> double {  // p <= q; each entry is read once, then cleared
    unsigned long long* f = F + (int64_t)p * a.gld + q;
    const long long v = (long long)*f;
    *f = 0ull;
    return ldexp((double)v, E[p] + E[q] - 46);
  };
  const double xx = rd(2 * i, 2 * j), yy = rd(2 * i + 1, 2 * j + 1), xy = rd(2 * i, 2 * j + 1);
  const double yx = (i == j) ? xy : rd(2 * i + 1, 2 * j);
  double2* G = a.G + (int64_t)b * a.g64stride;
  G[(int64_t)i * n + j] = make_double2(xx + yy, xy - yx);
  if (i != j) G[(int64_t)j * n + i] = make_double2(xx + yy, yx - xy);
  if (idx == 0 && a.ledger && a.ledger_class >= 0) {
    atomicAdd(&a.ledger[2 * a.ledger_class], (unsigned long long)(8.0 * (double)sh.x * n * n));
    atomicAdd(&a.ledger[2 * a.ledger_class + 1],
              (unsigned long long)(8.0 * (double)sh.x * n + 16.0 * (double)n * n));
  }
}

// ---------------------------------------------------------------- host
static std::mutex g_attr_mutex;
static bool g_attr_done[64] = {false};

cudaError_t gram_exact_launch(const GramArgs& a, int B, int n_cap, int64_t m_cap, cudaStream_t st) {
  if (B <= 0 || n_cap <= 0 || m_cap <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (dev >= 0 && dev < 64 && !g_attr_done[dev]) {
      e = cudaFuncSetAttribute(k_gram_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
      if (e != cudaSuccess) return e;
      g_attr_done[dev] = true;
    }
  }
  const int nct = g_nct(n_cap), nkt = g_nkt(m_cap);
  const int rs = (int)std::min<int64_t>(64, std::max<int64_t>(1, (m_cap + 511) / 512));
  k_gram_amax<<<dim3((2 * n_cap + 31) / 32, rs, B), 256, 0, st>>>(a);
  k_gram_exps<<<dim3((2 * n_cap + 127) / 128, B), 128, 0, st>>>(a);
  k_gram_pack<<<dim3(nct, std::min(nkt, 64), B), 256, 0, st>>>(a);
  {
    const int tiles = nct * (nct + 1) * ((nkt + G_SPLIT - 1) / G_SPLIT);
    k_gram_mma<<<dim3(std::min(tiles, G_CTAS), 1, B), 128, G_SMEM, st>>>(a);
  }
  k_gram_finalize<<<dim3((int)(((int64_t)n_cap * n_cap + 255) / 256), B), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ttn

// ---------------------------------------------------------------- C ABI
extern "C" ttn_status ttn_gram_exact(const void* M, int64_t m, int32_t n, void* G, void* cuda_stream) {
  using namespace ttn;
  if (!M || !G || m < 1 || n < 1 || n > 1024 || m > (1 << 16)) {
    set_error("ttn_gram_exact: need device M (m x n), G (n x n), 1 <= n <= 1024, 1 <= m <= 65536");
    return TTN_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(M) & 7) || (reinterpret_cast<uintptr_t>(G) & 15)) {
    set_error("ttn_gram_exact: M must be 8-byte and G 16-byte aligned");
    return TTN_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  GramArgs a;
  a.M = static_cast<const float2*>(M);
  a.G = static_cast<double2*>(G);
  a.cstride = 2 * n;
  a.gld = 2 * n;
  a.sstride = gram_slice_elems(m, n);
  int2* dshape = nullptr;
  int32_t* derr = nullptr;
  void* scratch = nullptr;
  const size_t b_amax = sizeof(unsigned) * 2 * n, b_exp = sizeof(int) * 2 * n;
  const size_t b_fix = sizeof(unsigned long long) * (size_t)(2 * n) * (2 * n);
  const size_t b_sl = sizeof(uint16_t) * (size_t)a.sstride;
  auto cleanup = [&]() {
    cudaFree(dshape);
    cudaFree(derr);
    cudaFree(scratch);
  };
  cudaError_t e = cudaMalloc(&dshape, sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&scratch, b_fix + b_sl + b_amax + b_exp + 1024);
  if (e == cudaSuccess) {
    unsigned char* p = static_cast<unsigned char*>(scratch);
    a.gfix = reinterpret_cast<unsigned long long*>(p);
    a.slices = reinterpret_cast<uint16_t*>(p + b_fix);
    a.amax = reinterpret_cast<unsigned*>(p + ((b_fix + b_sl + 255) / 256) * 256);
    a.expo = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(a.amax) + ((b_amax + 255) / 256) * 256);
    a.shape = dshape;
    a.err = derr;
    const int2 sh = make_int2((int)m, n);
    e = cudaMemcpyAsync(dshape, &sh, sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.gfix, 0, b_fix, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.amax, 0, b_amax, st);
    if (e == cudaSuccess) e = gram_exact_launch(a, 1, n, m, st);
  }
  int32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) {
    set_error(std::string("CUDA: ttn_gram_exact: ") + cudaGetErrorString(e));
    return TTN_ECUDA;
  }
  if (herr & GRAM_ERR_TIMEOUT) {
    set_error("ttn_gram_exact: a bounded wait of the tensor-core kernel expired");
    return TTN_ETIMEOUT;
  }
  if (herr) {
    set_error("ttn_gram_exact: non-finite entry or workspace overflow (flags " + std::to_string(herr) + ")");
    return TTN_EINVAL;
  }
  return TTN_OK;
}

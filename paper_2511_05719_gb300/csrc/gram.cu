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

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "gram.h"
#include "internal.h"
#include "tc100.cuh"

namespace ttn {

static constexpr int G_KT = 32;                  // rows of M per K-tile
static constexpr int G_TA = 128;                 // X-columns per A tile (MMA M)
static constexpr int G_TB = 64;                  // X-columns per B tile (MMA N)
static constexpr int G_TILE = G_TA * G_KT;       // bf16 elements of a packed 128 x 32 tile (8 KB)
static constexpr int G_TILE_B = G_TILE * 2;      // its bytes
static constexpr int G_SBO = G_KT / 8 * 128;     // bytes between 8-column groups of a tile
static constexpr int G_CHUNK = 256 / G_KT;       // K-tiles per exact FP32 accumulation (256 rows)
static constexpr int G_SPLIT = 4096 / G_KT;      // K-tiles per CTA (4096 rows)
static constexpr int G_NS = 3;                   // pipeline stages
static constexpr int G_STAGE = 3 * G_TILE_B + 3 * (G_TILE_B / 2);  // A digits (128 rows) + B digits (64)
static constexpr int G_SMEM = G_NS * G_STAGE;    // dynamic shared memory of k_gram_mma
static constexpr uint32_t G_WAIT = 1u << 22;     // polls of a bounded mbarrier wait
// tensor memory: five 64-column FP32 accumulators (columns 0..319), then the
// row's 64-bit fixed-point sums as low (320..383) and high (384..447) words
static constexpr int G_TMEM_COLS = 512;
static constexpr int G_TM_LO = 5 * G_TB, G_TM_HI = 6 * G_TB;

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
          const int N = __float2int_rn(ldexpf(x, 23 - E[c]));
          n1 = (N + 32768) >> 16;
          const int r1 = N - n1 * 65536;
          n2 = (r1 + 128) >> 8;
          n3 = r1 - n2 * 256;
        }
      }
      const int off = (cc >> 3) * (G_SBO / 2) + (rr >> 3) * 64 + (cc & 7) * 8 + (rr & 7);
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
// X^T X in 64-column blocks).  Thread t of the four warps owns accumulator
// row t (TMEM lane t); thread 0 also issues the bulk copies and the MMAs.
__global__ void __launch_bounds__(128, 1) k_gram_mma(GramArgs a, int nct_cap) {
  extern __shared__ __align__(1024) unsigned char g_smem[];
  __shared__ __align__(8) uint64_t bar_load[G_NS], bar_mma[G_NS], bar_acc;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const int b = blockIdx.z;
  const int2 sh = a.shape[b];
  const int64_t m = sh.x;
  const int n = sh.y, nc = 2 * n;
  if (n <= 0) return;
  const int NCT = g_nct(n), NKT = g_nkt(m);
  int p = blockIdx.x, ta = 0;
  while (ta < nct_cap && p >= 2 * nct_cap - 2 * ta) {
    p -= 2 * nct_cap - 2 * ta;
    ++ta;
  }
  const int tb = 2 * ta + p;
  if (ta >= NCT || tb * G_TB >= nc) return;
  const int kt0 = blockIdx.y * G_SPLIT;
  if (kt0 >= NKT) return;
  const int kt1 = min(NKT, kt0 + G_SPLIT);
  if (d_slice_elems(m, n) > a.sstride) return;  // flagged by the packing kernel

  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int i = 0; i < G_NS; ++i) {
      tc::mbar_init(&bar_load[i], 1);
      tc::mbar_init(&bar_mma[i], 1);
    }
    tc::mbar_init(&bar_acc, 1);
    tc::mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, G_TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lane quarter

  const uint16_t* S = a.slices + (int64_t)b * a.sstride;
  auto srcA = [&](int s, int kt) { return S + ((int64_t)(s * NCT + ta) * NKT + kt) * G_TILE; };
  auto srcB = [&](int s, int kt) {
    return S + ((int64_t)(s * NCT + (tb >> 1)) * NKT + kt) * G_TILE + (tb & 1) * (G_TILE / 2);
  };
  auto stage = [&](int st) { return g_smem + st * G_STAGE; };
  auto issue_load = [&](int st, int kt) {
    tc::mbar_expect_tx(&bar_load[st], G_STAGE);
    for (int s = 0; s < 3; ++s) tc::bulk_g2s(stage(st) + s * G_TILE_B, srcA(s, kt), G_TILE_B, &bar_load[st]);
    for (int s = 0; s < 3; ++s)
      tc::bulk_g2s(stage(st) + 3 * G_TILE_B + s * (G_TILE_B / 2), srcB(s, kt), G_TILE_B / 2, &bar_load[st]);
  };

  const uint32_t idesc = tc::instr_desc(1, G_TA, G_TB);
  const int nk = kt1 - kt0;
  int loads[G_NS], commits[G_NS];  // per stage: bulk loads issued, MMA commits (thread 0)
  for (int i = 0; i < G_NS; ++i) loads[i] = commits[i] = 0;
  if (tid == 0)
    for (int i = 0; i < G_NS - 1 && i < nk; ++i) {
      issue_load(i, kt0 + i);
      loads[i]++;
    }
  uint32_t acc_phase = 0;
  bool first_chunk = true;
  bool first[5] = {true, true, true, true, true};
  for (int i = 0; i < nk; ++i) {
    const int st = i % G_NS;
    const bool chunk_end = (i % G_CHUNK) == G_CHUNK - 1 || i == nk - 1;
    if (tid == 0 && !s_abort) {
      if (!tc::mbar_wait(&bar_load[st], (uint32_t)((i / G_NS) & 1), G_WAIT)) {
        s_abort = 1;
      } else {
        tc::tc_fence_after();
        if (i % G_CHUNK == 0)
          for (int g = 0; g < 5; ++g) first[g] = true;
        const uint32_t sa = tc::smem_u32(stage(st)), sb = sa + 3 * G_TILE_B;
#pragma unroll
        for (int ks = 0; ks < G_KT / 16; ++ks) {
#pragma unroll
          for (int s1 = 0; s1 < 3; ++s1) {
#pragma unroll
            for (int s2 = 0; s2 < 3; ++s2) {
              const int g = s1 + s2;
              const uint64_t ad = tc::smem_desc(sa + s1 * G_TILE_B + ks * 256, 128, G_SBO);
              const uint64_t bd = tc::smem_desc(sb + s2 * (G_TILE_B / 2) + ks * 256, 128, G_SBO);
              tc::mma_bf16(tmem + g * G_TB, ad, bd, idesc, first[g] ? 0u : 1u);
              first[g] = false;
            }
          }
        }
        tc::mma_commit(&bar_mma[st]);
        commits[st]++;
        // tile i + NS - 1 goes into the stage tile i - 1 used, once its MMAs are done
        const int nx = i + G_NS - 1;
        if (nx < nk) {
          const int so = nx % G_NS;
          bool ok = true;
          if (commits[so] > 0) ok = tc::mbar_wait(&bar_mma[so], (uint32_t)((commits[so] - 1) & 1), G_WAIT);
          if (!ok) {
            s_abort = 1;
          } else {
            issue_load(so, kt0 + nx);
            loads[so]++;
          }
        }
        if (chunk_end) tc::mma_commit(&bar_acc);
      }
    }
    if (chunk_end) {
      __syncthreads();
      if (s_abort) break;
      // every thread polls; the block agrees on the outcome before the
      // warp-collective TMEM loads
      const int ok = __syncthreads_and(tc::mbar_wait(&bar_acc, acc_phase, G_WAIT) ? 1 : 0);
      acc_phase ^= 1u;
      if (!ok) {
        if (tid == 0) s_abort = 1;
        break;
      }
      tc::tc_fence_after();
#pragma unroll
      for (int h = 0; h < G_TB / 32; ++h) {
        long long part[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) part[j] = 0;
#pragma unroll
        for (int g = 0; g < 5; ++g) {
          uint32_t r[32];
          tc::tmem_ld32(tmem + lane_off + g * G_TB + h * 32, r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j)
            part[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << (8 * (4 - g));
        }
        uint32_t lo[32], hi[32];
        if (!first_chunk) {
          tc::tmem_ld32(tmem + lane_off + G_TM_LO + h * 32, lo);
          tc::tmem_ld32(tmem + lane_off + G_TM_HI + h * 32, hi);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) part[j] += (long long)(((uint64_t)hi[j] << 32) | lo[j]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          lo[j] = (uint32_t)(uint64_t)part[j];
          hi[j] = (uint32_t)((uint64_t)part[j] >> 32);
        }
        tc::tmem_st32(tmem + lane_off + G_TM_LO + h * 32, lo);
        tc::tmem_st32(tmem + lane_off + G_TM_HI + h * 32, hi);
        tc::tmem_st_wait();
      }
      first_chunk = false;
      tc::tc_fence_before();
      __syncthreads();
    }
  }
  __syncthreads();
  if (s_abort) {
    // let the copies and MMAs already issued finish (bounded) before the
    // shared memory and tensor memory are released
    if (tid == 0) {
      tc::mma_commit(&bar_acc);
      tc::mbar_wait(&bar_acc, acc_phase, G_WAIT);
      for (int st = 0; st < G_NS; ++st)
        if (loads[st] > 0) tc::mbar_wait(&bar_load[st], (uint32_t)((loads[st] - 1) & 1), G_WAIT);
      g_flag(a, b, GRAM_ERR_TIMEOUT);
    }
  } else {
    tc::tc_fence_after();
    const int arow = ta * G_TA + tid;
    unsigned long long* F = a.gfix + (int64_t)b * a.gld * a.gld + (int64_t)arow * a.gld;
    for (int h = 0; h < G_TB / 32; ++h) {
      uint32_t lo[32], hi[32];
      tc::tmem_ld32(tmem + lane_off + G_TM_LO + h * 32, lo);
      tc::tmem_ld32(tmem + lane_off + G_TM_HI + h * 32, hi);
      tc::tmem_ld_wait();
      if (arow < nc) {
        for (int j = 0; j < 32; ++j) {
          const int c = tb * G_TB + h * 32 + j;
          const unsigned long long v = ((unsigned long long)hi[j] << 32) | lo[j];
          if (c >= arow && c < nc && v != 0ull) atomicAdd(&F[c], v);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, G_TMEM_COLS);
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
  k_gram_mma<<<dim3(nct * (nct + 1), (nkt + G_SPLIT - 1) / G_SPLIT, B), 128, G_SMEM, st>>>(a, nct);
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

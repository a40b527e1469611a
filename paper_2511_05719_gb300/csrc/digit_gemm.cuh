// Exact products of FP32 data on the tcgen05 tensor cores by digit splitting
// (one CTA's share).  Used by the exact Gram matrix of the centre moves
// (gram.cu) and by the contractions of a centre move (contract.cu).
//
// Operands arrive as bf16 "digit tiles": an FP32 row (or column) of a
// factor, scaled by a power of two so that its largest entry is below 1/2
// and rounded to an integer |N| <= 2^23, is split as N = n1 2^16 + n2 2^8 + n3
// with integer digits |n_s| <= 128, each exact in bf16.  A tile holds one
// digit of 128 (A) or 64 (B) rows x G_KT K-values in the K-major core-matrix
// layout of tcgen05.mma without swizzle: element (row r, k) at
// (r / 8) * G_SBO / 2 + (k / 8) * 64 + (r % 8) * 8 + k % 8 (bf16 units).
//
// D = A B^T = sum over digit pairs (s, t) of 2^(8 (6 - s - t)) A_s B_t^T.
// The nine products run as tcgen05.mma (kind::f16, BF16 operands, M = 128,
// N = 64, K = 16) into five FP32 accumulators in tensor memory, one per
// weight.  A product of two digits is below 2^14 and a weight group holds at
// most three, so 256 K-values sum to below 2^24: exact in FP32.  Every 256
// K-values the five accumulators are converted to integers and added, with
// their weights, into one 64-bit sum per entry kept in tensor memory; the
// epilogue hands each thread its row's 64 sums.  The result is the exact
// integer sum_k N_A N_B (|N_A N_B| <= 2^46, so up to 2^16 K-values).
//
// Digit splitting for error-free matrix products: Ozaki, Ogita, Oishi and
// Rump, Numer. Algorithms 59 (2012).
#pragma once

#include <cstdint>

#include "tc100.cuh"

namespace ttn {

static constexpr int G_KT = 32;                  // K-values per tile
static constexpr int G_TA = 128;                 // A rows per tile (MMA M)
static constexpr int G_TB = 64;                  // B rows per tile (MMA N)
static constexpr int G_TILE = G_TA * G_KT;       // bf16 elements of an A tile (8 KB)
static constexpr int G_TILE_B = G_TILE * 2;      // its bytes
static constexpr int G_SBO = G_KT / 8 * 128;     // bytes between 8-row groups of a tile
static constexpr int G_CHUNK = 256 / G_KT;       // K-tiles per exact FP32 accumulation
static constexpr int G_NS = 3;                   // pipeline stages
static constexpr int G_STAGE = 3 * G_TILE_B + 3 * (G_TILE_B / 2);  // A digits + B digits
static constexpr int G_SMEM = G_NS * G_STAGE;    // dynamic shared memory of a digit_gemm kernel
static constexpr uint32_t G_WAIT = 1u << 22;     // polls of a bounded mbarrier wait
// CTAs per trajectory of a digit-product kernel: each loops over the tiles
// its trajectory's actual shape needs (a grid sized by capacities would
// launch thousands of idle CTAs, each holding G_SMEM of shared memory while
// other streams' kernels wait for room)
static constexpr int G_CTAS = 64;
// tensor memory: five 64-column FP32 accumulators (columns 0..319), then the
// rows' 64-bit sums as low (320..383) and high (384..447) words
static constexpr int G_TMEM_COLS = 512;
static constexpr int G_TM_LO = 5 * G_TB, G_TM_HI = 6 * G_TB;

// Offset (bf16 units) of element (row r, K-value k) inside a digit tile.
__host__ __device__ __forceinline__ int digit_offset(int r, int k) {
  return (r >> 3) * (G_SBO / 2) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// Signed digits of x scaled by 2^(23 - e) (|x| < 2^e): x ~ (n1 2^16 + n2 2^8 + n3) 2^(e - 23).
__device__ __forceinline__ void digits3(float x, int e, int& n1, int& n2, int& n3) {
  const int N = __float2int_rn(ldexpf(x, 23 - e));
  n1 = (N + 32768) >> 16;
  const int r1 = N - n1 * 65536;
  n2 = (r1 + 128) >> 8;
  n3 = r1 - n2 * 256;
}

// A CTA computes one or more 128 x 64 tiles D = sum over K-tiles of A B^T,
// exactly, between digit_begin (mbarriers, tensor memory) and digit_end
// (release).  The tensor memory is allocated once per CTA: a CTA may not
// allocate again after it relinquishes its allocation permit.  The barrier
// phases run on across tiles, so the context counts, per pipeline stage, the
// loads issued and waited and the MMA commits.
struct DigitShared {
  uint64_t bar_load[G_NS], bar_mma[G_NS], bar_acc;
  uint32_t tmem_slot;
  int abort;
};

struct DigitCtx {
  uint32_t tmem;
  uint32_t issued[G_NS];     // bulk loads issued into each stage (thread 0)
  uint32_t waited[G_NS];     // of those, completions waited for (thread 0)
  uint32_t commits[G_NS];    // MMA commits reading each stage (thread 0)
  uint32_t acc_phase;        // completed phases of bar_acc (every thread)
};

// All 128 threads of the CTA.
__device__ __forceinline__ void digit_begin(DigitShared& sh, DigitCtx& c) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int i = 0; i < G_NS; ++i) {
      tc::mbar_init(&sh.bar_load[i], 1);
      tc::mbar_init(&sh.bar_mma[i], 1);
    }
    tc::mbar_init(&sh.bar_acc, 1);
    tc::mbar_fence_init();
    sh.abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&sh.tmem_slot, G_TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  c.tmem = sh.tmem_slot;
  for (int i = 0; i < G_NS; ++i) c.issued[i] = c.waited[i] = c.commits[i] = 0;
  c.acc_phase = 0;
}

// All 128 threads.  After an expired wait (sh.abort set) thread 0 lets the
// copies and MMAs already issued finish (bounded) before the shared memory
// and the tensor memory are released.
__device__ __forceinline__ void digit_end(DigitShared& sh, DigitCtx& c) {
  const int tid = threadIdx.x, warp = tid >> 5;
  __syncthreads();
  if (tid == 0) {
    if (sh.abort) {
      tc::mma_commit(&sh.bar_acc);
      tc::mbar_wait(&sh.bar_acc, c.acc_phase & 1, G_WAIT);
      for (int st = 0; st < G_NS; ++st)
        if (c.issued[st] > c.waited[st]) tc::mbar_wait(&sh.bar_load[st], (c.issued[st] - 1) & 1, G_WAIT);
    }
    for (int st = 0; st < G_NS; ++st)
      if (c.commits[st] > 0) tc::mbar_wait(&sh.bar_mma[st], (c.commits[st] - 1) & 1, G_WAIT);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(c.tmem, G_TMEM_COLS);
}

// One tile: D = sum over K-tiles [kt0, kt0 + nk) of A B^T, exactly.
// srcA(s, kt) / srcB(s, kt): global address of digit s's A tile (8 KB) / B
// tile (4 KB) for K-tile kt, 16-byte aligned.  epilogue(h, v): thread t
// (row t of the tile) receives its row's sums for columns h*32 .. h*32+31 as
// two's-complement 64-bit integers.  All 128 threads call it, between
// digit_begin and digit_end.  Returns false (sh.abort set, the epilogue not
// called) if a bounded wait expired; the caller then goes to digit_end.
template <typename FA, typename FB, typename FE>
__device__ bool digit_tile(DigitShared& sh, DigitCtx& c, int kt0, int nk, FA srcA, FB srcB, FE epilogue) {
  extern __shared__ __align__(1024) unsigned char g_smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t tmem = c.tmem;
  const uint32_t lane_off = (uint32_t)(warp * 32) << 16;  // this warp's TMEM lane quarter
  auto stage = [&](int st) { return g_smem + st * G_STAGE; };
  auto issue_load = [&](int st, int kt) {
    tc::mbar_expect_tx(&sh.bar_load[st], G_STAGE);
    for (int s = 0; s < 3; ++s) tc::bulk_g2s(stage(st) + s * G_TILE_B, srcA(s, kt), G_TILE_B, &sh.bar_load[st]);
    for (int s = 0; s < 3; ++s)
      tc::bulk_g2s(stage(st) + 3 * G_TILE_B + s * (G_TILE_B / 2), srcB(s, kt), G_TILE_B / 2, &sh.bar_load[st]);
    c.issued[st]++;
  };
  // a stage is reused only after the MMAs that read it completed
  auto stage_free = [&](int st) {
    return c.commits[st] == 0 || tc::mbar_wait(&sh.bar_mma[st], (c.commits[st] - 1) & 1, G_WAIT);
  };
  const uint32_t idesc = tc::instr_desc(1, G_TA, G_TB);
  if (tid == 0 && !sh.abort)
    for (int i = 0; i < G_NS - 1 && i < nk; ++i) {
      if (!stage_free(i)) {
        sh.abort = 1;
        break;
      }
      issue_load(i, kt0 + i);
    }
  bool first_chunk = true;
  bool first[5] = {true, true, true, true, true};
  for (int i = 0; i < nk; ++i) {
    const int st = i % G_NS;
    const bool chunk_end = (i % G_CHUNK) == G_CHUNK - 1 || i == nk - 1;
    if (tid == 0 && !sh.abort) {
      if (!tc::mbar_wait(&sh.bar_load[st], c.waited[st] & 1, G_WAIT)) {
        sh.abort = 1;
      } else {
        c.waited[st]++;
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
        tc::mma_commit(&sh.bar_mma[st]);
        c.commits[st]++;
        // tile i + NS - 1 goes into the stage tile i - 1 used, once its MMAs are done
        const int nx = i + G_NS - 1;
        if (nx < nk) {
          const int so = nx % G_NS;
          if (!stage_free(so)) sh.abort = 1;
          else issue_load(so, kt0 + nx);
        }
        if (chunk_end) tc::mma_commit(&sh.bar_acc);
      }
    }
    if (chunk_end) {
      __syncthreads();
      if (sh.abort) return false;
      // every thread polls; the block agrees on the outcome before the
      // warp-collective TMEM loads
      const int ok = __syncthreads_and(tc::mbar_wait(&sh.bar_acc, c.acc_phase & 1, G_WAIT) ? 1 : 0);
      c.acc_phase++;
      if (!ok) {
        if (tid == 0) sh.abort = 1;
        __syncthreads();
        return false;
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
  if (nk <= 0) return true;
  tc::tc_fence_after();
  for (int h = 0; h < G_TB / 32; ++h) {
    uint32_t lo[32], hi[32];
    tc::tmem_ld32(tmem + lane_off + G_TM_LO + h * 32, lo);
    tc::tmem_ld32(tmem + lane_off + G_TM_HI + h * 32, hi);
    tc::tmem_ld_wait();
    unsigned long long v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = ((unsigned long long)hi[j] << 32) | lo[j];
    epilogue(h, v);
  }
  // every thread's TMEM reads are done before the next tile's MMAs overwrite
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  return true;
}

// One tile in its own digit_begin / digit_end.
template <typename FA, typename FB, typename FE>
__device__ bool digit_gemm(int kt0, int nk, FA srcA, FB srcB, FE epilogue) {
  __shared__ DigitShared sh;
  DigitCtx c;
  digit_begin(sh, c);
  const bool ok = digit_tile(sh, c, kt0, nk, srcA, srcB, epilogue);
  digit_end(sh, c);
  return ok;
}

}  // namespace ttn

// Exact Gram matrix G = M^H M of complex64 bond matrices on the tensor cores
// (host interface).  See gram.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ttn {

struct GramArgs {
  const float2* M = nullptr;            // per trajectory b: M + b * mstride, m x n row-major complex64
  int64_t mstride = 0;
  const int2* shape = nullptr;          // [B] (m, n) of each trajectory's matrix (n = 0: skip)
  unsigned int* amax = nullptr;         // [B][cstride] |column| maxima (float bits), zero between calls
  int* expo = nullptr;                  // [B][cstride] column exponents
  int cstride = 0;                      // >= 2 n_cap
  uint16_t* slices = nullptr;           // [B][sstride] bf16 digit tiles
  int64_t sstride = 0;
  unsigned long long* gfix = nullptr;   // [B][gld * gld] fixed-point sums, zero between calls
  int gld = 0;                          // >= 2 n_cap
  double2* G = nullptr;                 // [B][g64stride] output n x n row-major complex128
  int64_t g64stride = 0;
  int32_t* err = nullptr;               // [B] error flags (or null)
  unsigned long long* ledger = nullptr; // profiling ledger (or null)
  int ledger_class = -1;
};

// Bytes of digit tiles one m x n matrix needs (the sstride a caller must
// provide for it).
int64_t gram_slice_elems(int64_t m, int n);

// Launches the five kernels for trajectories [0, B) on `st`; n_cap / m_cap
// bound every trajectory's n and m (grid sizes).  No host synchronisation.
cudaError_t gram_exact_launch(const GramArgs& a, int B, int n_cap, int64_t m_cap, cudaStream_t st);

// Error flag raised when a bounded wait of the tensor-core kernel expires or
// a matrix exceeds its workspace.
static constexpr int32_t GRAM_ERR_TIMEOUT = 16;
static constexpr int32_t GRAM_ERR_CAPACITY = 4;

}  // namespace ttn

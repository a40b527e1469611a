// Exact tensor-core contractions of a centre move (contract.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ttn {

// Per-trajectory operands of the two contractions of a move v -> w.  All
// device pointers; trajectory b's data at base + b * stride.
struct ContractArgs {
  const int32_t* dims;  // [B][ds] bond dimensions (the moved bond already holds k)
  int ds;
  int v, w;             // the move's nodes
  int leg_v;            // leg of v towards w (0 l, 1 r, 2 u)
  int leg_w;            // leg of w towards v
  const int32_t* nold;  // [B] bond dimension n before the move
  const int32_t* knew;  // [B] kept rank k
  const float2* M;      // [B][mstride] bond matrix M (m x n row-major complex64)
  int64_t mstride;
  const float2* V;      // [B][vstride] V_k (n x k row-major complex64)
  const float2* Rm;     // [B][vstride] R (k x n row-major complex64)
  int64_t vstride;
  float2* T;            // node tensors; T_v at T + b * tstride + off_v, T_w at + off_w
  int64_t tstride, off_v, off_w;
  float2* W;            // [B][wstride] absorb output (w's tensor with bond k)
  int64_t wstride;
  uint16_t* slices;     // [B][sstride] bf16 digit tiles
  int64_t sstride;
  int* expo;            // [B][rows_cap] row exponents
  int rows_cap;
  int32_t* err;         // [B] error flags (may be null)
  unsigned long long* ledger;  // profiling ledger (may be null)
  int ledger_form, ledger_absorb;  // ledger classes (-1: not recorded)
};

enum : int32_t { CONTRACT_ERR_CAPACITY = 4, CONTRACT_ERR_TIMEOUT = 16 };

// bf16 elements of digit tiles for Y = M V_k (m x n times n x k) and for
// R T_w (k x n times n x J).
int64_t contract_form_elems(int64_t m, int n, int k);
int64_t contract_absorb_elems(int n, int k, int64_t J);

// Launches for B trajectories; the caps bound the grids.
cudaError_t contract_form_launch(const ContractArgs& a, int B, int64_t m_cap, int n_cap, int k_cap, cudaStream_t st);
cudaError_t contract_absorb_launch(const ContractArgs& a, int B, int n_cap, int k_cap, int64_t J_cap,
                                   cudaStream_t st);

}  // namespace ttn

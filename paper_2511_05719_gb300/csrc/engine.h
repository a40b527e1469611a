// Host-facing entry points of the CUDA engine and decoder.
#pragma once

#include <cstddef>
#include <cstdint>

#include "internal.h"

namespace ttn {

struct RunRequest {
  int noise = 0, chi = 1, precision = 0;
  double theta = 0.0, gamma = 0.0, svd_eps = 0.0;
  uint64_t seed = 0, first_traj = 0, n_traj = 0;
  const double* theta_per_traj = nullptr;  // host, [n_traj]
  const double* gamma_per_traj = nullptr;
  int last_layer = -1;           // >= 0: stop after this layer (debug)
  double* debug_amps = nullptr;  // host [2^N * 2], with last_layer, one trajectory
  void* stream = nullptr;
  size_t max_device_bytes = 0;   // 0: 80% of free device memory
  int max_batch = 0;             // 0: as many as fit
  int svd_mode = 0;              // 0 auto, 1 one-sided Jacobi on M, 2/3 Gram matrix
  int gemm_mode = 0;             // 0 auto, 1 FMA units, 2 tensor cores for FP32 contractions
  int grad_wrt = -1;             // -1 none, 0 theta, 1 gamma: replay for the score
  double grad_h = 1e-4;          // replay step
};

struct RunOutputs {
  bool on_device = false;        // output pointers are device pointers
  bool fail_on_device = false;
  uint8_t* records = nullptr;
  uint8_t* fail = nullptr;
  double* log_prob = nullptr;
  double* discarded = nullptr;
  int32_t* near_ties = nullptr;
  double* score = nullptr;       // host [n_traj], with grad_wrt >= 0
  int err_flags = 0;
  uint64_t lost = 0;             // trajectories whose state lost its norm (fail byte 3)
  int batch = 0;
  size_t bytes_per_traj = 0;
  int decode_overflow = 0;
};

// Kernel classes of the profiling ledger.
enum KernelClass { KC_SVD = 0, KC_GRAM = 1, KC_EIG = 2, KC_FORMU = 3, KC_ABSORB = 4, KC_COPY = 5,
                   KC_OTHER = 6, KC_LOCAL = 7, NCLASS = 8 };
// Phases of the tridiagonal eigensolver timed by the ledger: tridiagonalise,
// phases/split, bisection, eigenvectors (inverse iteration + Gram-Schmidt),
// Rayleigh-Ritz, back-transformation.
static constexpr int EIG_PHASES = 6;
// Move-shape histogram of the profiling ledger: for every centre move
// (truncating or not) and bond dimension n before the move (clamped to
// MOVE_HIST_N - 1): number of moves, sum of m (rows of the bond matrix), sum
// of the kept rank k and SM cycles the Gram eigensolver spent on them (thread
// 0's clock from kernel entry to the rank selection), summed over
// trajectories.
static constexpr int MOVE_HIST_N = 513;
static constexpr int MOVE_HIST_F = 4;
static constexpr int MOVE_HIST_WORDS = 2 * MOVE_HIST_N * MOVE_HIST_F;

// Process-wide profiling state: while active, every run adds algorithmic
// flops/bytes per class to `ledger`, and launches of class `timed_class`
// (every class when timed_class == NCLASS) are bracketed by CUDA events whose
// elapsed times accumulate in `ms` and per class in `class_ms`.
struct Profile {
  bool active = false;
  int timed_class = -1;
  double ms = 0.0;
  uint64_t launches = 0;
  double flops[NCLASS] = {0};
  double bytes[NCLASS] = {0};
  uint64_t class_launches[NCLASS] = {0};
  double class_ms[NCLASS] = {0};
  double eig_phase_cycles[EIG_PHASES] = {0};
  double move_hist[MOVE_HIST_WORDS] = {0};
  uint64_t kernels = 0;          // kernel launches of the library (every class, decoder included)
};
Profile& profile();

ttn_status run_trajectories_device(const ttn_circuit& c, const RunRequest& rq, RunOutputs& out);

// Device bytes one trajectory of this circuit and request occupies (host-side
// sizing only; no CUDA call).
size_t run_bytes_per_traj(const ttn_circuit& c, const RunRequest& rq);

// Worst-case node-slot fill over the step program (host only; see engine.cu).
void slot_check(const ttn_circuit& c, int noise, int chi, double* worst_fill, int* worst_node,
                int* worst_step, int64_t* binding);

// Decodes nb records that live on the device; fail/color/score are device
// pointers when on_device, else host pointers.
ttn_status decode_device(const ttn_circuit& c, int nb, const uint8_t* d_records, uint8_t* fail,
                         int32_t* color, int64_t* score, void* stream, bool on_device);

// Allocation-free decoding with static device scratch (device pointers).
ttn_status decode_noalloc(const ttn_circuit& c, uint64_t n, const uint8_t* d_records, uint8_t* d_fail,
                          int32_t* d_color, int64_t* d_score, void* stream);

// Pipelined resident batch (see engine.cu).
struct PipelineImpl;
ttn_status pipeline_create(const ttn_circuit& c, const RunRequest& rq, int n_resident, int n_segments,
                           const double* theta_cycle, int n_theta, void* stream, PipelineImpl** out);
ttn_status pipeline_step(PipelineImpl* p, uint8_t* fail, double* log_prob, double* discarded, uint64_t* traj,
                         int32_t* n_done, bool on_device, void* stream);
int pipeline_group_size(const PipelineImpl* p);
int pipeline_segment_ms(const PipelineImpl* p, double* ms);
void pipeline_free(PipelineImpl* p);

ttn_status philox_uniforms_device(uint64_t seed, const uint64_t* trajs, uint64_t n_traj,
                                  const int32_t* events, int32_t n_events, double* out);

}  // namespace ttn

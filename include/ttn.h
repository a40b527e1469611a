/*
 * ttn.h -- C ABI of the GB300 tree-tensor-network trajectory simulator for
 * color-code syndrome-extraction circuits (arXiv 2511.05719).
 *
 * Everything is plain C: integers, doubles, host or device pointers, sizes.
 * No function throws; every call returns a ttn_status and leaves a message for
 * ttn_last_error() (thread-local) when it fails.
 *
 * Ownership: the caller owns every input and output buffer.  The library owns
 * the circuit handle and the device memory it allocates for a run (released
 * when the call returns, except the per-handle cache freed by
 * ttn_free_circuit).
 *
 * Pointers: when `cuda_stream` is NULL all buffers are host pointers and the
 * call is synchronous; otherwise they are device pointers and the work is
 * ordered on that stream (the call still synchronises before returning the
 * status, so the outputs are ready when it returns).
 */
#ifndef TTN_H
#define TTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TTN_OK = 0,
  TTN_EINVAL = 1,       /* bad argument (message says which)                 */
  TTN_ENOMEM = 2,       /* device or host allocation failed                  */
  TTN_ECUDA = 3,        /* a CUDA call failed                                */
  TTN_ETIMEOUT = 4,     /* a device-side bounded wait expired                */
  TTN_EUNSUPPORTED = 5, /* valid request this build does not implement       */
  TTN_EOVERFLOW = 6,    /* a per-shot bound was exceeded (message says which)*/
  TTN_ENUMERIC = 7      /* a trajectory's state lost its norm or became
                           non-finite (message names the trajectory and the
                           step); no result of the call is valid            */
} ttn_status;

/* Error channel after every layer on every qubit the layer does not measure
 * (Sec. III.A, Fig. 1b-d).  SRX: exp(-i theta X) (Eq. 1).  AD: Kraus operators
 * of Eqs. 2-3, unravelled exactly.  *_PTA: Pauli-twirled channel (Sec. IV.C):
 * SRX -> X with prob. sin^2 theta; AD -> (I,X,Y,Z) with probabilities
 * ((1+sqrt(1-g))^2/4, g/4, g/4, (1-sqrt(1-g))^2/4).  SRX_AD: SRX then AD.
 * DEPOL: single-qubit depolarizing noise (Sec. III.A's Pauli benchmark model,
 * applied at the same locations): X, Y, Z each with probability gamma / 3;
 * gamma is its strength p. */
typedef enum {
  TTN_NOISE_NONE = 0,
  TTN_NOISE_SRX = 1,
  TTN_NOISE_AD = 2,
  TTN_NOISE_SRX_PTA = 3,
  TTN_NOISE_AD_PTA = 4,
  TTN_NOISE_SRX_AD = 5,
  TTN_NOISE_DEPOL = 6
} ttn_noise;

/* Arithmetic of the tree tensors.  FP64: complex128 throughout.  FP32:
 * complex64 tensors and singular value decompositions, with probabilities,
 * log-probabilities and discarded weights accumulated in double.  MIXED:
 * complex64 tensors and contractions, with every isometry-centre
 * factorisation in FP64 -- the Gram matrix of the bond matrix formed exactly
 * on the tensor cores (see ttn_gram_exact), its Hermitian eigendecomposition
 * (cyclic Jacobi for bonds up to 64, tridiagonal above), the kept rank and
 * the singular values in double -- and probabilities, log-probabilities and
 * discarded weights in double.  svd_mode is ignored in MIXED runs; their
 * contractions Y = M V_k and the neighbour absorb run on the FP32 FMA units
 * unless gemm_mode asks for the exact digit products on the tcgen05 tensor
 * cores (3, one final rounding to complex64) or the 3xTF32 tile (2). */
typedef enum { TTN_PREC_FP64 = 0, TTN_PREC_FP32 = 1, TTN_PREC_MIXED = 2 } ttn_precision;

/* Qubit -> TTN leaf assignment (App. B).  DEFAULT: qubit i on leaf i.
 * OPTIMIZED: recursive spectral bisection of the gate-similarity graph
 * (Eq. 9).  EXPLICIT: the caller's leaf_of_qubit array.  SEARCH: among
 * TTN_LAYOUT_SEARCH_CANDIDATES candidates -- OPTIMIZED, bisections of
 * similarities with off-diagonal entries scaled by seeded factors in
 * [0.95, 1.05], and seeded runs of Algorithm 1 (k-way spectral clustering
 * merged into two groups, random even split as fallback) -- the one with the
 * smallest noise-free bond dimension (ttn_layout_noise_free_chi) is kept,
 * the earlier on ties (App. B samples candidates and keeps the smallest
 * chi_exact; this cost needs no simulation of the noisy circuit, and under
 * strong noise it ranks layouts less well).  Costs under a second of host time at
 * d = 7, C = 7. */
typedef enum {
  TTN_LAYOUT_DEFAULT = 0,
  TTN_LAYOUT_OPTIMIZED = 1,
  TTN_LAYOUT_EXPLICIT = 2,
  TTN_LAYOUT_SEARCH = 3
} ttn_layout;
#define TTN_LAYOUT_SEARCH_CANDIDATES 16

typedef struct {
  int32_t distance;              /* code distance d: odd, 3..11          */
  int32_t rounds;                /* C >= 1 syndrome-extraction cycles    */
  int32_t layout;                /* ttn_layout                           */
  const int32_t* leaf_of_qubit;  /* [n_qubits] distinct leaves in [0, 2^D),
                                    EXPLICIT only; copied by the call     */
} ttn_circuit_params;

typedef struct {
  int32_t noise;                 /* ttn_noise                            */
  double theta;                  /* SRX angle of Eq. 1 (rad)             */
  double gamma;                  /* AD probability of Eq. 2              */
  int32_t chi;                   /* bond-dimension cap, 1..4096.  Inside a
                                    gate a bond reaches 2 chi; in FP32 the
                                    Gram-path eigensolver takes bonds up to
                                    512, so a larger bond on that path (chi
                                    above 256 on a circuit whose bonds grow
                                    that far) stops the run with a capacity
                                    error (ECUDA); svd_mode 1 has no such
                                    limit                                 */
  int32_t precision;             /* ttn_precision                        */
  uint64_t seed;                 /* Philox key                           */
  uint64_t first_traj;           /* index of the first trajectory        */
  double svd_eps;                /* singular values <= svd_eps * s_max are
                                    dropped; <= 0 selects 1e-13 (FP64),
                                    5e-7 (FP32) or 1e-6 (MIXED)           */
  const double* theta_per_traj;  /* optional [n_traj], overrides theta    */
  const double* gamma_per_traj;  /* optional [n_traj], overrides gamma    */
  int32_t svd_mode;              /* factorisation of a centre move:
                                    0 auto (FP64: Jacobi; FP32: Gram for
                                      bonds above 64 and, with the
                                      tridiagonal eigensolver, for every
                                      move of a tensor of 2^17 elements or
                                      more and of a circuit above 32
                                      qubits),
                                    1 one-sided Jacobi on the tensor,
                                    2 Gram matrix; eigensolver two-sided
                                      Jacobi in shared memory up to 128 KB
                                      of Gram matrix, tridiagonal above,
                                    3 Gram matrix, tridiagonal eigensolver
                                      at every size                       */
  int32_t gemm_mode;             /* FP32 contractions (Gram matrix, Y = M V,
                                    neighbour absorb): 0 auto (tensor cores
                                    on Gram-path moves), 1 FP32 FMA units,
                                    2 tensor cores for every move.  Tensor
                                    cores use TF32 with a 3-term split
                                    (FP32-level accuracy).  MIXED runs: 0
                                    and 1 FMA, 2 the 3xTF32 tile, 3 exact
                                    tcgen05 digit products.  FP64 runs
                                    ignore it.                            */
} ttn_run_params;

typedef struct ttn_circuit ttn_circuit;  /* opaque, library-owned */

/* Builds the color code [[ (3d^2+1)/4, 1, d ]] (Sec. II.A), its C-cycle
 * syndrome-extraction circuit with noise locations (Sec. III, Fig. 1a), the
 * qubit-to-leaf layout (App. B) and the decoder graphs (App. A.2).
 * EINVAL on a bad distance, rounds, layout or explicit leaf map. */
ttn_status ttn_build_circuit(const ttn_circuit_params* params, ttn_circuit** out);
void ttn_free_circuit(ttn_circuit* circuit);

/* Sizes: qubits N = n + 2 * #plaquettes, data n, layers, record bits per
 * trajectory (rounds * 2 * #plaquettes syndrome bits -- round, plaquette,
 * Z before X -- then the n final data bits), stochastic events, ops, leaves. */
ttn_status ttn_circuit_info(const ttn_circuit* circuit, int32_t* n_qubits, int32_t* n_data,
                            int32_t* n_layers, int32_t* n_record_bits, int32_t* n_events,
                            int32_t* n_ops, int32_t* n_leaves);

/* The op list, 6 int32 per op: kind (PREP_Z 0, PREP_X 1, CNOT 2, MEAS_Z 3,
 * MEAS_X 4, NOISE 5), a (qubit / control), b (target / location id), event id
 * (-1 if none), record bit (-1 if none), layer.  ops: host [n_ops][6]. */
ttn_status ttn_circuit_ops(const ttn_circuit* circuit, int32_t* ops);

/* Bond dimension the noise-free circuit needs on a layout (host only, no
 * GPU): the largest Schmidt rank across any tree bond after any layer,
 * from a stabilizer tableau of the circuit without its noise operations
 * (the noise-free limit of chi_exact, App. B, Table III).  leaf_of_qubit:
 * host [n_qubits] distinct leaves, or NULL for the circuit's own layout.
 * chi: host scalar (INT64_MAX if above 2^61). */
ttn_status ttn_layout_noise_free_chi(const ttn_circuit* circuit, const int32_t* leaf_of_qubit,
                                     int64_t* chi);

/* The qubit -> leaf map in use.  leaf_of_qubit: host [n_qubits]. */
ttn_status ttn_circuit_layout(const ttn_circuit* circuit, int32_t* leaf_of_qubit);

/* Runs trajectories first_traj .. first_traj + n_traj - 1 (Sec. III.C): the
 * whole circuit on the TTN, Born-sampled measurements, Kraus-branch or Pauli
 * draws from Philox4x32-10 keyed by (seed, trajectory, event), then decodes
 * (App. A.2).  Outputs (any may be NULL): records [n_traj][n_record_bits]
 * (u8 0/1), logical_fail [n_traj] (u8: 0/1 decoded logical outcome, 2 the
 * decoder's bound was exceeded), log_prob [n_traj] (log p of the
 * sampled record and branches), discarded [n_traj] (sum of discarded
 * squared singular values), near_ties [n_traj] (draws with |u - p| < 1e-9
 * (FP64) or 1e-5 (FP32)).  Records and fail bytes depend only on (seed,
 * trajectory index), not on batching (except draws within rounding of a
 * probability); log_prob and discarded agree across batchings to rounding,
 * since a few of their FP64 reductions are atomic and order-dependent.  EOVERFLOW if a decoding instance exceeds the decoder's
 * bound; ENOMEM if one trajectory does not fit on the device; ENUMERIC if a
 * trajectory's state lost its norm or became non-finite (the whole call
 * fails: leaving such a trajectory out would bias p_L). */
ttn_status ttn_run_trajectories(const ttn_circuit* circuit, const ttn_run_params* params,
                                uint64_t n_traj, uint8_t* records, uint8_t* logical_fail,
                                double* log_prob, double* discarded, int32_t* near_ties,
                                void* cuda_stream);

/* Mixed batch (the paper runs one (d, chi) configuration at a time; this
 * serves sweeps that mix distances, bond dimensions and noise strengths, with
 * each item's trajectories independent of the others as in Sec. III.C).
 * Item i runs n_traj[i] trajectories of circuits[i] under params[i] (its
 * own noise model, strengths, chi, precision, seed and first_traj; per-
 * trajectory strengths as in ttn_run_trajectories) and writes their fail
 * bytes (meaning as in ttn_run_trajectories) to logical_fail[i]
 * ([n_traj[i]] u8; may be NULL for an item with n_traj[i] == 0) and, when
 * log_prob and log_prob[i] are non-NULL, the log-probabilities of the
 * sampled records to log_prob[i] ([n_traj[i]] double).  Outputs are DEVICE
 * pointers when cuda_stream is non-NULL, else host.  Every item's results equal
 * those of ttn_run_trajectories with the same arguments.  All items are in
 * flight at once, each on its own stream created by the library (from one
 * host thread per item), so that items whose kernels fill few SMs overlap;
 * they start after the work queued on cuda_stream and are complete when the
 * call returns.  The device budget (80 % of free memory) is split over the
 * items in proportion to n_traj[i] x the item's bytes per trajectory when
 * they do not all fit, and each item runs in chunks within its share.  While
 * the profiler is active the items run one after another.  n_items in
 * [1, TTN_MIXED_MAX_ITEMS].  Returns the lowest-index item's failure (its
 * message prefixed with "item i"), EOVERFLOW only if no item failed
 * otherwise; EINVAL on a bad item before anything runs. */
#define TTN_MIXED_MAX_ITEMS 64
ttn_status ttn_run_mixed(int32_t n_items, const ttn_circuit* const* circuits,
                         const ttn_run_params* params, const uint64_t* n_traj,
                         uint8_t* const* logical_fail, double* const* log_prob,
                         void* cuda_stream);

/* Monte Carlo p_L = failures / valid shots (App. A.3, steps i-iii) with its
 * binomial standard error sigma = sqrt(p (1-p) / valid shots); shots with a
 * fail byte above 1 are not valid.  Host outputs. */
ttn_status ttn_logical_error_rate(const ttn_circuit* circuit, const ttn_run_params* params,
                                  uint64_t shots, double* p_L, double* sigma, uint64_t* n_fail);

/* Gradient of p_L by the score-function estimator (the paper has no
 * gradient; this extends its Monte Carlo step, App. A.3):
 *   dp_L/dx = E[ fail * d/dx log p(trajectory; x) ],  x = theta (wrt 0) or
 * gamma (wrt 1).  Each trajectory is run once, then replayed twice with all its
 * sampled choices (measurement outcomes, damping branches, Pauli draws)
 * forced, at x + h and x - h; the score is the central difference of the
 * replayed log-probabilities (h <= 0 selects 1e-4).  Outputs (host): p_L,
 * dpL, its standard error dpL_sigma, and optionally the per-shot score
 * [shots].  EINVAL when the model does not depend on x. */
ttn_status ttn_grad(const ttn_circuit* circuit, const ttn_run_params* params, uint64_t shots,
                    int32_t wrt, double h, double* p_L, double* dpL, double* dpL_sigma,
                    double* score);

/* Threshold crossing (Sec. IV.A: thresholds are read off where the p_L
 * curves of different distances cross; the paper then fits Eq. 4).  The
 * paper has no search; this locates one crossing directly.
 *
 * ttn_newton_crossing: safeguarded Newton iteration for a root of f(x),
 * whose estimates come from `eval` (called with the point and the
 * 0-based evaluation index; it returns f, its standard error, f' and its
 * standard error, and TTN_OK, or a status that aborts the search and is
 * returned).  The iterate stays in [x_lo, x_hi]; once two evaluations differ
 * in sign their interval is kept as a bracket and a Newton step that leaves
 * it, or a slope within twice its error, is replaced by bisection.  The
 * search stops when a step is below max(x_tol, 2 sigma_x), sigma_x =
 * sigma_f / |f'|, or at max_iter evaluations.  Outputs: x_star (the last
 * Newton or bisection point), x_sigma (sigma_x at the last evaluation; +inf
 * if its slope was not resolved), iters (evaluations made), converged
 * (1 if a stopping rule fired), trace [max_iter][5] (x, f, sigma_f, f',
 * sigma_f' per evaluation).  Any output but x_star may be NULL.  With neither
 * a resolved slope nor a bracket the search stops, not converged.  EINVAL on
 * x_lo >= x_hi, x0 outside, max_iter outside [1, 1000], x_tol <= 0, or
 * non-finite evaluator output. */
typedef ttn_status (*ttn_crossing_eval)(void* ctx, double x, int32_t iter, double* f,
                                        double* f_sigma, double* df, double* df_sigma);
ttn_status ttn_newton_crossing(ttn_crossing_eval eval, void* ctx, double x0, double x_lo,
                               double x_hi, int32_t max_iter, double x_tol, double* x_star,
                               double* x_sigma, int32_t* iters, int32_t* converged,
                               double* trace);

/* The crossing of the p_L(x) curves of circuits a and b (e.g. d = 5 and
 * d = 7), x = theta (wrt 0) or gamma (wrt 1), the other parameters from
 * params: ttn_newton_crossing on f(x) = ln p_L^a(x) - ln p_L^b(x), where
 * each evaluation runs ttn_grad on both circuits with `shots` fresh
 * trajectories (first_traj advances by shots per evaluation), f' = the
 * score-function estimates of d ln p_L / dx, and the errors follow by the
 * delta method.  The logarithm makes power-law failure curves nearly
 * linear near the crossing.  EINVAL as ttn_grad and ttn_newton_crossing, or
 * when a circuit shows no logical failure at an evaluated point. */
ttn_status ttn_crossing(const ttn_circuit* a, const ttn_circuit* b, const ttn_run_params* params,
                        uint64_t shots, int32_t wrt, double h, double x0, double x_lo,
                        double x_hi, int32_t max_iter, double x_tol, double* x_star,
                        double* x_sigma, int32_t* iters, int32_t* converged, double* trace);

/* Threshold fit of Eq. 4 (Sec. IV.A): p_fail = A + B x + C x^2 with
 * x = (p_err - tau) d^(1/nu), by weighted least squares over n points
 * (distance d[i], strength p_err[i], failure rate p_fail[i], its standard
 * error sigma[i] > 0; host arrays).  Levenberg-Marquardt from (tau0, nu0),
 * with A, B, C first solved linearly at that start; stops when an accepted
 * step lowers chi^2 by less than 1e-14 relative, or after max_iter steps.
 * Outputs (host): params[5] = (A, B, C, tau, nu); cov[25] = (J^T W J)^-1 at
 * the optimum, row-major (may be NULL); chi2 (may be NULL); iters (may be
 * NULL).  EINVAL on n < 6, a single distance, d < 2, sigma <= 0,
 * non-finite input, nu0 <= 0, or a singular fit. */
ttn_status ttn_threshold_fit(int32_t n, const int32_t* d, const double* p_err, const double* p_fail,
                             const double* sigma, double tau0, double nu0, int32_t max_iter,
                             double* params, double* cov, double* chi2, int32_t* iters);

/* The sums behind ttn_grad, for combining shards run on several ranks (each
 * rank its own first_traj range; the paper's shots are independent, Sec.
 * III.C): over the valid shots (fail byte <= 1) their number n_valid, the
 * failures n_fail, sum_fs = sum of fail * score and sum_fs2 = sum of
 * (fail * score)^2, the score being ttn_grad's d/dx log p.  Then p_L =
 * n_fail / n_valid, dp_L/dx = sum_fs / n_valid and its standard error
 * sqrt((sum_fs2 / n - (sum_fs / n)^2) / (n - 1)), n = n_valid, exactly as
 * ttn_grad forms them.  Arguments and errors as ttn_grad; outputs are host
 * scalars. */
ttn_status ttn_grad_sums(const ttn_circuit* circuit, const ttn_run_params* params, uint64_t shots,
                         int32_t wrt, double h, uint64_t* n_valid, uint64_t* n_fail,
                         double* sum_fs, double* sum_fs2);

/* Host-only check of the device memory layout (no GPU needed).  Each node
 * of the tree has a fixed slot of 4 cl cr cu elements, c the structural caps
 * min(chi, 2^{qubits on the smaller side}) of its three bonds.  This replays
 * the circuit's step program with every centre move keeping the largest
 * rank its kernels allow (min(n, cap) for the n-column bond matrix, even
 * where rounding exceeds the exact rank; cap = the bond's structural cap
 * when the move truncates, twice that while a gate's operator index rides
 * on the bond) and every threading step doubling bonds as the kernels do,
 * and reports the largest ratio of need to capacity seen over the node
 * slots and the per-trajectory workspaces each step uses (worst_fill; <= 1
 * means no trajectory, whatever its rounding, can overflow either), where
 * (worst_node, worst_step; -1 = the initial state) and how many truncating
 * moves have a structural cap below both chi and n (binding_moves: moves
 * where a cap at chi alone would keep more).  Outputs other than worst_fill
 * may be NULL. */
ttn_status ttn_slot_check(const ttn_circuit* circuit, int32_t noise, int32_t chi,
                          double* worst_fill, int32_t* worst_node, int32_t* worst_step,
                          int64_t* binding_moves);

/* Decodes n records ([n][n_record_bits] u8) with the concatenated MWPM
 * decoder (App. A.2) on the device.  fail [n] u8, color [n] int32 (winning
 * colour), score [n] int64 (total matching weight).  color/score may be NULL. */
ttn_status ttn_decode(const ttn_circuit* circuit, uint64_t n, const uint8_t* records,
                      uint8_t* fail, int32_t* color, int64_t* score, void* cuda_stream);

/* Pipelined resident batch of trajectories (Sec. III.C trajectories, the
 * same semantics and random draws as ttn_run_trajectories).  n_resident
 * trajectories stay on the device in n_segments groups of
 * G = n_resident / n_segments; the circuit's step program is cut into
 * n_segments segments of about equal worst-case cost.  Creating the pipeline
 * runs group g through its first g segments (synchronously on cuda_stream);
 * afterwards every ttn_pipeline_step runs one segment of every group, each
 * group on its own library-created stream ordered after cuda_stream, and the
 * group that finished its last segment is decoded (App. A.2) and restarts
 * with the next G trajectory indices.  So every step completes exactly G
 * trajectories, first_traj, first_traj + 1, ... in order of completion.
 * Trajectory t uses theta_cycle[t % n_theta] as its SRX angle when
 * n_theta > 0 (host array, copied), else params->theta; per-trajectory
 * arrays in params are rejected (EINVAL).  max_device_bytes bounds the
 * resident batch (0: 85 % of free memory; ENOMEM if it does not fit).
 * The groups' streams overlap only if the GPU has as many hardware work
 * queues: set CUDA_DEVICE_MAX_CONNECTIONS (up to 32) above n_segments before
 * the process starts CUDA.  The host enqueues the groups' launches
 * interleaved, TTN_PIPELINE_CHUNK (environment, default 16) program steps of
 * one group at a time.  *out: library-owned handle, released by
 * ttn_pipeline_free. */
typedef struct ttn_pipeline ttn_pipeline;
ttn_status ttn_pipeline_create(const ttn_circuit* circuit, const ttn_run_params* params, int32_t n_resident,
                               int32_t n_segments, const double* theta_cycle, int32_t n_theta,
                               uint64_t max_device_bytes, void* cuda_stream, ttn_pipeline** out);
/* One pipeline step.  Outputs of the G trajectories it completed (any may
 * be NULL): logical_fail [G] (u8 as in ttn_run_trajectories), log_prob [G],
 * discarded [G] -- DEVICE pointers when outputs_on_device, else host -- and
 * traj [G] (host: their trajectory indices), *n_done = G.  Synchronises
 * cuda_stream.  ENUMERIC / ETIMEOUT / ECUDA as in ttn_run_trajectories;
 * EOVERFLOW if a decoding instance exceeded the decoder's bound (fail byte
 * 2, the other outputs valid). */
ttn_status ttn_pipeline_step(ttn_pipeline* pipeline, uint8_t* logical_fail, double* log_prob,
                             double* discarded, uint64_t* traj, int32_t* n_done, int32_t outputs_on_device,
                             void* cuda_stream);
/* G, the trajectories each step completes (0 for NULL). */
int32_t ttn_pipeline_group_size(const ttn_pipeline* pipeline);
/* Device time (ms, CUDA events on the group's stream) each segment took in
 * the last step, ms[0 .. n_segments); returns n_segments (0 for NULL).  The
 * slowest segment sets a step's duration. */
int32_t ttn_pipeline_segment_ms(const ttn_pipeline* pipeline, double* ms);
void ttn_pipeline_free(ttn_pipeline* pipeline);

/* Exact Gram matrix G = M^H M of one complex64 matrix on the tensor cores:
 * the kernel of the isometry-centre factorisation (Sec. III.B: the centre
 * moves by the Schmidt decomposition of a bond matrix; the device path takes
 * it from G's FP64 eigendecomposition).  M: DEVICE m x n row-major complex64
 * (interleaved re, im floats), 8-byte aligned; G: DEVICE n x n row-major
 * complex128, 16-byte aligned, written.  G is exact, up to one final
 * rounding to double, for M with every column rounded to 23 bits below its
 * largest entry (entry error <= 2^-24 max|M_column|).  1 <= n <= 1024,
 * 1 <= m <= 65536 (EINVAL otherwise).  The call allocates and frees its own
 * scratch and synchronises cuda_stream (NULL = default stream); ETIMEOUT if
 * a bounded wait of the tensor-core kernel expires. */
ttn_status ttn_gram_exact(const void* M, int64_t m, int32_t n, void* G, void* cuda_stream);

/* Kept eigenpairs of a batch of Hermitian positive semi-definite Gram
 * matrices: the centre move's FP64 eigensolver (Sec. III.B: the Schmidt
 * decomposition of a bond matrix M, taken from G = M^H M = V S^2 V^H) run on
 * its own.  G: DEVICE [batch][n][n] row-major complex128, 16-byte aligned,
 * read only.  route 0: cyclic Jacobi in shared memory (n^2 <= 8192);
 * 1: Householder tridiagonalisation, Sturm bisection, inverse iteration and
 * a Rayleigh-Ritz step in one CTA per matrix (n <= 512); 2: as 1 with the
 * back-transformation spread over CTAs and V_k rounded to complex64; 3: the
 * MIXED runs' combination -- route 2, with bonds up to 64 taken by the
 * Jacobi body inside the same launch.  Kept: the singular values above eps_keep times the
 * largest (for routes 1 and 2 at least sqrt(2^-52) relative), at most kcap
 * of them, at least one.  Outputs (DEVICE): V [batch][n][kcap] complex128,
 * the k_b kept right singular vectors as columns in descending order,
 * columns k_b.. zero; s [batch][n] all singular values descending; k [batch]
 * the kept ranks.  1 <= kcap <= n <= 512, 0 <= eps_keep < 1 (EINVAL
 * otherwise).  Allocates and frees its own scratch and synchronises
 * cuda_stream; ENUMERIC if a matrix was zero or non-finite or the Jacobi
 * sweeps did not converge. */
ttn_status ttn_eig_gram(const void* G, int32_t batch, int32_t n, int32_t kcap, int32_t route, double eps_keep,
                        void* V, double* s, int32_t* k, void* cuda_stream);

/* Allocation-free variant of ttn_decode.  The paper has no counterpart: it
 * serves callers that cannot allocate device memory -- an application whose
 * memory pool or caching allocator already owns the GPU, or a framework whose
 * allocator hooks forbid direct driver allocations.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: the decoder tables and per-shot
 * scratch live in static device arrays of about 2 MB that every GPU loading
 * the library holds until exit.  records [n][n_record_bits], fail [n], color
 * [n], score [n] are always DEVICE pointers of the current device, ordered on
 * cuda_stream (NULL = the default stream; color/score may be NULL).  Every
 * call copies the packed tables from host memory, decodes NA_SHOTS = 8 shots
 * per launch (one thread per shot, so its throughput is far below
 * ttn_decode's), reads two overflow counters back and synchronises
 * cuda_stream before returning.  Results equal ttn_decode's.  Limits:
 * (rounds + 1) * #faces + 1 <= 145 detector nodes (EINVAL beyond that, e.g.
 * d = 7 with more than 7 rounds); any number of shots.  Every call resolves
 * the static arrays' device addresses on the current device (no allocation;
 * a device reset between calls is safe); the first call on a device may load
 * the module's device code, so make it before any stream capture.  The first
 * call with a circuit packs its decoder tables into host memory kept with the
 * circuit.  All calls share the static arrays, so calls that overlap on the
 * GPU race; order them on one stream. */
ttn_status ttn_decode_noalloc(const ttn_circuit* circuit, uint64_t n, const uint8_t* records,
                              uint8_t* fail, int32_t* color, int64_t* score, void* cuda_stream);

/* Runs one trajectory through the end of `layer` (0-based; -1 = before the
 * first op) and writes its 2^N amplitudes, little-endian in the qubit index
 * (qubit q = bit q), as interleaved (re, im) doubles.  N <= 24, at most 16
 * leaves and chi <= 64.  Host buffer amps [2^N * 2]. */
ttn_status ttn_debug_state(const ttn_circuit* circuit, const ttn_run_params* params,
                           uint64_t traj, int32_t layer, double* amps);

/* Philox4x32-10 uniform draws u(seed, traj_i, event_j) of the simulator, for
 * n_traj x n_events pairs, computed on the device.  out: host [n_traj][n_events]. */
ttn_status ttn_philox_uniforms(uint64_t seed, const uint64_t* trajs, uint64_t n_traj,
                               const int32_t* events, int32_t n_events, double* out);

/* Profiling ledger.  Kernel classes: 0 one-sided Jacobi SVD move, 1 Gram
 * GEMM, 2 Gram eigendecomposition, 3 U = M V GEMM, 4 bond absorption GEMM,
 * 5 tensor copies, 6 other move kernels, 7 gate threading, single-qubit,
 * measurement and damping kernels.  Between ttn_profile_begin(c) and
 * ttn_profile_end, every run adds each class's algorithmic flops and bytes
 * (counted from the live bond dimensions: complex GEMM 8mnk, Jacobi
 * eigensolver 36n^3, tridiagonal eigensolver 16/3 n^3 + 8n^2 k, thin SVD
 * 24mn^2 + 44n^3, bytes = operands read + written) and the device time of
 * every launch of class c (CUDA events on the launch stream; c = -1 times
 * nothing, c = 8 times every class).  flops, bytes, launches: host [8] or
 * NULL.  ttn_profile_class_ms: the timed device milliseconds per class of the
 * current (or last) profile, host [8]. */
ttn_status ttn_profile_begin(int32_t timed_class);
ttn_status ttn_profile_end(double* timed_ms, uint64_t* timed_launches, double* flops,
                           double* bytes, uint64_t* launches);
ttn_status ttn_profile_class_ms(double* class_ms);
/* SM clock cycles of the tridiagonal eigensolver's phases in the current (or
 * last) profile, summed over trajectories (thread 0 of each CTA): tridiagonal
 * reduction, phases/split, bisection, eigenvectors (inverse iteration and
 * Gram-Schmidt), Rayleigh-Ritz, back-transformation.  Host [6]. */
ttn_status ttn_profile_eig_phases(double* cycles);
/* Centre-move shapes of the current (or last) profile, summed over
 * trajectories: hist[(t * 513 + n) * 4 + f] for t = 1 on truncating moves
 * (0 otherwise), n = bond dimension before the move (clamped to 512) and
 * f = 0 number of moves, 1 sum of m (rows of the m x n bond matrix), 2 sum of
 * the kept rank, 3 SM cycles of the Gram eigensolver (kernel entry to rank
 * selection).  Host [2 * 513 * 4].  Profiling only; no Sec. of the paper
 * defines it. */
ttn_status ttn_profile_move_hist(double* hist);
/* Kernel launches of the library in the current (or last) profile: every
 * engine kernel, the tensor-core Gram kernels and the decoder's. */
ttn_status ttn_profile_kernels(uint64_t* kernels);

const char* ttn_status_string(ttn_status status);
const char* ttn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TTN_H */

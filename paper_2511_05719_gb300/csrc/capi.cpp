// extern "C" boundary of the library (declared in include/ttn.h).  Argument
// checking, circuit handles and marshalling; all simulation work runs in the
// CUDA engine and decoder.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "engine.h"
#include "internal.h"

namespace ttn {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ttn

using namespace ttn;

static ttn_status fail_with(ttn_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

extern "C" {

const char* ttn_status_string(ttn_status s) {
  switch (s) {
    case TTN_OK: return "ok";
    case TTN_EINVAL: return "invalid argument";
    case TTN_ENOMEM: return "out of memory";
    case TTN_ECUDA: return "CUDA error";
    case TTN_ETIMEOUT: return "device wait timed out";
    case TTN_EUNSUPPORTED: return "unsupported";
    case TTN_EOVERFLOW: return "per-shot bound exceeded";
    case TTN_ENUMERIC: return "trajectory lost its norm";
  }
  return "unknown status";
}

const char* ttn_last_error(void) { return g_last_error.c_str(); }

ttn_status ttn_build_circuit(const ttn_circuit_params* p, ttn_circuit** out) {
  if (!p || !out) return fail_with(TTN_EINVAL, "null argument");
  *out = nullptr;
  if (p->distance < 3 || p->distance > 11 || p->distance % 2 == 0)
    return fail_with(TTN_EINVAL, "distance must be odd and in [3, 11]");
  if (p->rounds < 1 || p->rounds > 64) return fail_with(TTN_EINVAL, "rounds must be in [1, 64]");
  if (p->layout < TTN_LAYOUT_DEFAULT || p->layout > TTN_LAYOUT_SEARCH)
    return fail_with(TTN_EINVAL, "unknown layout");
  ttn_circuit* c = new (std::nothrow) ttn_circuit();
  if (!c) return fail_with(TTN_ENOMEM, "host allocation failed");
  c->d = p->distance;
  c->C = p->rounds;
  c->code = build_code(c->d);
  c->n = c->code.n;
  c->P = c->code.P;
  c->N = c->n + 2 * c->P;
  c->ops = build_ops(c->code, c->C, &c->n_layers, &c->n_events, &c->n_locations);
  c->n_rec = c->C * 2 * c->P + c->n;
  c->D = 1;
  while ((1 << c->D) < c->N) ++c->D;
  c->L = 1 << c->D;
  if (p->layout == TTN_LAYOUT_DEFAULT) {
    c->leaf_of_qubit.resize(c->N);
    for (int q = 0; q < c->N; ++q) c->leaf_of_qubit[q] = q;
  } else if (p->layout == TTN_LAYOUT_OPTIMIZED) {
    c->leaf_of_qubit = optimized_layout(c->code, c->ops, c->N, c->L);
  } else if (p->layout == TTN_LAYOUT_SEARCH) {
    c->leaf_of_qubit = searched_layout(c->code, c->ops, c->N, c->L, TTN_LAYOUT_SEARCH_CANDIDATES);
  } else {
    if (!p->leaf_of_qubit) {
      delete c;
      return fail_with(TTN_EINVAL, "explicit layout needs leaf_of_qubit");
    }
    std::vector<int> seen(c->L, 0);
    c->leaf_of_qubit.assign(p->leaf_of_qubit, p->leaf_of_qubit + c->N);
    for (int q = 0; q < c->N; ++q) {
      int l = c->leaf_of_qubit[q];
      if (l < 0 || l >= c->L || seen[l]) {
        delete c;
        return fail_with(TTN_EINVAL, "leaf_of_qubit must hold distinct leaves in [0, 2^D)");
      }
      seen[l] = 1;
    }
  }
  c->dec = build_decoder_tables(c->code, c->C);
  *out = c;
  return TTN_OK;
}

void ttn_free_circuit(ttn_circuit* c) { delete c; }

ttn_status ttn_circuit_info(const ttn_circuit* c, int32_t* n_qubits, int32_t* n_data,
                            int32_t* n_layers, int32_t* n_record_bits, int32_t* n_events,
                            int32_t* n_ops, int32_t* n_leaves) {
  if (!c) return fail_with(TTN_EINVAL, "null circuit");
  if (n_qubits) *n_qubits = c->N;
  if (n_data) *n_data = c->n;
  if (n_layers) *n_layers = c->n_layers;
  if (n_record_bits) *n_record_bits = c->n_rec;
  if (n_events) *n_events = c->n_events;
  if (n_ops) *n_ops = (int32_t)c->ops.size();
  if (n_leaves) *n_leaves = c->L;
  return TTN_OK;
}

ttn_status ttn_circuit_ops(const ttn_circuit* c, int32_t* ops) {
  if (!c || !ops) return fail_with(TTN_EINVAL, "null argument");
  for (size_t i = 0; i < c->ops.size(); ++i) {
    const Op& o = c->ops[i];
    int32_t* r = ops + 6 * i;
    r[0] = o.kind;
    r[1] = o.a;
    r[2] = o.b;
    r[3] = o.event;
    r[4] = o.rec;
    r[5] = o.layer;
  }
  return TTN_OK;
}

ttn_status ttn_layout_noise_free_chi(const ttn_circuit* c, const int32_t* leaf_of_qubit, int64_t* chi) {
  if (!c || !chi) return fail_with(TTN_EINVAL, "null argument");
  std::vector<int> lay(c->leaf_of_qubit.begin(), c->leaf_of_qubit.end());
  if (leaf_of_qubit) {
    std::vector<int> seen(c->L, 0);
    for (int q = 0; q < c->N; ++q) {
      const int l = leaf_of_qubit[q];
      if (l < 0 || l >= c->L || seen[l]) return fail_with(TTN_EINVAL, "leaf_of_qubit must hold distinct leaves in [0, 2^D)");
      seen[l] = 1;
      lay[q] = l;
    }
  }
  const int bits = noise_free_bond_bits(c->ops, c->N, c->L, lay);
  *chi = bits >= 62 ? INT64_MAX : ((int64_t)1 << bits);
  return TTN_OK;
}

ttn_status ttn_circuit_layout(const ttn_circuit* c, int32_t* leaf_of_qubit) {
  if (!c || !leaf_of_qubit) return fail_with(TTN_EINVAL, "null argument");
  for (int q = 0; q < c->N; ++q) leaf_of_qubit[q] = c->leaf_of_qubit[q];
  return TTN_OK;
}

static ttn_status check_params(const ttn_circuit* c, const ttn_run_params* p) {
  if (!c || !p) return fail_with(TTN_EINVAL, "null argument");
  if (p->noise < TTN_NOISE_NONE || p->noise > TTN_NOISE_DEPOL) return fail_with(TTN_EINVAL, "unknown noise model");
  if (p->precision != TTN_PREC_FP64 && p->precision != TTN_PREC_FP32 && p->precision != TTN_PREC_MIXED)
    return fail_with(TTN_EINVAL, "unknown precision");
  if (p->chi < 1 || p->chi > 4096) return fail_with(TTN_EINVAL, "chi must be in [1, 4096]");
  if (!std::isfinite(p->theta)) return fail_with(TTN_EINVAL, "theta must be finite");
  if (!(p->gamma >= 0.0 && p->gamma <= 1.0)) return fail_with(TTN_EINVAL, "gamma must be in [0, 1]");
  if (p->svd_mode < 0 || p->svd_mode > 3) return fail_with(TTN_EINVAL, "svd_mode must be 0, 1, 2 or 3");
  if (p->gemm_mode < 0 || p->gemm_mode > 3) return fail_with(TTN_EINVAL, "gemm_mode must be 0, 1, 2 or 3");
  return TTN_OK;
}

static RunRequest make_request(const ttn_run_params* p, uint64_t n_traj, void* stream) {
  RunRequest rq;
  rq.noise = p->noise;
  rq.chi = p->chi;
  rq.precision = p->precision;
  rq.theta = p->theta;
  rq.gamma = p->gamma;
  rq.svd_eps = p->svd_eps > 0 ? p->svd_eps
                              : (p->precision == TTN_PREC_FP64 ? 1e-13 : (p->precision == TTN_PREC_MIXED ? 1e-6 : 5e-7));
  rq.seed = p->seed;
  rq.first_traj = p->first_traj;
  rq.n_traj = n_traj;
  rq.theta_per_traj = p->theta_per_traj;
  rq.gamma_per_traj = p->gamma_per_traj;
  rq.stream = stream;
  rq.svd_mode = p->svd_mode;
  rq.gemm_mode = p->gemm_mode;
  return rq;
}

}  // extern "C"

// One run on `stream` (device outputs when on_device); max_bytes bounds the
// device arena (0: 80 % of free memory).
static ttn_status run_one(const ttn_circuit* c, const ttn_run_params* p, uint64_t n_traj,
                          uint8_t* records, uint8_t* logical_fail, double* log_prob, double* discarded,
                          int32_t* near_ties, void* stream, bool on_device, size_t max_bytes) {
  RunRequest rq = make_request(p, n_traj, stream);
  rq.max_device_bytes = max_bytes;
  if (p->theta_per_traj || p->gamma_per_traj) {
    // per-trajectory strengths are read on the host
    cudaPointerAttributes at{};
    const double* probe = p->theta_per_traj ? p->theta_per_traj : p->gamma_per_traj;
    if (cudaPointerGetAttributes(&at, probe) == cudaSuccess && at.type == cudaMemoryTypeDevice)
      return fail_with(TTN_EINVAL, "theta_per_traj / gamma_per_traj must be host arrays");
    cudaGetLastError();
  }
  RunOutputs out;
  out.on_device = on_device;
  out.fail_on_device = on_device;
  out.records = records;
  out.fail = logical_fail;
  out.log_prob = log_prob;
  out.discarded = discarded;
  out.near_ties = near_ties;
  ttn_status s = run_trajectories_device(*c, rq, out);
  if (s != TTN_OK) return s;
  if (out.decode_overflow > 0) {
    set_error("decoder: " + std::to_string(out.decode_overflow) +
              " shot(s) exceeded the matching bound (fail byte 2)");
    return TTN_EOVERFLOW;
  }
  return TTN_OK;
}

extern "C" {

ttn_status ttn_run_trajectories(const ttn_circuit* c, const ttn_run_params* p, uint64_t n_traj,
                                uint8_t* records, uint8_t* logical_fail, double* log_prob,
                                double* discarded, int32_t* near_ties, void* cuda_stream) {
  ttn_status s = check_params(c, p);
  if (s != TTN_OK) return s;
  if (n_traj == 0) return TTN_OK;
  return run_one(c, p, n_traj, records, logical_fail, log_prob, discarded, near_ties, cuda_stream,
                 cuda_stream != nullptr, 0);
}

ttn_status ttn_run_mixed(int32_t n_items, const ttn_circuit* const* circuits, const ttn_run_params* params,
                         const uint64_t* n_traj, uint8_t* const* logical_fail, double* const* log_prob,
                         void* cuda_stream) {
  if (n_items < 1 || n_items > TTN_MIXED_MAX_ITEMS)
    return fail_with(TTN_EINVAL, "n_items must be in [1, " + std::to_string(TTN_MIXED_MAX_ITEMS) + "]");
  if (!circuits || !params || !n_traj || !logical_fail) return fail_with(TTN_EINVAL, "null argument");
  for (int i = 0; i < n_items; ++i) {
    ttn_status s = check_params(circuits[i], &params[i]);
    if (s != TTN_OK) return fail_with(s, "item " + std::to_string(i) + ": " + ttn_last_error());
    if (n_traj[i] > 0 && !logical_fail[i])
      return fail_with(TTN_EINVAL, "item " + std::to_string(i) + ": null logical_fail");
  }
  // Split the device budget over the items in proportion to what each would
  // hold with all its trajectories resident.
  size_t freeb = 0, totb = 0;
  if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess)
    return fail_with(TTN_ECUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(cudaGetLastError()));
  const double budget = 0.80 * (double)freeb;
  std::vector<double> need(n_items, 0.0);
  double total = 0.0;
  for (int i = 0; i < n_items; ++i) {
    RunRequest rq = make_request(&params[i], n_traj[i], nullptr);
    need[i] = (double)n_traj[i] * (double)run_bytes_per_traj(*circuits[i], rq);
    total += need[i];
  }
  std::vector<size_t> share(n_items, 0);
  for (int i = 0; i < n_items; ++i)
    share[i] = (size_t)(total <= budget ? budget : budget * need[i] / total);
  // Item streams start after the work already queued on the caller's stream.
  std::vector<cudaStream_t> streams(n_items, nullptr);
  cudaEvent_t ready = nullptr;
  auto cleanup = [&]() {
    for (cudaStream_t st : streams)
      if (st) cudaStreamDestroy(st);
    if (ready) cudaEventDestroy(ready);
  };
  for (int i = 0; i < n_items; ++i)
    if (cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      cleanup();
      return fail_with(TTN_ECUDA, "cudaStreamCreateWithFlags failed");
    }
  if (cuda_stream) {
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, (cudaStream_t)cuda_stream) != cudaSuccess) {
      cleanup();
      return fail_with(TTN_ECUDA, "event on the caller's stream failed");
    }
    for (int i = 0; i < n_items; ++i) cudaStreamWaitEvent(streams[i], ready, 0);
  }
  int device = 0;
  cudaGetDevice(&device);
  std::vector<ttn_status> status(n_items, TTN_OK);
  std::vector<std::string> msg(n_items);
  auto work = [&](int i) {
    if (n_traj[i] == 0) return;
    cudaSetDevice(device);  // the current device is per host thread
    status[i] = run_one(circuits[i], &params[i], n_traj[i], nullptr, logical_fail[i],
                        log_prob ? log_prob[i] : nullptr, nullptr, nullptr, streams[i],
                        cuda_stream != nullptr, share[i]);
    if (status[i] != TTN_OK) msg[i] = ttn_last_error();
  };
  if (profile().active || n_items == 1) {
    // the profiler accumulates on the host: keep it on one thread
    for (int i = 0; i < n_items; ++i) work(i);
  } else {
    // no exception may leave the C ABI: items whose thread cannot be
    // created run on the calling thread after the others are started
    std::vector<std::thread> th;
    int started = 0;
    try {
      th.reserve(n_items);
      for (; started < n_items; ++started) th.emplace_back(work, started);
    } catch (...) {
    }
    for (int i = started; i < n_items; ++i) work(i);
    for (std::thread& t : th) t.join();
  }
  cleanup();
  // report the lowest-index failure; decoder overflow (fail byte 2) last
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i < n_items; ++i) {
      const bool over = status[i] == TTN_EOVERFLOW;
      if (status[i] != TTN_OK && over == (pass == 1))
        return fail_with(status[i], "item " + std::to_string(i) + ": " + msg[i]);
    }
  return TTN_OK;
}

ttn_status ttn_logical_error_rate(const ttn_circuit* c, const ttn_run_params* p, uint64_t shots,
                                  double* p_L, double* sigma, uint64_t* n_fail) {
  ttn_status s = check_params(c, p);
  if (s != TTN_OK) return s;
  if (shots == 0) return fail_with(TTN_EINVAL, "shots must be > 0");
  std::vector<uint8_t> fail(shots);
  s = ttn_run_trajectories(c, p, shots, nullptr, fail.data(), nullptr, nullptr, nullptr, nullptr);
  if (s != TTN_OK) return s;
  uint64_t nf = 0, nv = 0;
  for (uint8_t f : fail) {
    nf += f == 1;
    nv += f <= 1;  // 2: decoder bound exceeded
  }
  if (nv == 0) return fail_with(TTN_EOVERFLOW, "no valid shots");
  double pl = (double)nf / (double)nv;
  if (p_L) *p_L = pl;
  if (sigma) *sigma = std::sqrt(pl * (1.0 - pl) / (double)nv);
  if (n_fail) *n_fail = nf;
  return TTN_OK;
}

}  // extern "C"

namespace {
// Runs `shots` trajectories with the score replay and accumulates, over the
// valid shots (fail byte <= 1), their count, failures, sum of fail * score
// and of its square.  EOVERFLOW (after the sums) if some shots exceeded the
// decoder's bound.
struct GradSums {
  uint64_t n = 0, n_fail = 0;
  double s1 = 0.0, s2 = 0.0;
};

ttn_status grad_run(const ttn_circuit* c, const ttn_run_params* p, uint64_t shots, int32_t wrt, double h,
                    GradSums& g, double* score) {
  ttn_status s = check_params(c, p);
  if (s != TTN_OK) return s;
  if (shots < 2) return fail_with(TTN_EINVAL, "shots must be >= 2");
  if (wrt != 0 && wrt != 1) return fail_with(TTN_EINVAL, "wrt must be 0 (theta) or 1 (gamma)");
  if (p->theta_per_traj || p->gamma_per_traj)
    return fail_with(TTN_EINVAL, "ttn_grad takes one theta and one gamma");
  if (h <= 0.0) h = 1e-4;
  if (wrt == 1 && (p->gamma - h < 0.0 || p->gamma + h > 1.0))
    return fail_with(TTN_EINVAL, "gamma +- h must stay in [0, 1]");
  const bool srx_like = p->noise == TTN_NOISE_SRX || p->noise == TTN_NOISE_SRX_PTA || p->noise == TTN_NOISE_SRX_AD;
  const bool ad_like = p->noise == TTN_NOISE_AD || p->noise == TTN_NOISE_AD_PTA || p->noise == TTN_NOISE_SRX_AD ||
                       p->noise == TTN_NOISE_DEPOL;
  if ((wrt == 0 && !srx_like) || (wrt == 1 && !ad_like))
    return fail_with(TTN_EINVAL, "the noise model does not depend on that parameter");
  RunRequest rq = make_request(p, shots, nullptr);
  rq.grad_wrt = wrt;
  rq.grad_h = h;
  std::vector<uint8_t> fail(shots);
  std::vector<double> sc(shots);
  RunOutputs out;
  out.fail = fail.data();
  out.score = sc.data();
  s = run_trajectories_device(*c, rq, out);
  if (s != TTN_OK) return s;
  // score-function estimator: dp_L/dx = E[fail * d/dx log p(trajectory)]
  double n = 0, nf = 0, m1 = 0, m2 = 0;
  for (uint64_t i = 0; i < shots; ++i) {
    if (fail[i] > 1) continue;  // decoder bound exceeded: not counted
    const double f = fail[i];
    const double x = f * sc[i];
    n += 1;
    nf += f;
    m1 += x;
    m2 += x * x;
  }
  g.n = (uint64_t)n;
  g.n_fail = (uint64_t)nf;
  g.s1 = m1;
  g.s2 = m2;
  if (score) std::memcpy(score, sc.data(), sizeof(double) * shots);
  if (out.decode_overflow > 0) {
    set_error("decoder: some shots exceeded the matching bound and were not counted");
    return TTN_EOVERFLOW;
  }
  return TTN_OK;
}
}  // namespace

extern "C" {

ttn_status ttn_grad(const ttn_circuit* c, const ttn_run_params* p, uint64_t shots, int32_t wrt,
                    double h, double* p_L, double* dpL, double* dpL_sigma, double* score) {
  GradSums g;
  ttn_status s = grad_run(c, p, shots, wrt, h, g, score);
  if (s != TTN_OK && s != TTN_EOVERFLOW) return s;
  const double n = (double)g.n;
  if (n < 2) return fail_with(TTN_EOVERFLOW, "no decodable shots");
  const double mean = g.s1 / n, var = fmax(0.0, g.s2 / n - mean * mean);
  if (p_L) *p_L = (double)g.n_fail / n;
  if (dpL) *dpL = mean;
  if (dpL_sigma) *dpL_sigma = std::sqrt(var / (n - 1));
  return s;
}

ttn_status ttn_grad_sums(const ttn_circuit* c, const ttn_run_params* p, uint64_t shots, int32_t wrt,
                         double h, uint64_t* n_valid, uint64_t* n_fail, double* sum_fs,
                         double* sum_fs2) {
  if (!n_valid || !n_fail || !sum_fs || !sum_fs2) return fail_with(TTN_EINVAL, "null argument");
  GradSums g;
  ttn_status s = grad_run(c, p, shots, wrt, h, g, nullptr);
  if (s != TTN_OK && s != TTN_EOVERFLOW) return s;
  *n_valid = g.n;
  *n_fail = g.n_fail;
  *sum_fs = g.s1;
  *sum_fs2 = g.s2;
  return s;
}


ttn_status ttn_newton_crossing(ttn_crossing_eval eval, void* ctx, double x0, double x_lo, double x_hi,
                               int32_t max_iter, double x_tol, double* x_star, double* x_sigma,
                               int32_t* iters, int32_t* converged, double* trace) {
  if (!eval || !x_star) return fail_with(TTN_EINVAL, "null argument");
  if (!(x_lo < x_hi) || !std::isfinite(x_lo) || !std::isfinite(x_hi))
    return fail_with(TTN_EINVAL, "need finite x_lo < x_hi");
  if (!(x0 >= x_lo && x0 <= x_hi)) return fail_with(TTN_EINVAL, "x0 must lie in [x_lo, x_hi]");
  if (max_iter < 1 || max_iter > 1000) return fail_with(TTN_EINVAL, "max_iter must be in [1, 1000]");
  if (!(x_tol > 0.0)) return fail_with(TTN_EINVAL, "x_tol must be > 0");
  // Safeguarded Newton on f(x) = 0.  A bracket [blo, bhi] with f of opposite
  // signs at its ends is kept once two evaluations differ in sign; a Newton
  // step that leaves it, or a slope not resolved above twice its error,
  // falls back to bisection.  Stops when the step is below
  // max(x_tol, 2 sigma_x), sigma_x = sigma_f / |f'| (the estimate is then
  // within its own noise), or when f is exactly zero with nonzero error.
  bool bracketed = false;
  double blo = x_lo, bhi = x_hi, px = 0.0;
  int slo = 0, ps = 0;  // sign of f at blo; sign at the previous point
  double x = x0, est = x0, sig = HUGE_VAL;
  int conv = 0, it = 0;
  while (it < max_iter) {
    double f = 0, sf = 0, df = 0, sdf = 0;
    ttn_status s = eval(ctx, x, it, &f, &sf, &df, &sdf);
    if (s != TTN_OK) {
      if (iters) *iters = it;
      return s;
    }
    if (!std::isfinite(f) || !std::isfinite(df) || !(sf >= 0.0) || !(sdf >= 0.0)) {
      if (iters) *iters = it;
      return fail_with(TTN_EINVAL, "crossing evaluator returned non-finite values");
    }
    if (trace) {
      double* t = trace + 5 * (size_t)it;
      t[0] = x, t[1] = f, t[2] = sf, t[3] = df, t[4] = sdf;
    }
    ++it;
    const bool slope_ok = df != 0.0 && std::fabs(df) > 2.0 * sdf;
    sig = slope_ok ? sf / std::fabs(df) : HUGE_VAL;
    if (f == 0.0 && sf > 0.0) {  // statistically at the crossing
      est = x;
      conv = 1;
      break;
    }
    const int sg = f > 0.0 ? 1 : (f < 0.0 ? -1 : 0);
    if (sg != 0) {
      if (bracketed) {
        if (x > blo && x < bhi) {
          if (sg == slo) blo = x;
          else bhi = x;
        }
      } else if (ps != 0 && sg != ps) {
        bracketed = true;
        blo = std::min(x, px);
        bhi = std::max(x, px);
        slo = x < px ? sg : ps;
      }
      px = x;
      ps = sg;
    }
    double xn;
    if (slope_ok) xn = x - f / df;
    else if (bracketed) xn = 0.5 * (blo + bhi);
    else {  // neither a slope nor a bracket: no step to take
      est = x;
      break;
    }
    if (bracketed && !(xn > blo && xn < bhi)) xn = 0.5 * (blo + bhi);
    xn = std::min(x_hi, std::max(x_lo, xn));
    est = xn;
    if (std::fabs(xn - x) <= std::max(x_tol, 2.0 * sig)) {
      conv = 1;
      break;
    }
    x = xn;
  }
  *x_star = est;
  if (x_sigma) *x_sigma = sig;
  if (iters) *iters = it;
  if (converged) *converged = conv;
  return TTN_OK;
}

}  // extern "C"

namespace {
// f(x) = ln p_L^a(x) - ln p_L^b(x) from two ttn_grad runs of fresh
// trajectories (first_traj advances by `shots` per evaluation).
struct CrossingCtx {
  const ttn_circuit* a;
  const ttn_circuit* b;
  ttn_run_params p;
  uint64_t shots;
  int32_t wrt;
  double h;
};

ttn_status crossing_eval(void* vctx, double x, int32_t iter, double* f, double* f_sigma, double* df,
                         double* df_sigma) {
  const CrossingCtx& c = *static_cast<const CrossingCtx*>(vctx);
  ttn_run_params q = c.p;
  if (c.wrt == 0) q.theta = x;
  else q.gamma = x;
  q.first_traj = c.p.first_traj + (uint64_t)iter * c.shots;
  double pl[2], g[2], sg[2];
  const ttn_circuit* circ[2] = {c.a, c.b};
  for (int i = 0; i < 2; ++i) {
    ttn_status s = ttn_grad(circ[i], &q, c.shots, c.wrt, c.h, &pl[i], &g[i], &sg[i], nullptr);
    if (s != TTN_OK && s != TTN_EOVERFLOW) return s;  // EOVERFLOW: those shots are not counted
    if (!(pl[i] > 0.0))
      return fail_with(TTN_EINVAL, std::string("no logical failures on circuit ") + (i ? "b" : "a") +
                                       " at x = " + std::to_string(x) + ": raise shots or move x0");
  }
  const double n = (double)c.shots;
  *f = std::log(pl[0]) - std::log(pl[1]);
  // delta method: var(ln p) = (1 - p) / (n p); d ln p / dx = p' / p
  *f_sigma = std::sqrt((1.0 - pl[0]) / (n * pl[0]) + (1.0 - pl[1]) / (n * pl[1]));
  *df = g[0] / pl[0] - g[1] / pl[1];
  *df_sigma = std::sqrt((sg[0] / pl[0]) * (sg[0] / pl[0]) + (sg[1] / pl[1]) * (sg[1] / pl[1]));
  return TTN_OK;
}
}  // namespace

extern "C" {

ttn_status ttn_crossing(const ttn_circuit* a, const ttn_circuit* b, const ttn_run_params* params,
                        uint64_t shots, int32_t wrt, double h, double x0, double x_lo, double x_hi,
                        int32_t max_iter, double x_tol, double* x_star, double* x_sigma, int32_t* iters,
                        int32_t* converged, double* trace) {
  ttn_status s = check_params(a, params);
  if (s != TTN_OK) return s;
  s = check_params(b, params);
  if (s != TTN_OK) return s;
  if (shots < 2) return fail_with(TTN_EINVAL, "shots must be >= 2");
  if (wrt != 0 && wrt != 1) return fail_with(TTN_EINVAL, "wrt must be 0 (theta) or 1 (gamma)");
  if (params->theta_per_traj || params->gamma_per_traj)
    return fail_with(TTN_EINVAL, "ttn_crossing takes one theta and one gamma");
  if (h <= 0.0) h = 1e-4;
  if (wrt == 1 && (x_lo - h < 0.0 || x_hi + h > 1.0))
    return fail_with(TTN_EINVAL, "gamma +- h must stay in [0, 1] over [x_lo, x_hi]");
  CrossingCtx ctx{a, b, *params, shots, wrt, h};
  return ttn_newton_crossing(crossing_eval, &ctx, x0, x_lo, x_hi, max_iter, x_tol, x_star, x_sigma, iters,
                             converged, trace);
}

}  // extern "C"

namespace {
// Solves the k x k system M z = v in place by Gaussian elimination with
// partial pivoting; false if M is singular to working precision.
bool solve_small(int k, std::vector<double> M, std::vector<double> v, std::vector<double>& z) {
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int r = c + 1; r < k; ++r)
      if (std::fabs(M[r * k + c]) > std::fabs(M[piv * k + c])) piv = r;
    if (!(std::fabs(M[piv * k + c]) > 1e-300)) return false;
    if (piv != c) {
      for (int j = 0; j < k; ++j) std::swap(M[c * k + j], M[piv * k + j]);
      std::swap(v[c], v[piv]);
    }
    for (int r = c + 1; r < k; ++r) {
      const double m = M[r * k + c] / M[c * k + c];
      for (int j = c; j < k; ++j) M[r * k + j] -= m * M[c * k + j];
      v[r] -= m * v[c];
    }
  }
  z.assign(k, 0.0);
  for (int r = k - 1; r >= 0; --r) {
    double t = v[r];
    for (int j = r + 1; j < k; ++j) t -= M[r * k + j] * z[j];
    z[r] = t / M[r * k + r];
  }
  return true;
}

// Eq. 4 residuals r_i = (A + B x_i + C x_i^2 - y_i) / sigma_i, x_i =
// (p_i - tau) d_i^(1/nu), and their Jacobian [n][5] in (A, B, C, tau, nu).
double eq4_residuals(const double* q, int n, const int32_t* d, const double* p, const double* y,
                     const double* sg, std::vector<double>& r, std::vector<double>* J) {
  double chi2 = 0.0;
  r.resize(n);
  if (J) J->resize((size_t)5 * n);
  for (int i = 0; i < n; ++i) {
    const double ld = std::log((double)d[i]);
    const double s = std::exp(ld / q[4]);  // d^(1/nu)
    const double x = (p[i] - q[3]) * s;
    r[i] = (q[0] + q[1] * x + q[2] * x * x - y[i]) / sg[i];
    chi2 += r[i] * r[i];
    if (J) {
      const double dmdx = q[1] + 2.0 * q[2] * x;
      double* Ji = J->data() + (size_t)5 * i;
      Ji[0] = 1.0 / sg[i];
      Ji[1] = x / sg[i];
      Ji[2] = x * x / sg[i];
      Ji[3] = -dmdx * s / sg[i];
      Ji[4] = -dmdx * x * ld / (q[4] * q[4]) / sg[i];
    }
  }
  return chi2;
}
}  // namespace

extern "C" {

ttn_status ttn_threshold_fit(int32_t n, const int32_t* d, const double* p_err, const double* p_fail,
                             const double* sigma, double tau0, double nu0, int32_t max_iter, double* params,
                             double* cov, double* chi2_out, int32_t* iters) {
  if (!d || !p_err || !p_fail || !sigma || !params) return fail_with(TTN_EINVAL, "null argument");
  if (n < 6) return fail_with(TTN_EINVAL, "need at least 6 points for 5 parameters");
  if (max_iter < 1 || max_iter > 100000) return fail_with(TTN_EINVAL, "max_iter must be in [1, 100000]");
  if (!(nu0 > 0.0) || !std::isfinite(tau0)) return fail_with(TTN_EINVAL, "need finite tau0 and nu0 > 0");
  bool two_d = false;
  for (int i = 0; i < n; ++i) {
    if (d[i] < 2) return fail_with(TTN_EINVAL, "distances must be >= 2");
    if (!(sigma[i] > 0.0) || !std::isfinite(p_err[i]) || !std::isfinite(p_fail[i]))
      return fail_with(TTN_EINVAL, "need finite points and sigma > 0");
    if (d[i] != d[0]) two_d = true;
  }
  if (!two_d) return fail_with(TTN_EINVAL, "need at least two distances");
  // start: (A, B, C) by weighted linear least squares at (tau0, nu0)
  double q[5] = {0.0, 0.0, 0.0, tau0, nu0};
  std::vector<double> r, J;
  eq4_residuals(q, n, d, p_err, p_fail, sigma, r, &J);
  {
    std::vector<double> M(9, 0.0), v(3, 0.0), z;
    for (int i = 0; i < n; ++i) {
      const double* Ji = J.data() + (size_t)5 * i;
      const double yi = p_fail[i] / sigma[i];
      for (int a = 0; a < 3; ++a) {
        v[a] += Ji[a] * yi;
        for (int b = 0; b < 3; ++b) M[a * 3 + b] += Ji[a] * Ji[b];
      }
    }
    if (!solve_small(3, M, v, z)) return fail_with(TTN_EINVAL, "points do not determine A, B, C at the start");
    q[0] = z[0], q[1] = z[1], q[2] = z[2];
  }
  // Levenberg-Marquardt (Marquardt's diagonal scaling)
  double chi2 = eq4_residuals(q, n, d, p_err, p_fail, sigma, r, &J);
  double lambda = 1e-3;
  int it = 0;
  std::vector<double> JTJ(25), g(5), step;
  for (; it < max_iter; ++it) {
    std::fill(JTJ.begin(), JTJ.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    for (int i = 0; i < n; ++i) {
      const double* Ji = J.data() + (size_t)5 * i;
      for (int a = 0; a < 5; ++a) {
        g[a] -= Ji[a] * r[i];
        for (int b = 0; b < 5; ++b) JTJ[a * 5 + b] += Ji[a] * Ji[b];
      }
    }
    bool improved = false;
    double gain = 0.0;
    for (int tries = 0; tries < 40 && !improved; ++tries) {
      std::vector<double> M = JTJ;
      for (int a = 0; a < 5; ++a) M[a * 5 + a] += lambda * std::max(JTJ[a * 5 + a], 1e-300);
      if (!solve_small(5, M, g, step)) {
        lambda *= 10.0;
        continue;
      }
      double qn[5];
      for (int a = 0; a < 5; ++a) qn[a] = q[a] + step[a];
      if (!(qn[4] > 0.0)) {
        lambda *= 10.0;
        continue;
      }
      std::vector<double> rn;
      const double c2 = eq4_residuals(qn, n, d, p_err, p_fail, sigma, rn, nullptr);
      if (std::isfinite(c2) && c2 < chi2) {
        gain = chi2 - c2;
        std::copy(qn, qn + 5, q);
        chi2 = eq4_residuals(q, n, d, p_err, p_fail, sigma, r, &J);
        lambda = std::max(lambda / 10.0, 1e-12);
        improved = true;
      } else {
        lambda *= 10.0;
      }
    }
    if (!improved || gain <= 1e-14 * std::max(chi2, 1e-300)) {
      ++it;
      break;
    }
  }
  for (int a = 0; a < 5; ++a) params[a] = q[a];
  if (chi2_out) *chi2_out = chi2;
  if (iters) *iters = it;
  if (cov) {
    // covariance (J^T W J)^-1 at the optimum, column by column
    std::fill(JTJ.begin(), JTJ.end(), 0.0);
    for (int i = 0; i < n; ++i) {
      const double* Ji = J.data() + (size_t)5 * i;
      for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) JTJ[a * 5 + b] += Ji[a] * Ji[b];
    }
    for (int c = 0; c < 5; ++c) {
      std::vector<double> e(5, 0.0), z;
      e[c] = 1.0;
      if (!solve_small(5, JTJ, e, z)) return fail_with(TTN_EINVAL, "singular normal matrix at the optimum");
      for (int a = 0; a < 5; ++a) cov[a * 5 + c] = z[a];
    }
  }
  return TTN_OK;
}

ttn_status ttn_slot_check(const ttn_circuit* c, int32_t noise, int32_t chi, double* worst_fill,
                          int32_t* worst_node, int32_t* worst_step, int64_t* binding_moves) {
  if (!c || !worst_fill) return fail_with(TTN_EINVAL, "null argument");
  if (noise < TTN_NOISE_NONE || noise > TTN_NOISE_SRX_AD) return fail_with(TTN_EINVAL, "unknown noise model");
  if (chi < 1 || chi > 4096) return fail_with(TTN_EINVAL, "chi must be in [1, 4096]");
  double wf = 0.0;
  int wn = -1, ws = -1;
  int64_t nb = 0;
  slot_check(*c, noise, chi, &wf, &wn, &ws, &nb);
  *worst_fill = wf;
  if (worst_node) *worst_node = wn;
  if (worst_step) *worst_step = ws;
  if (binding_moves) *binding_moves = nb;
  return TTN_OK;
}

ttn_status ttn_decode(const ttn_circuit* c, uint64_t n, const uint8_t* records, uint8_t* fail,
                      int32_t* color, int64_t* score, void* cuda_stream) {
  if (!c || !records || !fail) return fail_with(TTN_EINVAL, "null argument");
  if (n == 0) return TTN_OK;
  if (cuda_stream) return decode_device(*c, (int)n, records, fail, color, score, cuda_stream, true);
  uint8_t* d = nullptr;
  if (cudaMalloc(&d, n * c->n_rec) != cudaSuccess) return fail_with(TTN_ENOMEM, "device allocation failed");
  if (cudaMemcpy(d, records, n * c->n_rec, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return fail_with(TTN_ECUDA, "copy of records failed");
  }
  ttn_status s = decode_device(*c, (int)n, d, fail, color, score, nullptr, false);
  cudaFree(d);
  return s;
}

ttn_status ttn_decode_noalloc(const ttn_circuit* c, uint64_t n, const uint8_t* records, uint8_t* fail,
                              int32_t* color, int64_t* score, void* cuda_stream) {
  if (!c || !records || !fail) return fail_with(TTN_EINVAL, "null argument");
  if (n == 0) return TTN_OK;
  return decode_noalloc(*c, n, records, fail, color, score, cuda_stream);
}

ttn_status ttn_debug_state(const ttn_circuit* c, const ttn_run_params* p, uint64_t traj,
                           int32_t layer, double* amps) {
  ttn_status s = check_params(c, p);
  if (s != TTN_OK) return s;
  if (!amps) return fail_with(TTN_EINVAL, "null amps");
  if (c->N > 24 || c->L > 16) return fail_with(TTN_EUNSUPPORTED, "debug state needs N <= 24 and <= 16 leaves");
  if (p->chi > 64) return fail_with(TTN_EUNSUPPORTED, "debug state needs chi <= 64");
  if (layer < -1 || layer >= c->n_layers) return fail_with(TTN_EINVAL, "layer out of range");
  ttn_run_params q = *p;
  q.first_traj = traj;
  q.theta_per_traj = nullptr;
  q.gamma_per_traj = nullptr;
  RunRequest rq = make_request(&q, 1, nullptr);
  rq.last_layer = layer;
  rq.debug_amps = amps;
  if (p->theta_per_traj) rq.theta = p->theta_per_traj[0];
  if (p->gamma_per_traj) rq.gamma = p->gamma_per_traj[0];
  RunOutputs out;
  return run_trajectories_device(*c, rq, out);
}

ttn_status ttn_profile_begin(int32_t timed_class) {
  if (timed_class < -1 || timed_class > NCLASS) return fail_with(TTN_EINVAL, "unknown kernel class");
  Profile& p = profile();
  p = Profile();
  p.active = true;
  p.timed_class = timed_class;
  return TTN_OK;
}

ttn_status ttn_profile_end(double* timed_ms, uint64_t* timed_launches, double* flops, double* bytes,
                           uint64_t* launches) {
  Profile& p = profile();
  if (!p.active) return fail_with(TTN_EINVAL, "profiling was not started");
  if (timed_ms) *timed_ms = p.ms;
  if (timed_launches) *timed_launches = p.launches;
  for (int c = 0; c < NCLASS; ++c) {
    if (flops) flops[c] = p.flops[c];
    if (bytes) bytes[c] = p.bytes[c];
    if (launches) launches[c] = p.class_launches[c];
  }
  p.active = false;
  return TTN_OK;
}

ttn_status ttn_profile_eig_phases(double* cycles) {
  if (!cycles) return fail_with(TTN_EINVAL, "null argument");
  const Profile& p = profile();
  for (int i = 0; i < EIG_PHASES; ++i) cycles[i] = p.eig_phase_cycles[i];
  return TTN_OK;
}

ttn_status ttn_pipeline_create(const ttn_circuit* c, const ttn_run_params* p, int32_t n_resident,
                               int32_t n_segments, const double* theta_cycle, int32_t n_theta,
                               uint64_t max_device_bytes, void* cuda_stream, ttn_pipeline** out) {
  ttn_status s = check_params(c, p);
  if (s != TTN_OK) return s;
  if (!out) return fail_with(TTN_EINVAL, "null argument");
  *out = nullptr;
  if (n_segments < 1 || n_resident < n_segments || n_resident % n_segments != 0)
    return fail_with(TTN_EINVAL, "n_resident must be a positive multiple of n_segments >= 1");
  if (n_theta < 0 || (n_theta > 0 && !theta_cycle)) return fail_with(TTN_EINVAL, "theta_cycle / n_theta");
  for (int i = 0; i < n_theta; ++i)
    if (!std::isfinite(theta_cycle[i])) return fail_with(TTN_EINVAL, "theta_cycle must be finite");
  if (p->theta_per_traj || p->gamma_per_traj)
    return fail_with(TTN_EINVAL, "per-trajectory strengths: pass theta_cycle to the pipeline");
  RunRequest rq = make_request(p, 0, cuda_stream);
  rq.max_device_bytes = (size_t)max_device_bytes;
  ttn::PipelineImpl* impl = nullptr;
  s = ttn::pipeline_create(*c, rq, n_resident, n_segments, theta_cycle, n_theta, cuda_stream, &impl);
  if (s != TTN_OK) return s;
  *out = reinterpret_cast<ttn_pipeline*>(impl);
  return TTN_OK;
}

ttn_status ttn_pipeline_step(ttn_pipeline* p, uint8_t* logical_fail, double* log_prob, double* discarded,
                             uint64_t* traj, int32_t* n_done, int32_t outputs_on_device, void* cuda_stream) {
  if (!p) return fail_with(TTN_EINVAL, "null pipeline");
  return ttn::pipeline_step(reinterpret_cast<ttn::PipelineImpl*>(p), logical_fail, log_prob, discarded, traj,
                            n_done, outputs_on_device != 0, cuda_stream);
}

int32_t ttn_pipeline_group_size(const ttn_pipeline* p) {
  return p ? ttn::pipeline_group_size(reinterpret_cast<const ttn::PipelineImpl*>(p)) : 0;
}

int32_t ttn_pipeline_segment_ms(const ttn_pipeline* p, double* ms) {
  if (!p || !ms) return 0;
  return ttn::pipeline_segment_ms(reinterpret_cast<const ttn::PipelineImpl*>(p), ms);
}

void ttn_pipeline_free(ttn_pipeline* p) {
  if (p) ttn::pipeline_free(reinterpret_cast<ttn::PipelineImpl*>(p));
}

ttn_status ttn_profile_move_hist(double* hist) {
  if (!hist) return fail_with(TTN_EINVAL, "null argument");
  const Profile& p = profile();
  for (int i = 0; i < MOVE_HIST_WORDS; ++i) hist[i] = p.move_hist[i];
  return TTN_OK;
}

ttn_status ttn_profile_kernels(uint64_t* kernels) {
  if (!kernels) return fail_with(TTN_EINVAL, "null argument");
  *kernels = profile().kernels;
  return TTN_OK;
}

ttn_status ttn_profile_class_ms(double* class_ms) {
  if (!class_ms) return fail_with(TTN_EINVAL, "null argument");
  const Profile& p = profile();
  for (int c = 0; c < NCLASS; ++c) class_ms[c] = p.class_ms[c];
  return TTN_OK;
}

ttn_status ttn_philox_uniforms(uint64_t seed, const uint64_t* trajs, uint64_t n_traj,
                               const int32_t* events, int32_t n_events, double* out) {
  if (!trajs || !events || !out || n_events < 0) return fail_with(TTN_EINVAL, "bad argument");
  if (n_traj == 0 || n_events == 0) return TTN_OK;
  return philox_uniforms_device(seed, trajs, n_traj, events, n_events, out);
}

}  // extern "C"

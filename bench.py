"""Benchmark of the TTN trajectory simulator (one JSON line on rank 0).

Workload: d = 7 color code, 7 rounds, SRX with theta swept over 8 values in
[0.01, 0.15] rad (trajectory t at theta_(t mod 8)), chi = 128, MIXED
precision (complex64 tensors and contractions, FP64 isometry-centre
factorisations, FP64 probabilities).  Inputs are synthetic and seeded (the
paper's workloads are themselves synthetic circuits).

A step is one step of the pipelined resident batch (ttn_pipeline_*):
`--resident` trajectories stay on the device in `--segments` groups; every
step runs one program segment of every group (each group on its own stream)
and completes exactly `resident / segments` whole trajectories -- circuit on
the tree tensor network, Born / Kraus sampling, decoding.  All steps do the
same work (one full trajectory per group), so every timed step is a
steady-state step.  Creating the pipeline (filling it) is untimed.

value: completed trajectories/s with device-side outputs (CUDA events on the
caller's stream, max over ranks).  e2e: the same metric through the same
call with host output buffers (fail byte, log-probability, discarded weight
copied back every step).  Trajectories are sharded across ranks by index (no
collective on the data path: weak scaling).  Every step streams hundreds of
MB per trajectory, far above L2, so no L2 flush is needed between steps.

--impl reference: the CPU oracle (plain numpy TTN, float64) on the host
cores, on the same workload: a complete d = 7, one-round trajectory cut into
`--steps` equal op-count steps, scaled to 7-round trajectories by the number
of rounds.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the pipeline runs one stream per group: give the GPU enough hardware work
# queues that the streams do not share one (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import workloads as WL  # noqa: E402

METRIC = "d=7 trajectories/s (chi=128), batched vs plain at matched p_L; grad/fwd cost"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 (152 SMs x 2 FP64 FMA/clk x 2 flops x ~2.06 GHz)


def peaks():
    """(bf16 sustained TFLOP/s, source) from MEASURED_PEAKS.json, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["bf16_tflops_sustained"]), "of measured (bf16 sustained)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback (bf16 sustained 1.7 PFLOP/s)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ttn", choices=["ttn", "reference"])
    ap.add_argument("--resident", type=int, default=192, help="trajectories on the device per rank")
    ap.add_argument("--segments", type=int, default=32, help="pipeline segments (resident must be a multiple)")
    ap.add_argument("--distance", type=int, default=7)
    ap.add_argument("--rounds", type=int, default=7)
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--precision", default="mixed")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 single-instance leg")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient / forward cost leg")
    return ap.parse_args()


def workload_name(a):
    centre = "fp64centre" if a.precision in ("mixed", "fp64") else "fp32centre"
    return "d%d_C%d_srx_theta_sweep8_chi%d_%s_%s" % (a.distance, a.rounds, a.chi, a.precision, centre)


def run_config(a):
    return {"workload": workload_name(a), "distance": a.distance, "rounds": a.rounds, "chi": a.chi,
            "resident_trajectories": a.resident, "segments": a.segments,
            "trajectories_per_step": a.resident // a.segments,
            "l2": "working set per step far above L2 (no flush)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def oracle_c1_trajectory(a, n_chunks=1, warm_chunks=0):
    """The CPU oracle (plain numpy TTN, float64, threaded BLAS) on one complete
    one-round trajectory of the workload's code (the oracle's own layout,
    App. B), timed in n_chunks equal op-count chunks after warm_chunks chunks
    of an untimed trajectory.  Returns (chunk seconds, total ops, theta)."""
    from oracle.circuit import build_circuit
    from oracle.layout import optimized_layout
    from oracle import ttn as TT
    from oracle.channels import SRX
    circ = build_circuit(a.distance, 1)
    lay = optimized_layout(circ)
    theta = WL.M3["thetas"][3]
    n_ops = len(circ.ops)
    bounds = [round(n_ops * k / n_chunks) for k in range(n_chunks + 1)]
    if warm_chunks > 0:
        TT.run_trajectory(circ, SRX, theta, 0.0, WL.M3["seed"], 1, chi=a.chi, leaf_of_qubit=lay,
                          max_ops=bounds[min(warm_chunks, n_chunks)])
    stamps = {}
    marks = set(bounds[1:])

    def on_op(i):
        if i + 1 in marks:
            stamps[i + 1] = time.perf_counter()

    t0 = time.perf_counter()
    TT.run_trajectory(circ, SRX, theta, 0.0, WL.M3["seed"], 0, chi=a.chi, leaf_of_qubit=lay, on_op=on_op)
    prev, chunks = t0, []
    for b in bounds[1:]:
        chunks.append(stamps[b] - prev)
        prev = stamps[b]
    return chunks, n_ops, theta


def cpu_sample_text(a, n_ops, theta, secs):
    return ("plain numpy TTN oracle (float64, threaded BLAS, oracle-side layout): one complete d=%d "
            "one-round trajectory (%d ops, theta=%.3f, chi=%d) in %.1f s; a %d-round trajectory counted "
            "as %d one-round ones (later rounds cost more, so this overstates the CPU rate)"
            % (a.distance, n_ops, theta, a.chi, secs, a.rounds, a.rounds))


def cpu_baseline(a):
    chunks, n_ops, theta = oracle_c1_trajectory(a)
    secs = sum(chunks)
    return {"value": 1.0 / (a.rounds * secs), "unit": "trajectories/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": cpu_sample_text(a, n_ops, theta, secs)}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    K = max(1, a.steps)
    chunks, n_ops, theta = oracle_c1_trajectory(a, n_chunks=K, warm_chunks=a.warmup)
    secs = sum(chunks)
    v = 1.0 / (a.rounds * secs)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "trajectories/s",
            "n_gpus": a.gpus, "steps": K, "warmup": a.warmup, "ms_per_step": 1e3 * secs / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": run_config(a),
            "cpu_baseline": {"value": v, "unit": "trajectories/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": cpu_sample_text(a, n_ops, theta, secs) +
                             "; %d steps of equal op count" % K},
            "e2e": {"value": v, "unit": "trajectories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def plain_fp64_single(a, P, torch):
    """The plain FP64 single-instance GPU path: one trajectory per call,
    complex128 tensors, FP64 Gram matrices on the FMA units and the FP64
    tridiagonal eigensolver, no batching and no pipelining.  A complete d = 7
    trajectory of it is a long run, so the sample is one complete one-round
    trajectory, counted as 1 / rounds of a full one (later rounds cost more:
    this overstates its rate, i.e. understates the batched path's gain)."""
    circ1 = P.Circuit(a.distance, 1, layout="optimized")
    theta = WL.M3["thetas"][3]
    kw = dict(noise="srx", theta=theta, chi=a.chi, precision="fp64", seed=WL.M3["seed"],
              svd_mode="gram_tri")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.run_trajectories(circ1, 1, first_traj=3, **kw)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return {"value": 1.0 / (a.rounds * secs), "unit": "trajectories/s",
            "sample": "one complete d=%d one-round trajectory (theta=%.3f, chi=%d), FP64, one trajectory "
                      "per call, %.1f s, counted as 1/%d of a %d-round trajectory"
                      % (a.distance, theta, a.chi, secs, a.rounds, a.rounds)}


def grad_fwd(a, P, torch):
    """Cost of the gradient estimate against the forward p_L on the gradient
    workload's d = 5, chi = 64 setting (MIXED, one syndrome round per
    trajectory so the leg stays short): ttn_grad = forward pass plus the two
    forced replays at theta +- h, on the same shots."""
    g = WL.M5
    circ = P.Circuit(5, 1, layout="optimized")
    shots, th = 64, g["theta0"]
    kw = dict(noise="srx", theta=th, chi=64, precision="mixed", seed=g["seed"])
    P.logical_error_rate(circ, 8, **kw)  # warm-up (library load, first launches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.logical_error_rate(circ, shots, **kw)
    torch.cuda.synchronize()
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    P.grad(circ, shots, wrt="theta", h=g["dtheta"], **kw)
    torch.cuda.synchronize()
    tg = time.perf_counter() - t0
    return {"grad_s": tg, "fwd_s": tf, "ratio": tg / tf if tf > 0 else None,
            "sample": "d=5, 1 round, chi=64, MIXED, SRX theta=%.3f, %d shots; score-function gradient "
                      "(forward + forced replays at theta +- %.0e)" % (th, shots, g["dtheta"])}


def roofline(a, prof, cls, wall_s):
    """achieved: the class's ledger flops / its event-timed device time (per
    launch, as the launches ran); aggregate: the same flops / the timed wall
    time, i.e. the rate of all concurrent launches of the class together."""
    fl = prof["flops"][cls]
    ms = prof["class_ms"][cls]
    achieved = fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    bf16, src = peaks()
    if cls == "eig":
        bound, peak, psrc = "alu", FP64_PEAK_TFLOPS, "FP64 nominal (MEASURED_PEAKS has no FP64 entry)"
    elif cls == "gram":
        # 9 bf16 digit products of the real Gram X^T X (X = m x 2n), upper
        # triangle only: 36 m n^2 executed flops per 8 m n^2 algorithmic
        bound, peak = "tensor", bf16 * 8.0 / 36.0
        psrc = src + " x 8/36 (algorithmic complex Gram flops per executed bf16 digit-product flops)"
    else:  # form_u, absorb (FP32 FMA in MIXED runs by default) and the rest
        bound, peak, psrc = "alu", 152 * 128 * 2 * 2.070e9 / 1e12, "FP32 FMA: 152 SMs x 128 lanes x 2 x 2070 MHz"
    agg = fl / wall_s / 1e12 if wall_s > 0 else 0.0
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else 0.0, "traffic": None, "kernel_class": cls,
            "launches": prof["launches"][cls], "kernel_ms": ms,
            "per_launch_ms": ms / max(1, prof["launches"][cls]), "peak_source": psrc,
            "aggregate_tflops": agg, "aggregate_frac": agg / peak if peak else 0.0}


def note(msg):
    print("[bench] " + msg, file=sys.stderr, flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import paper_2511_05719_gb300 as P
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if a.resident % a.segments:
        raise SystemExit("--resident must be a multiple of --segments")
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream()
    circ = P.Circuit(a.distance, a.rounds, layout="optimized")
    seed = WL.M3["seed"]
    t_fill = time.perf_counter()
    pipe = P.Pipeline(circ, a.resident, a.segments, noise="srx", theta=0.0, chi=a.chi, precision=a.precision,
                      seed=seed, first_traj=rank << 40, theta_cycle=WL.M3["thetas"], stream=stream.cuda_stream)
    torch.cuda.synchronize()
    fill_s = time.perf_counter() - t_fill
    G = pipe.group_size
    note("pipeline filled in %.1f s (%d resident, %d per step)" % (fill_s, a.resident, G))
    K, W = a.steps, a.warmup
    fails = torch.zeros(K * G, dtype=torch.uint8, device=dev)
    logp = torch.zeros(K * G, dtype=torch.float64, device=dev)
    disc = torch.zeros(K * G, dtype=torch.float64, device=dev)
    trajs = []
    # warm-up steps, profiled per kernel class: the dominant class
    P.profile_begin("all")
    wout = dict(fail=torch.zeros(G, dtype=torch.uint8, device=dev),
                log_prob=torch.zeros(G, dtype=torch.float64, device=dev))
    for i in range(W):
        t1 = time.perf_counter()
        pipe.step(wout, stream=stream.cuda_stream)
        note("warm-up step %d: %.1f s" % (i, time.perf_counter() - t1))
    torch.cuda.synchronize()
    wprof = P.profile_end()
    cms = wprof["class_ms"]
    dom = max(cms, key=lambda c: cms[c]) if W > 0 else "eig"
    # timed steps: device outputs; only the dominant class's launches carry events
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    P.profile_begin(dom)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(K):
        sl = slice(k * G, (k + 1) * G)
        t1 = time.perf_counter()
        r = pipe.step(dict(fail=fails[sl], log_prob=logp[sl], discarded=disc[sl]), stream=stream.cuda_stream)
        trajs.append(r["traj"])
        seg_ms = pipe.segment_ms()
        note("timed step %d: %.1f s; segments (s): %s" % (k, time.perf_counter() - t1,
                                                       " ".join("%.1f" % (x / 1e3) for x in seg_ms)))
    e1.record(stream)
    torch.cuda.synchronize()
    prof = P.profile_end()
    seg_ms = [round(x / 1e3, 2) for x in pipe.segment_ms()]
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        ms = float(t.item())
    value = world * K * G / (ms / 1e3)
    # end to end: host output buffers through the same call
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, a.e2e_steps)):
        pipe.step()
    e2e_s = time.perf_counter() - t0
    pipe.close()
    ne = max(1, a.e2e_steps)
    e2e = {"value": world * ne * G / e2e_s, "unit": "trajectories/s",
           # theta, gamma and trajectory index of the restarting group in; fail
           # byte, log-probability, discarded weight of the completing group
           # and every resident trajectory's error word out
           "h2d_bytes_per_step": 24 * G,
           "d2h_bytes_per_step": 17 * G + 4 * a.resident}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    # p_L per theta over the timed trajectories
    f = fails.cpu().numpy()
    tr = np.concatenate(trajs)
    th = np.asarray(WL.M3["thetas"])[(tr % len(WL.M3["thetas"])).astype(np.int64)]
    pl = {}
    for x in WL.M3["thetas"]:
        m = np.isclose(th, x)
        n = int(m.sum())
        nf = int(f[m].sum()) if n else 0
        pl["%.3f" % x] = {"n": n, "fail": nf, "p_L": nf / n if n else None}
    line = {"metric": METRIC,
            "value": value, "unit": "trajectories/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
            "config": run_config(a),
            "clocks": ck, "e2e": e2e, "gpu_launches": int(prof["kernels"]),
            "roofline": roofline(a, prof, dom, ms / 1e3),
            "fill_s": fill_s, "segment_s_last_step": seg_ms,
            "device_ms_by_class_warmup": {k: round(v, 1) for k, v in cms.items()},
            "ledger_tflop_per_traj": {k: v / 1e12 / max(1, K * G) for k, v in prof["flops"].items()},
            "pL_by_theta": pl,
            "eig_phase_Gcycles": {k: round(v / 1e9, 2) for k, v in prof["eig_phase_cycles"].items()},
            "mean_log_prob": float(logp.cpu().numpy().mean()), "mean_discarded": float(disc.cpu().numpy().mean())}
    if not a.no_plain:
        note("plain FP64 single-instance leg")
        pl1 = plain_fp64_single(a, P, torch)
        pl1["batched_over_plain"] = value / pl1["value"] if pl1["value"] > 0 else None
        line["plain_fp64_single"] = pl1
    if not a.no_grad:
        note("grad / forward cost leg")
        line["grad_fwd"] = grad_fwd(a, P, torch)
    if not a.no_cpu_baseline and world == 1:
        note("CPU oracle baseline")
        line["cpu_baseline"] = cpu_baseline(a)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

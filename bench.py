"""Benchmark of the TTN trajectory simulator (one JSON line on rank 0).

A step is one batch of trajectories of the whole hot path -- circuit on the
tree tensor network, Born / Kraus sampling, decoding -- through the C ABI.
Default workload: d = 7 color code, 7 rounds, SRX with theta swept over 8
values in [0.01, 0.15] rad (trajectory i of a batch at theta_(i mod 8)),
chi = 128, complex64 tensors.  Inputs are synthetic and seeded (the paper's
workloads are themselves synthetic circuits).

value: trajectories/s with device-side outputs (CUDA events on the launch
stream, max over ranks).  e2e: the same metric through the same call with
host buffers (device -> host copies of records / fail bits / log-probs
inside the timed region).  Trajectories are sharded across ranks by index
(no collective on the data path: weak scaling).  Every launch works on the
full per-trajectory arena (hundreds of MB per trajectory, far above L2), so
no L2 flush is needed between steps.
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

import workloads as WL  # noqa: E402

FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max clock
METRIC = "d=7 trajectories/s (chi=128), batched vs plain at matched p_L; grad/fwd cost"
TENSOR_CLASSES = ("gram", "form_u", "absorb")   # on the tensor cores in FP32 Gram-path moves


def tensor_peak():
    """Effective 3xTF32 complex-FP32 peak: the measured bf16 dense peak x the
    nominal TF32/bf16 ratio (1.1 / 2.25 PFLOP/s), / 3 for the three TF32
    passes each FP32 product takes.  Returns (TFLOP/s, source)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        bf16, src = float(pk["bf16_tflops_sustained"]), "of measured (bf16 sustained)"
    except (OSError, KeyError, ValueError):
        bf16, src = 1700.0, "of fallback (bf16 sustained 1.7 PFLOP/s)"
    return bf16 * (1.1 / 2.25) / 3.0, src + " x 1.1/2.25 (TF32) / 3 (3xTF32 passes)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ttn", choices=["ttn", "reference"])
    ap.add_argument("--batch", type=int, default=0,
                    help="trajectories per step and rank (0: 64 for d >= 7, else 512)")
    ap.add_argument("--distance", type=int, default=7)
    ap.add_argument("--rounds", type=int, default=7)
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--roofline-class", default="auto")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_name(a):
    return "d%d_C%d_srx_theta_sweep8_chi%d_%s" % (a.distance, a.rounds, a.chi, a.precision)


def default_batch(a):
    # d >= 7: 64 trajectories per step.  The eigensolver runs one CTA per
    # trajectory and is latency-bound, so a step's time grows slowly with the
    # batch until every SM holds one (d=7, C=1: 12.0 s at 16, 24.1 s at 152,
    # 47.3 s at 304 trajectories on 152 SMs).  64 keeps most of that gain
    # while five default steps (3 warm-up, 1 timed, 1 end-to-end) of the
    # 7-round circuit stay near a quarter of an hour; --batch 152 gives the
    # highest throughput.
    return a.batch if a.batch > 0 else (64 if a.distance >= 7 else 512)


def run_config(a, B):
    """The workload both arms report (the same keys and values)."""
    return {"workload": workload_name(a), "trajectories_per_step": B, "rounds": a.rounds,
            "distance": a.distance, "chi": a.chi,
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


def cpu_baseline(a, seconds):
    """The plain CPU TTN oracle (numpy, float64) on a bounded sample of the
    same workload: one trajectory's ops in program order for about `seconds`,
    extrapolated by op count to trajectories/s."""
    from oracle.circuit import build_circuit
    from oracle import ttn as TT
    from oracle.channels import SRX
    import paper_2511_05719_gb300 as P  # only for the circuit's leaf layout
    circ = build_circuit(a.distance, a.rounds)
    layout = P.Circuit(a.distance, a.rounds, layout="optimized").layout()
    thetas = WL.M3["thetas"]
    total = len(circ.ops)
    done = 0
    # one trajectory in program order, stopped after about `seconds`
    t1 = time.time()
    r = TT.run_trajectory(circ, SRX, thetas[3], 0.0, WL.M3["seed"], 0, chi=a.chi,
                          leaf_of_qubit=list(layout), deadline=t1 + seconds)
    elapsed = time.time() - t1
    done = r["ops_done"]
    traj_s = (done / total) / elapsed if elapsed > 0 else 0.0
    cores = os.cpu_count()
    return {"value": traj_s, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
            "sample": "plain numpy TTN (float64, threaded BLAS) on the first %d of %d ops of one "
                      "trajectory (theta=%.3f), %.1f s, extrapolated by op count"
                      % (done, total, thetas[3], elapsed)}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    seconds = max(5.0, min(60.0, a.cpu_seconds))
    vals = []
    cb = None
    for _ in range(max(1, a.steps)):
        cb = cpu_baseline(a, seconds / max(1, a.steps))
        vals.append(cb["value"])
    v = float(np.mean(vals))
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v,
            "unit": "trajectories/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": run_config(a, default_batch(a)),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


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
    B = default_batch(a)
    circ = P.Circuit(a.distance, a.rounds, layout="optimized")
    thetas = WL.theta_sweep_per_traj(B, WL.M3["thetas"])
    stream = torch.cuda.Stream()
    dev = torch.device("cuda", local)
    out = dict(records=torch.empty((B, circ.n_record_bits), dtype=torch.uint8, device=dev),
               fail=torch.empty(B, dtype=torch.uint8, device=dev),
               log_prob=torch.empty(B, dtype=torch.float64, device=dev),
               discarded=torch.empty(B, dtype=torch.float64, device=dev))
    seed = WL.M3["seed"]
    step_id = [0]

    def step(device_out=True):
        first = (rank * 1_000_000 + step_id[0]) * B
        step_id[0] += 1
        kw = dict(noise="srx", theta=0.0, chi=a.chi, precision=a.precision, seed=seed,
                  first_traj=first, theta_per_traj=thetas)
        try:
            if device_out:
                P.run_trajectories(circ, B, out=out, stream=stream.cuda_stream, **kw)
                return None
            return P.run_trajectories(circ, B, **kw)
        except P.TTNError as e:
            if e.status == 6:      # decoder bound exceeded on some shots: counted, not fatal
                return None
            raise

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    P.profile_begin("all")   # device time of every launch, per kernel class (CUDA events)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = P.profile_end()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        ms = float(t.item())
    traj = world * a.steps * B
    value = traj / (ms / 1e3)
    lost = int((out["fail"] == 3).sum().item())   # of the last timed step (fail byte 3)
    # end to end: host buffers through the same call (one step)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step(device_out=False)
    e2e_s = time.perf_counter() - t0
    # bytes the call copies per step: theta, gamma and trajectory index in
    # (8 B each per trajectory); records, fail byte, log-probability,
    # discarded weight, near-tie count, error word and two error-step words out
    e2e = {"value": world * B / e2e_s, "unit": "trajectories/s",
           "h2d_bytes_per_step": 24 * B,
           "d2h_bytes_per_step": B * (circ.n_record_bits + 1 + 8 + 8 + 4 + 4 + 8)}
    # roofline of the dominant kernel class (most device time in the timed region)
    cms = prof["class_ms"]
    rclass = a.roofline_class if a.roofline_class != "auto" else max(cms, key=lambda c: cms[c])
    fl = prof["flops"][rclass]
    by = prof["bytes"][rclass]
    tms = cms[rclass]
    achieved = fl / (tms / 1e3) / 1e12 if tms > 0 else 0.0
    roof = {"bound": "alu", "achieved": achieved, "peak": FP32_ALU_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP32_ALU_PEAK_TFLOPS if achieved else 0.0,
            "traffic": None, "kernel_class": rclass, "launches": prof["launches"][rclass],
            "kernel_ms": tms, "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x 2070 MHz"}
    if a.precision == "fp32" and rclass in TENSOR_CLASSES:
        pk, src = tensor_peak()
        roof.update(bound="tensor", peak=pk, frac=achieved / pk if achieved else 0.0, peak_source=src)
    if a.precision == "fp64":
        roof["peak"] = 1.25
        roof["frac"] = achieved / 1.25 if achieved else 0.0
        roof["peak_source"] = "FP64 nominal 1.25 TFLOP/s"
    if rank != 0:
        return
    line = {"metric": METRIC,
            "value": value, "unit": "trajectories/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64" if a.precision == "fp32" else "c128",
            "data": "synthetic",
            "config": dict(run_config(a, B), lost_trajectories_last_step=lost),
            "clocks": ck, "e2e": e2e, "gpu_launches": int(sum(prof["launches"].values())),
            "roofline": roof,
            "ledger_tflop": {k: v / 1e12 for k, v in prof["flops"].items()},
            "device_ms_by_class": {k: round(v, 1) for k, v in cms.items()}}
    if not a.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(a, a.cpu_seconds)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

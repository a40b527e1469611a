"""Resumable p_L estimation with a JSON checkpoint and a JSONL run log.

Every trajectory is fixed by (seed, trajectory index) (Sec. III.C: the
samples are independent), so a Monte Carlo estimate can stop after any batch
and continue later without changing its result: the state to keep is the
next trajectory index and the counts so far.  After each batch the state
is written atomically (temporary file, then rename); a later call with the
same circuit and run parameters continues from it, and one with different
parameters is refused rather than mixed in.  The optional log gets one JSON
line per batch: throughput, running p_L and its binomial error, discarded
singular weight and near-tie counts of the batch."""
import json
import math
import os
import time

import numpy as np

STATE_VERSION = 1
_PARAM_KEYS = ("noise", "theta", "gamma", "chi", "precision", "seed", "first_traj", "svd_eps",
               "svd_mode", "gemm_mode")


def _params(circuit, shots, run_kw):
    p = dict(distance=int(circuit.distance), rounds=int(circuit.rounds), shots=int(shots))
    defaults = dict(noise="srx", theta=0.0, gamma=0.0, chi=16, precision="fp64", seed=0,
                    first_traj=0, svd_eps=0.0, svd_mode="auto", gemm_mode="auto")
    for k in _PARAM_KEYS:
        v = run_kw.get(k, defaults[k])
        p[k] = v if isinstance(v, str) else (float(v) if isinstance(v, float) else int(v))
    return p


def _write_atomic(path, obj):
    tmp = "%s.tmp.%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(obj, f, sort_keys=True)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def _result(st):
    nf, nv = st["n_fail"], st["n_valid"]
    p = nf / nv if nv else float("nan")
    sigma = math.sqrt(p * (1 - p) / nv) if nv else float("nan")
    return p, sigma, nf, nv


def logical_error_rate_resumable(circuit, shots, state_path, batch=1024, log_path=None, run=None,
                                 **run_kw):
    """p_L over `shots` trajectories in batches of `batch`, checkpointed to
    `state_path` after each batch.  Returns (p_L, sigma, n_fail, n_valid);
    shots with a fail byte above 1 (decoder bound exceeded, lost state) are
    not valid.  `run` defaults to run_trajectories (keyword arguments as
    there, except per-trajectory strengths and outputs)."""
    if shots < 1 or batch < 1:
        raise ValueError("shots and batch must be >= 1")
    for k in run_kw:
        if k not in _PARAM_KEYS:
            raise ValueError("unsupported run argument %r" % k)
    if run is None:
        from ._lib import run_trajectories as run
    params = _params(circuit, shots, run_kw)
    st = dict(version=STATE_VERSION, params=params, next_traj=0, n_fail=0, n_valid=0, n_lost=0,
              n_overflow=0, done=False)
    if os.path.exists(state_path):
        with open(state_path) as f:
            old = json.load(f)
        if old.get("version") != STATE_VERSION or old.get("params") != params:
            raise ValueError("checkpoint %s belongs to another run: %r" % (state_path, old.get("params")))
        st = old
    base = params["first_traj"]
    while st["next_traj"] < shots:
        n = min(batch, shots - st["next_traj"])
        kw = dict(run_kw)
        kw["first_traj"] = base + st["next_traj"]
        t0 = time.perf_counter()
        out = run(circuit, n, **kw)
        dt = time.perf_counter() - t0
        fail = np.asarray(out["fail"])
        nf, nv = int((fail == 1).sum()), int((fail <= 1).sum())
        st["n_fail"] += nf
        st["n_valid"] += nv
        st["n_overflow"] += int((fail == 2).sum())
        st["n_lost"] += int((fail == 3).sum())
        st["next_traj"] += n
        st["done"] = st["next_traj"] >= shots
        _write_atomic(state_path, st)
        if log_path:
            p, sigma, _, _ = _result(st)
            disc = np.asarray(out.get("discarded", np.zeros(0)), dtype=np.float64)
            ties = np.asarray(out.get("near_ties", np.zeros(0)))
            line = dict(first_traj=kw["first_traj"], n=n, seconds=dt,
                        trajectories_per_s=n / dt if dt > 0 else None, n_fail=nf, n_valid=nv,
                        p_L=p, sigma=sigma, next_traj=st["next_traj"],
                        discarded_mean=float(disc.mean()) if disc.size else None,
                        discarded_max=float(disc.max()) if disc.size else None,
                        near_ties=int(ties.sum()) if ties.size else None)
            with open(log_path, "a") as f:
                f.write(json.dumps(line) + "\n")
    return _result(st)

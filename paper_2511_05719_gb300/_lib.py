"""ctypes marshalling for libttn.so (see include/ttn.h for the contract)."""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

NOISE = {"none": 0, "srx": 1, "ad": 2, "srx_pta": 3, "ad_pta": 4, "srx_ad": 5, "depol": 6}
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2}
LAYOUT = {"default": 0, "optimized": 1, "explicit": 2, "search": 3}

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_dblp = ctypes.POINTER(ctypes.c_double)
c_u8p = ctypes.POINTER(ctypes.c_uint8)
c_u64p = ctypes.POINTER(ctypes.c_uint64)
c_i64p = ctypes.POINTER(ctypes.c_int64)


class CircuitParams(ctypes.Structure):
    _fields_ = [("distance", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("leaf_of_qubit", c_i32p)]


class RunParams(ctypes.Structure):
    _fields_ = [("noise", ctypes.c_int32), ("theta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("chi", ctypes.c_int32), ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("first_traj", ctypes.c_uint64), ("svd_eps", ctypes.c_double),
                ("theta_per_traj", c_dblp), ("gamma_per_traj", c_dblp),
                ("svd_mode", ctypes.c_int32), ("gemm_mode", ctypes.c_int32)]


class TTNError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("ttn status %d: %s" % (status, message))
        self.status = status


EXPORTS = ["ttn_build_circuit", "ttn_free_circuit", "ttn_circuit_info", "ttn_circuit_ops",
           "ttn_circuit_layout", "ttn_run_trajectories", "ttn_logical_error_rate", "ttn_decode",
           "ttn_debug_state", "ttn_philox_uniforms", "ttn_profile_begin", "ttn_profile_end",
           "ttn_grad", "ttn_decode_noalloc", "ttn_profile_class_ms", "ttn_profile_eig_phases",
           "ttn_profile_move_hist", "ttn_gram_exact", "ttn_eig_gram", "ttn_pipeline_create", "ttn_pipeline_step",
           "ttn_pipeline_group_size", "ttn_pipeline_free", "ttn_profile_kernels", "ttn_pipeline_segment_ms",
           "ttn_run_mixed", "ttn_newton_crossing", "ttn_crossing", "ttn_threshold_fit", "ttn_grad_sums",
           "ttn_slot_check", "ttn_layout_noise_free_chi",
           "ttn_status_string",
           "ttn_last_error"]

# f(x) evaluator of ttn_newton_crossing: (ctx, x, iter, *f, *f_sigma, *df, *df_sigma) -> status
CROSSING_EVAL = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32,
                                 c_dblp, c_dblp, c_dblp, c_dblp)


def library_path():
    return os.path.join(_HERE, "libttn.so")


def load_library():
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise TTNError(-1, "libttn.so is not built (run paper_2511_05719_gb300.build.build())")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.ttn_build_circuit.argtypes = [ctypes.POINTER(CircuitParams), ctypes.POINTER(vp)]
    lib.ttn_free_circuit.argtypes = [vp]
    lib.ttn_free_circuit.restype = None
    lib.ttn_circuit_info.argtypes = [vp] + [c_i32p] * 7
    lib.ttn_circuit_ops.argtypes = [vp, c_i32p]
    lib.ttn_circuit_layout.argtypes = [vp, c_i32p]
    lib.ttn_run_trajectories.argtypes = [vp, ctypes.POINTER(RunParams), ctypes.c_uint64, vp, vp, vp,
                                         vp, vp, vp]
    lib.ttn_run_mixed.argtypes = [ctypes.c_int32, vp, vp, vp, vp, vp, vp]
    lib.ttn_newton_crossing.argtypes = [CROSSING_EVAL, vp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int32, ctypes.c_double, c_dblp,
                                        c_dblp, c_i32p, c_i32p, c_dblp]
    lib.ttn_crossing.argtypes = [vp, vp, ctypes.POINTER(RunParams), ctypes.c_uint64, ctypes.c_int32,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int32, ctypes.c_double, c_dblp, c_dblp, c_i32p, c_i32p,
                                 c_dblp]
    lib.ttn_threshold_fit.argtypes = [ctypes.c_int32, c_i32p, c_dblp, c_dblp, c_dblp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int32, c_dblp, c_dblp, c_dblp, c_i32p]
    lib.ttn_grad_sums.argtypes = [vp, ctypes.POINTER(RunParams), ctypes.c_uint64, ctypes.c_int32,
                                  ctypes.c_double, c_u64p, c_u64p, c_dblp, c_dblp]
    lib.ttn_layout_noise_free_chi.argtypes = [vp, c_i32p, c_i64p]
    lib.ttn_slot_check.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, c_dblp, c_i32p, c_i32p, c_i64p]
    lib.ttn_logical_error_rate.argtypes = [vp, ctypes.POINTER(RunParams), ctypes.c_uint64, c_dblp,
                                           c_dblp, c_u64p]
    lib.ttn_decode.argtypes = [vp, ctypes.c_uint64, vp, vp, vp, vp, vp]
    lib.ttn_decode_noalloc.argtypes = [vp, ctypes.c_uint64, vp, vp, vp, vp, vp]
    lib.ttn_gram_exact.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, vp]
    lib.ttn_eig_gram.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_double, vp, vp, vp, vp]
    lib.ttn_pipeline_create.argtypes = [vp, ctypes.POINTER(RunParams), ctypes.c_int32, ctypes.c_int32, vp,
                                        ctypes.c_int32, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
    lib.ttn_pipeline_step.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, vp]
    lib.ttn_pipeline_group_size.argtypes = [vp]
    lib.ttn_pipeline_group_size.restype = ctypes.c_int32
    lib.ttn_pipeline_free.argtypes = [vp]
    lib.ttn_pipeline_segment_ms.argtypes = [vp, c_dblp]
    lib.ttn_pipeline_segment_ms.restype = ctypes.c_int32
    lib.ttn_profile_kernels.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.ttn_pipeline_free.restype = None
    lib.ttn_debug_state.argtypes = [vp, ctypes.POINTER(RunParams), ctypes.c_uint64, ctypes.c_int32,
                                    c_dblp]
    lib.ttn_philox_uniforms.argtypes = [ctypes.c_uint64, c_u64p, ctypes.c_uint64, c_i32p,
                                        ctypes.c_int32, c_dblp]
    lib.ttn_grad.argtypes = [vp, ctypes.POINTER(RunParams), ctypes.c_uint64, ctypes.c_int32,
                             ctypes.c_double, c_dblp, c_dblp, c_dblp, c_dblp]
    lib.ttn_profile_begin.argtypes = [ctypes.c_int32]
    lib.ttn_profile_class_ms.argtypes = [c_dblp]
    lib.ttn_profile_eig_phases.argtypes = [c_dblp]
    lib.ttn_profile_end.argtypes = [c_dblp, c_u64p, c_dblp, c_dblp, c_u64p]
    lib.ttn_status_string.restype = ctypes.c_char_p
    lib.ttn_status_string.argtypes = [ctypes.c_int]
    lib.ttn_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        f = getattr(lib, name)
        if name not in ("ttn_free_circuit", "ttn_status_string", "ttn_last_error"):
            f.restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(status):
    if status != 0:
        lib = load_library()
        raise TTNError(status, lib.ttn_last_error().decode())


def _ptr(a, ctype=None):
    """Data pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


class Circuit:
    """Color-code syndrome-extraction circuit (d, C) with its TTN layout."""

    def __init__(self, distance, rounds, layout="optimized", leaf_of_qubit=None):
        lib = load_library()
        p = CircuitParams()
        p.distance = distance
        p.rounds = rounds
        self._leaves = None
        if leaf_of_qubit is not None:
            layout = "explicit"
            self._leaves = np.ascontiguousarray(leaf_of_qubit, dtype=np.int32)
            p.leaf_of_qubit = self._leaves.ctypes.data_as(c_i32p)
        p.layout = LAYOUT[layout]
        h = ctypes.c_void_p()
        _check(lib.ttn_build_circuit(ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        vals = [ctypes.c_int32() for _ in range(7)]
        _check(lib.ttn_circuit_info(h, *[ctypes.byref(v) for v in vals]))
        (self.n_qubits, self.n_data, self.n_layers, self.n_record_bits, self.n_events,
         self.n_ops, self.n_leaves) = [v.value for v in vals]
        self.distance, self.rounds = distance, rounds

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _LIB is not None:
            _LIB.ttn_free_circuit(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def ops(self):
        out = np.zeros((self.n_ops, 6), dtype=np.int32)
        _check(load_library().ttn_circuit_ops(self._h, out.ctypes.data_as(c_i32p)))
        return out

    def noise_free_chi(self, leaf_of_qubit=None):
        """Bond dimension the noise-free circuit needs on a layout (this
        circuit's own when leaf_of_qubit is None); host only."""
        out = ctypes.c_int64()
        lay = None if leaf_of_qubit is None else np.ascontiguousarray(leaf_of_qubit, dtype=np.int32)
        _check(load_library().ttn_layout_noise_free_chi(
            self._h, None if lay is None else lay.ctypes.data_as(c_i32p), ctypes.byref(out)))
        return out.value

    def layout(self):
        out = np.zeros(self.n_qubits, dtype=np.int32)
        _check(load_library().ttn_circuit_layout(self._h, out.ctypes.data_as(c_i32p)))
        return out


SVD_MODE = {"auto": 0, "jacobi": 1, "gram": 2, "gram_tri": 3}
GEMM_MODE = {"auto": 0, "fma": 1, "tensor": 2, "exact": 3}


def _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                theta_per_traj=None, gamma_per_traj=None, svd_mode="auto", gemm_mode="auto"):
    p = RunParams()
    p.noise = NOISE[noise] if isinstance(noise, str) else int(noise)
    p.theta = float(theta)
    p.gamma = float(gamma)
    p.chi = int(chi)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.seed = int(seed)
    p.first_traj = int(first_traj)
    p.svd_eps = float(svd_eps)
    p.svd_mode = SVD_MODE[svd_mode] if isinstance(svd_mode, str) else int(svd_mode)
    p.gemm_mode = GEMM_MODE[gemm_mode] if isinstance(gemm_mode, str) else int(gemm_mode)
    keep = []
    if theta_per_traj is not None:
        a = np.ascontiguousarray(theta_per_traj, dtype=np.float64)
        keep.append(a)
        p.theta_per_traj = a.ctypes.data_as(c_dblp)
    if gamma_per_traj is not None:
        a = np.ascontiguousarray(gamma_per_traj, dtype=np.float64)
        keep.append(a)
        p.gamma_per_traj = a.ctypes.data_as(c_dblp)
    return p, keep


def run_trajectories(circuit, n_traj, noise="srx", theta=0.0, gamma=0.0, chi=16,
                     precision="fp64", seed=0, first_traj=0, svd_eps=0.0,
                     theta_per_traj=None, gamma_per_traj=None, out=None, stream=None,
                     svd_mode="auto", gemm_mode="auto"):
    """Runs n_traj trajectories.  With `out=None` returns host numpy arrays
    {records, fail, log_prob, discarded, near_ties}.  With `out` a dict of
    torch CUDA tensors (any subset of those keys) and `stream` a CUDA stream
    handle (int), writes them on the device."""
    lib = load_library()
    p, keep = _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                          theta_per_traj, gamma_per_traj, svd_mode, gemm_mode)
    if out is None:
        out = dict(records=np.zeros((n_traj, circuit.n_record_bits), dtype=np.uint8),
                   fail=np.zeros(n_traj, dtype=np.uint8),
                   log_prob=np.zeros(n_traj), discarded=np.zeros(n_traj),
                   near_ties=np.zeros(n_traj, dtype=np.int32))
        st = None
    else:
        st = ctypes.c_void_p(int(stream)) if stream is not None else None
        if st is None:
            raise ValueError("device outputs need a CUDA stream handle")
    _check(lib.ttn_run_trajectories(circuit.handle, ctypes.byref(p), n_traj,
                                    _ptr(out.get("records")), _ptr(out.get("fail")),
                                    _ptr(out.get("log_prob")), _ptr(out.get("discarded")),
                                    _ptr(out.get("near_ties")), st))
    del keep
    return out


class Pipeline:
    """Pipelined resident batch (ttn_pipeline_*): n_resident trajectories on
    the device in n_segments groups; every step() runs one program segment of
    every group and completes group_size trajectories.  theta_cycle: optional
    SRX angles, trajectory t at theta_cycle[t % len]."""

    def __init__(self, circuit, n_resident, n_segments, noise="srx", theta=0.0, gamma=0.0, chi=16,
                 precision="mixed", seed=0, first_traj=0, theta_cycle=None, svd_eps=0.0, gemm_mode="auto",
                 max_device_bytes=0, stream=None):
        lib = load_library()
        p, keep = _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                              gemm_mode=gemm_mode)
        cyc = None if theta_cycle is None else np.ascontiguousarray(theta_cycle, dtype=np.float64)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(int(stream)) if stream else None
        self.circuit = circuit
        self._lib = lib
        _check(lib.ttn_pipeline_create(circuit.handle, ctypes.byref(p), int(n_resident), int(n_segments),
                                       _ptr(cyc), 0 if cyc is None else cyc.size, int(max_device_bytes),
                                       st, ctypes.byref(h)))
        del keep
        self.handle = h
        self.group_size = int(lib.ttn_pipeline_group_size(h))

    def step(self, out=None, stream=None):
        """One step.  out=None: returns host {fail, log_prob, discarded,
        traj}; else `out` holds torch CUDA tensors (fail uint8 [G], log_prob
        and discarded float64 [G]) written on the device, and `stream` is a
        CUDA stream handle (int).  The trajectory indices are returned in
        host memory either way."""
        G = self.group_size
        traj = np.zeros(G, dtype=np.uint64)
        nd = ctypes.c_int32()
        st = ctypes.c_void_p(int(stream)) if stream else None
        if out is None:
            res = dict(fail=np.zeros(G, dtype=np.uint8), log_prob=np.zeros(G), discarded=np.zeros(G))
            on_dev = 0
        else:
            res = out
            on_dev = 1
        _check(self._lib.ttn_pipeline_step(self.handle, _ptr(res.get("fail")), _ptr(res.get("log_prob")),
                                           _ptr(res.get("discarded")), _ptr(traj), ctypes.byref(nd),
                                           on_dev, st))
        res = dict(res)
        res["traj"] = traj[:nd.value]
        return res

    def segment_ms(self):
        """Device milliseconds of each segment in the last step."""
        buf = np.zeros(1024)
        n = self._lib.ttn_pipeline_segment_ms(self.handle, buf.ctypes.data_as(c_dblp))
        return buf[:n].copy()

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ttn_pipeline_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_mixed(items, out=None, stream=None):
    """Mixed batch: `items` is a list of dicts, each with `circuit` and
    `n_traj` plus any keyword of run_trajectories (noise, theta, gamma, chi,
    precision, seed, first_traj, svd_eps, theta_per_traj, gamma_per_traj,
    svd_mode, gemm_mode).  All items are in flight at once (ttn_run_mixed).
    With `out=None` returns a list of host dicts {fail, log_prob}; with `out`
    a list of dicts of torch CUDA tensors (`fail` uint8, optional `log_prob`
    float64) and `stream` a CUDA stream handle (int), writes them on the
    device."""
    lib = load_library()
    n = len(items)
    circs = (ctypes.c_void_p * max(1, n))()
    params = (RunParams * max(1, n))()
    counts = (ctypes.c_uint64 * max(1, n))()
    fails = (ctypes.c_void_p * max(1, n))()
    lps = (ctypes.c_void_p * max(1, n))()
    keep = []
    opts = ("noise", "theta", "gamma", "chi", "precision", "seed", "first_traj", "svd_eps",
            "theta_per_traj", "gamma_per_traj", "svd_mode", "gemm_mode")
    defaults = dict(noise="srx", theta=0.0, gamma=0.0, chi=16, precision="fp64", seed=0,
                    first_traj=0, svd_eps=0.0, theta_per_traj=None, gamma_per_traj=None,
                    svd_mode="auto", gemm_mode="auto")
    if out is None:
        out = [dict(fail=np.zeros(int(it["n_traj"]), dtype=np.uint8),
                    log_prob=np.zeros(int(it["n_traj"]))) for it in items]
        st = None
    else:
        if stream is None:
            raise ValueError("device outputs need a CUDA stream handle")
        st = ctypes.c_void_p(int(stream))
    for i, it in enumerate(items):
        unknown = set(it) - set(opts) - {"circuit", "n_traj"}
        if unknown:
            raise ValueError("unknown item keys: %s" % sorted(unknown))
        kw = dict(defaults)
        kw.update({k: it[k] for k in opts if k in it})
        p, kp = _run_params(**kw)
        keep.extend(kp)
        params[i] = p
        circs[i] = it["circuit"].handle.value
        counts[i] = int(it["n_traj"])
        fp, lp = _ptr(out[i].get("fail")), _ptr(out[i].get("log_prob"))
        fails[i] = fp.value if fp is not None else None
        lps[i] = lp.value if lp is not None else None
    _check(lib.ttn_run_mixed(n, circs, params, counts, fails, lps, st))
    del keep
    return out


def _crossing_out(max_iter):
    return (ctypes.c_double(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32(),
            np.zeros((max_iter, 5)))


def _crossing_result(xs, sx, it, cv, tr):
    n = it.value
    return dict(x=xs.value, sigma=sx.value, iters=n, converged=bool(cv.value), trace=tr[:n].copy())


def newton_crossing(f, x0, x_lo, x_hi, max_iter=20, x_tol=1e-4):
    """ttn_newton_crossing with a Python evaluator f(x, iter) -> (f, f_sigma,
    df, df_sigma).  Returns {x, sigma, iters, converged, trace}."""
    lib = load_library()
    errors = []

    def cb(ctx, x, it, pf, psf, pdf, psdf):
        try:
            v = f(x, it)
            pf[0], psf[0], pdf[0], psdf[0] = [float(t) for t in v]
            return 0
        except Exception as e:  # reported after the call
            errors.append(e)
            return 1

    cfn = CROSSING_EVAL(cb)
    xs, sx, it, cv, tr = _crossing_out(max_iter)
    st = lib.ttn_newton_crossing(cfn, None, x0, x_lo, x_hi, max_iter, x_tol, ctypes.byref(xs),
                                 ctypes.byref(sx), ctypes.byref(it), ctypes.byref(cv),
                                 tr.ctypes.data_as(c_dblp))
    if errors:
        raise errors[0]
    _check(st)
    return _crossing_result(xs, sx, it, cv, tr)


def crossing(circuit_a, circuit_b, shots, x0, x_lo, x_hi, wrt="theta", noise="srx", theta=0.0,
             gamma=0.0, chi=16, precision="fp64", seed=0, first_traj=0, svd_eps=0.0, h=0.0,
             max_iter=10, x_tol=1e-4, svd_mode="auto", gemm_mode="auto"):
    """ttn_crossing: the crossing of the p_L(x) curves of two circuits,
    x = theta or gamma.  Returns {x, sigma, iters, converged, trace}."""
    lib = load_library()
    p, keep = _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                          svd_mode=svd_mode, gemm_mode=gemm_mode)
    w = {"theta": 0, "gamma": 1}[wrt] if isinstance(wrt, str) else int(wrt)
    xs, sx, it, cv, tr = _crossing_out(max_iter)
    _check(lib.ttn_crossing(circuit_a.handle, circuit_b.handle, ctypes.byref(p), shots, w, h, x0, x_lo,
                            x_hi, max_iter, x_tol, ctypes.byref(xs), ctypes.byref(sx), ctypes.byref(it),
                            ctypes.byref(cv), tr.ctypes.data_as(c_dblp)))
    del keep
    return _crossing_result(xs, sx, it, cv, tr)


def threshold_fit(d, p_err, p_fail, sigma, tau0, nu0=1.0, max_iter=500):
    """Eq. 4 fit (ttn_threshold_fit): {A, B, C, tau, nu, cov (5x5), chi2, iters}."""
    lib = load_library()
    d = np.ascontiguousarray(d, dtype=np.int32)
    x = [np.ascontiguousarray(a, dtype=np.float64) for a in (p_err, p_fail, sigma)]
    n = d.size
    if any(a.size != n for a in x):
        raise ValueError("d, p_err, p_fail and sigma must have the same length")
    prm, cov = np.zeros(5), np.zeros((5, 5))
    c2, it = ctypes.c_double(), ctypes.c_int32()
    _check(lib.ttn_threshold_fit(n, d.ctypes.data_as(c_i32p), *[a.ctypes.data_as(c_dblp) for a in x],
                                 tau0, nu0, max_iter, prm.ctypes.data_as(c_dblp),
                                 cov.ctypes.data_as(c_dblp), ctypes.byref(c2), ctypes.byref(it)))
    return dict(A=prm[0], B=prm[1], C=prm[2], tau=prm[3], nu=prm[4], cov=cov, chi2=c2.value,
                iters=it.value)


def logical_error_rate(circuit, shots, noise="srx", theta=0.0, gamma=0.0, chi=16,
                       precision="fp64", seed=0, first_traj=0, svd_eps=0.0, svd_mode="auto",
                       gemm_mode="auto"):
    lib = load_library()
    p, keep = _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                          svd_mode=svd_mode, gemm_mode=gemm_mode)
    pl, sg, nf = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    _check(lib.ttn_logical_error_rate(circuit.handle, ctypes.byref(p), shots, ctypes.byref(pl),
                                      ctypes.byref(sg), ctypes.byref(nf)))
    return pl.value, sg.value, nf.value


def gram_exact(M, stream=None):
    """ttn_gram_exact: the exact Gram matrix M^H M (complex128, n x n) of a
    torch CUDA complex64 matrix M (m x n), on the tensor cores."""
    import torch
    if not isinstance(M, torch.Tensor) or not M.is_cuda or M.dtype != torch.complex64 or M.dim() != 2:
        raise ValueError("gram_exact: M must be a 2-d complex64 CUDA tensor")
    M = M.contiguous()
    m, n = M.shape
    G = torch.empty((n, n), dtype=torch.complex128, device=M.device)
    st = ctypes.c_void_p(int(stream)) if stream else None
    _check(load_library().ttn_gram_exact(_ptr(M), int(m), int(n), _ptr(G), st))
    return G


EIG_ROUTES = {"jacobi": 0, "tridiagonal": 1, "tridiagonal_split": 2, "mixed": 3}


def eig_gram(G, kcap=None, route="tridiagonal", eps_keep=1e-7, stream=None):
    """ttn_eig_gram: kept right singular vectors and singular values of a
    batch of Hermitian PSD Gram matrices G (CUDA complex128, [batch, n, n] or
    [n, n]).  Returns (V [batch, n, kcap] complex128, s [batch, n] float64
    descending, k [batch] int32)."""
    import torch
    if not isinstance(G, torch.Tensor) or not G.is_cuda or G.dtype != torch.complex128 or G.dim() not in (2, 3):
        raise ValueError("eig_gram: G must be a complex128 CUDA tensor [batch, n, n] or [n, n]")
    if route not in EIG_ROUTES:
        raise ValueError("eig_gram: route must be one of %s" % sorted(EIG_ROUTES))
    squeeze = G.dim() == 2
    G = (G[None] if squeeze else G).contiguous()
    B, n, n2 = G.shape
    if n != n2:
        raise ValueError("eig_gram: G must be square")
    kcap = n if kcap is None else int(kcap)
    V = torch.empty((B, n, kcap), dtype=torch.complex128, device=G.device)
    s = torch.empty((B, n), dtype=torch.float64, device=G.device)
    k = torch.empty((B,), dtype=torch.int32, device=G.device)
    st = ctypes.c_void_p(int(stream)) if stream else None
    _check(load_library().ttn_eig_gram(_ptr(G), int(B), int(n), kcap, EIG_ROUTES[route], float(eps_keep),
                                       _ptr(V), _ptr(s), _ptr(k), st))
    return (V[0], s[0], k[0]) if squeeze else (V, s, k)


def decode(circuit, records):
    """Decodes host records [n][n_record_bits] -> (fail u8, colour i32, score i64)."""
    lib = load_library()
    rec = np.ascontiguousarray(records, dtype=np.uint8)
    n = rec.shape[0]
    fail = np.zeros(n, dtype=np.uint8)
    color = np.zeros(n, dtype=np.int32)
    score = np.zeros(n, dtype=np.int64)
    _check(lib.ttn_decode(circuit.handle, n, _ptr(rec), _ptr(fail), _ptr(color), _ptr(score), None))
    return fail, color, score


def debug_state(circuit, traj, layer, noise="srx", theta=0.0, gamma=0.0, chi=16,
                precision="fp64", seed=0, svd_eps=0.0, svd_mode="auto", gemm_mode="auto"):
    lib = load_library()
    p, keep = _run_params(noise, theta, gamma, chi, precision, seed, 0, svd_eps,
                          svd_mode=svd_mode, gemm_mode=gemm_mode)
    amps = np.zeros(2 * (1 << circuit.n_qubits))
    _check(lib.ttn_debug_state(circuit.handle, ctypes.byref(p), traj, layer,
                               amps.ctypes.data_as(c_dblp)))
    return amps[0::2] + 1j * amps[1::2]


def philox_uniforms(seed, trajs, events):
    lib = load_library()
    t = np.ascontiguousarray(trajs, dtype=np.uint64)
    e = np.ascontiguousarray(events, dtype=np.int32)
    out = np.zeros((t.size, e.size))
    _check(lib.ttn_philox_uniforms(seed, t.ctypes.data_as(c_u64p), t.size,
                                   e.ctypes.data_as(c_i32p), e.size, out.ctypes.data_as(c_dblp)))
    return out


KERNEL_CLASSES = ["svd_jacobi", "gram", "eig", "form_u", "absorb", "copy", "other", "local"]
EIG_PHASES = ["tridiagonalise", "split", "bisection", "eigenvectors", "rayleigh_ritz", "back_transform"]


def profile_begin(timed_class=-1):
    """Starts the profiling ledger; launches of `timed_class` are timed
    ("all" times every class, at some launch overhead)."""
    if isinstance(timed_class, str):
        timed_class = len(KERNEL_CLASSES) if timed_class == "all" else KERNEL_CLASSES.index(timed_class)
    _check(load_library().ttn_profile_begin(int(timed_class)))


def profile_end():
    nc = len(KERNEL_CLASSES)
    ms, nl = ctypes.c_double(), ctypes.c_uint64()
    fl = (ctypes.c_double * nc)()
    by = (ctypes.c_double * nc)()
    la = (ctypes.c_uint64 * nc)()
    cm = (ctypes.c_double * nc)()
    lib = load_library()
    _check(lib.ttn_profile_end(ctypes.byref(ms), ctypes.byref(nl), fl, by, la))
    _check(lib.ttn_profile_class_ms(cm))
    ep = (ctypes.c_double * 6)()
    _check(lib.ttn_profile_eig_phases(ep))
    mh = (ctypes.c_double * (2 * 513 * 4))()
    _check(lib.ttn_profile_move_hist(mh))
    hist = np.array(list(mh)).reshape(2, 513, 4)
    nk = ctypes.c_uint64()
    _check(lib.ttn_profile_kernels(ctypes.byref(nk)))
    return dict(timed_ms=ms.value, timed_launches=nl.value, move_hist=hist, kernels=nk.value,
                flops=dict(zip(KERNEL_CLASSES, list(fl))), bytes=dict(zip(KERNEL_CLASSES, list(by))),
                launches=dict(zip(KERNEL_CLASSES, list(la))), class_ms=dict(zip(KERNEL_CLASSES, list(cm))),
                eig_phase_cycles=dict(zip(EIG_PHASES, list(ep))))


def grad(circuit, shots, wrt="theta", noise="srx", theta=0.0, gamma=0.0, chi=16, precision="fp64",
         seed=0, first_traj=0, h=1e-4, svd_eps=0.0, svd_mode="auto", gemm_mode="auto",
         return_score=False):
    """Score-function estimate of dp_L/d(theta or gamma): (p_L, dpL, sigma[, score])."""
    lib = load_library()
    p, keep = _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                          svd_mode=svd_mode, gemm_mode=gemm_mode)
    pl, g, sg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    score = np.zeros(shots) if return_score else None
    _check(lib.ttn_grad(circuit.handle, ctypes.byref(p), shots, 0 if wrt == "theta" else 1, h,
                        ctypes.byref(pl), ctypes.byref(g), ctypes.byref(sg),
                        score.ctypes.data_as(c_dblp) if return_score else None))
    if return_score:
        return pl.value, g.value, sg.value, score
    return pl.value, g.value, sg.value


def grad_sums(circuit, shots, wrt="theta", noise="srx", theta=0.0, gamma=0.0, chi=16,
              precision="fp64", seed=0, first_traj=0, h=1e-4, svd_eps=0.0, svd_mode="auto",
              gemm_mode="auto"):
    """ttn_grad_sums: (n_valid, n_fail, sum_fs, sum_fs2) of the score-function estimator."""
    lib = load_library()
    p, keep = _run_params(noise, theta, gamma, chi, precision, seed, first_traj, svd_eps,
                          svd_mode=svd_mode, gemm_mode=gemm_mode)
    nv, nf = ctypes.c_uint64(), ctypes.c_uint64()
    s1, s2 = ctypes.c_double(), ctypes.c_double()
    st = lib.ttn_grad_sums(circuit.handle, ctypes.byref(p), shots, 0 if wrt == "theta" else 1, h,
                           ctypes.byref(nv), ctypes.byref(nf), ctypes.byref(s1), ctypes.byref(s2))
    if st not in (0, 6):      # 6: some shots exceeded the decoder's bound and were not counted
        _check(st)
    del keep
    return nv.value, nf.value, s1.value, s2.value


def slot_check(circuit, noise="srx", chi=16):
    """ttn_slot_check: {worst_fill, worst_node, worst_step, binding_moves}."""
    lib = load_library()
    wf, wn, ws, nb = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib.ttn_slot_check(circuit.handle, NOISE[noise] if isinstance(noise, str) else int(noise),
                              chi, ctypes.byref(wf), ctypes.byref(wn), ctypes.byref(ws),
                              ctypes.byref(nb)))
    return dict(worst_fill=wf.value, worst_node=wn.value, worst_step=ws.value,
                binding_moves=nb.value)


def logical_error_rate_fn(circuit, shots, **kw):
    """torch.autograd.Function whose forward is p_L(theta) and whose backward
    is the score-function dp_L/dtheta from ttn_grad."""
    import torch

    class _PL(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta):
            pl, g, sg = grad(circuit, shots, wrt="theta", theta=float(theta), **kw)
            ctx.g = g
            return torch.tensor(pl, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            return gout * ctx.g

    return _PL.apply


def decode_noalloc(circuit, records, fail, color=None, score=None, stream=None):
    """Allocation-free decoding of records already on the device (torch CUDA
    tensors on the current device: records uint8 [n][n_record_bits], fail
    uint8 [n], color int32 [n], score int64 [n]).  The library decodes with
    static device scratch and calls no cudaMalloc, for callers whose memory
    pool owns the device.  `stream` is a CUDA stream handle (int); 0 or None =
    the default stream.  Every tensor is checked here (device, layout, dtype,
    size) because the kernel reads and writes them as raw device memory."""
    import torch
    cur = torch.cuda.current_device() if torch.cuda.is_available() else None
    n = None

    def need(name, t, dtype, rows, cols=None):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != cur:
            raise ValueError("decode_noalloc: %s must be a CUDA tensor on the current device" % name)
        if not t.is_contiguous():
            raise ValueError("decode_noalloc: %s must be contiguous" % name)
        if t.dtype != dtype:
            raise ValueError("decode_noalloc: %s must be %s, got %s" % (name, dtype, t.dtype))
        if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
            raise ValueError("decode_noalloc: %s must have shape (n, %d)" % (name, cols))
        if t.numel() < rows * (cols or 1):
            raise ValueError("decode_noalloc: %s holds fewer than %d entries" % (name, rows * (cols or 1)))

    if not isinstance(records, torch.Tensor) or records.dim() != 2:
        raise ValueError("decode_noalloc: records must be a 2-d torch tensor (n, n_record_bits)")
    n = int(records.shape[0])
    need("records", records, torch.uint8, n, circuit.n_record_bits)
    need("fail", fail, torch.uint8, n)
    if color is not None:
        need("color", color, torch.int32, n)
    if score is not None:
        need("score", score, torch.int64, n)
    st = ctypes.c_void_p(int(stream)) if stream else None
    _check(load_library().ttn_decode_noalloc(circuit.handle, n, _ptr(records), _ptr(fail),
                                             _ptr(color), _ptr(score), st))
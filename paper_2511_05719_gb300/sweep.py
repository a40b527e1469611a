"""Threshold sweep from the command line: p_L at every (distance, strength)
point of a grid (Sec. IV.A: failure curves over the physical error strength
for several distances), each point checkpointed so an interrupted sweep
resumes, then optionally the Eq. 4 fit over all points.

    python -m paper_2511_05719_gb300.sweep --distances 3,5 --rounds d \\
        --noise srx --strengths 0.02,0.04,0.06 --chi 64 --shots 20000 \\
        --state-dir sweep_state --fit

One JSON line per point on stdout (distance, rounds, strength, p_L, sigma,
n_fail, n_valid), and a final line with the fit when --fit is given."""
import argparse
import json
import math
import os
import sys


def parse(argv):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--distances", required=True, help="comma-separated odd distances")
    ap.add_argument("--rounds", default="d", help="syndrome rounds: an integer, or d for C = d")
    ap.add_argument("--noise", default="srx", choices=["srx", "ad", "srx_pta", "ad_pta", "srx_ad"])
    ap.add_argument("--strengths", required=True,
                    help="comma-separated theta (srx models) or gamma (ad models) values")
    ap.add_argument("--theta", type=float, default=0.0, help="fixed theta for srx_ad gamma sweeps")
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--layout", default="optimized", choices=["default", "optimized", "search"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--shots", type=int, default=10000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--state-dir", default="sweep_state")
    ap.add_argument("--log", default=None, help="JSONL log of every batch")
    ap.add_argument("--fit", action="store_true", help="fit Eq. 4 over all points")
    ap.add_argument("--tau0", type=float, default=None, help="starting threshold of the fit")
    a = ap.parse_args(argv)
    a.distances = [int(x) for x in a.distances.split(",")]
    a.strengths = [float(x) for x in a.strengths.split(",")]
    if any(d < 3 or d % 2 == 0 for d in a.distances):
        ap.error("distances must be odd and >= 3")
    return a


def main(argv=None, run=None, circuit=None, fit=None, out=sys.stdout):
    """`run`, `circuit` and `fit` default to the library's run_trajectories,
    Circuit and threshold_fit."""
    from .checkpoint import logical_error_rate_resumable
    a = parse(argv)
    if circuit is None or fit is None:
        from . import _lib
        circuit = circuit or _lib.Circuit
        fit = fit or _lib.threshold_fit
    os.makedirs(a.state_dir, exist_ok=True)
    wrt = "gamma" if a.noise in ("ad", "ad_pta", "srx_ad") else "theta"
    pts = []
    for d in a.distances:
        C = d if a.rounds == "d" else int(a.rounds)
        circ = circuit(d, C, layout=a.layout)
        for x in a.strengths:
            kw = dict(noise=a.noise, chi=a.chi, precision=a.precision, seed=a.seed)
            if wrt == "gamma":
                kw.update(gamma=x, theta=a.theta)
            else:
                kw.update(theta=x)
            state = os.path.join(a.state_dir, "d%d_C%d_%s_%s%.6g_chi%d_%s.json"
                                 % (d, C, a.noise, wrt, x, a.chi, a.precision))
            p, s, nf, nv = logical_error_rate_resumable(circ, a.shots, state, batch=a.batch,
                                                        log_path=a.log, run=run, **kw)
            rec = dict(distance=d, rounds=C, noise=a.noise, strength=x, chi=a.chi, p_L=p, sigma=s,
                       n_fail=nf, n_valid=nv)
            pts.append(rec)
            out.write(json.dumps(rec) + "\n")
            out.flush()
    if a.fit:
        use = [r for r in pts if r["n_valid"] > 0 and 0 < r["n_fail"] < r["n_valid"]]
        tau0 = a.tau0 if a.tau0 is not None else sorted(a.strengths)[len(a.strengths) // 2]
        r = fit([q["distance"] for q in use], [q["strength"] for q in use], [q["p_L"] for q in use],
                [q["sigma"] for q in use], tau0=tau0)
        out.write(json.dumps(dict(fit="eq4", tau=r["tau"], nu=r["nu"],
                                  tau_sigma=math.sqrt(max(r["cov"][3][3], 0.0)),
                                  A=r["A"], B=r["B"], C=r["C"], chi2=r["chi2"],
                                  points=len(use))) + "\n")
    return pts


if __name__ == "__main__":
    main()

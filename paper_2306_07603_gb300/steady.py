"""Error of the FP32-deviation form against the FP64 form, per field.

Runs every cavity of a workload from rest in FP64 until the max-norm
velocity residual of one step (max|u^n - u^(n-1)| / max|u^n|) is below
``tol`` for every cavity, or ``max_steps`` steps. The FP32-deviation form
then runs from rest for the same number of steps (the equal-step error, for
every cavity, steady or not), and on to ``fp32_factor`` times as many: its
trajectory leaves the FP64 one during the transient and relaxes towards its
own steady state along the slowest cavity mode, so for the cavities whose
FP64 run did reach ``tol`` (steady) the error is also reported after the
longer run, where it has levelled off. Fields: u, v, psi, and P minus its
mean (the mean pressure is a neutral mode of the scheme); error =
max|a - b| / max|b|. Cavities whose FP64 run does not settle are also
compared by their time-mean fields over a common window (``--window``; with
``--mean-all`` every cavity).
Both runs use the library only; the FP64 form is the one whose steps match
the oracle to 1e-12.

    python -m paper_2306_07603_gb300.steady --workload sweep257
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .solver import Solver, cavity
from .workloads import WORKLOAD_OPTIONS, WORKLOADS


def _solver(specs, precision, **opts):
    return Solver([cavity(c.nx, c.ny, c.Re, c.n, theta_deg=c.theta_deg, U_lid=c.U_lid, L=c.L,
                          H=c.H) for c in specs], precision=precision, **opts)


def _fields(s, ncav):
    out = []
    for k in range(ncav):
        m = s.macros(k)
        m["P"] = (m["rho"] - 1.0) / 3.0   # rho = rho0 + P / c_s^2 with rho0 = 1, c = 1
        out.append(m)
    return out


def _errors(a, b):
    err = {q: float(np.abs(a[q] - b[q]).max() / np.abs(b[q]).max()) for q in ("u", "v", "psi")}
    pa, pb = a["P"] - a["P"].mean(), b["P"] - b["P"].mean()
    err["P - mean"] = float(np.abs(pa - pb).max() / np.abs(pb).max())
    return err


def _mean_fields(s, ncav, steps, every):
    """Advances `steps` steps, sampling the fields every `every` steps; returns
    their time means (u, v, psi, P) per cavity."""
    acc = None
    n = 0
    for _ in range(steps // every):
        s.step(every)
        f = _fields(s, ncav)
        if acc is None:
            acc = [{q: m[q].copy() for q in ("u", "v", "psi", "P")} for m in f]
        else:
            for a, m in zip(acc, f):
                for q in a:
                    a[q] += m[q]
        n += 1
    return [{q: a[q] / n for q in a} for a in acc]


def compare(workload="sweep257", tol=1e-8, max_steps=200000, chunk=2000, kernel="auto",
            fp32_factor=3, window=0, every=1000, only=None, mean_all=False):
    """FP64 run to `tol` (or `max_steps`), then the FP32-deviation run (see the
    module docstring). With `window` > 0, the cavities whose FP64 run did not
    reach `tol` are also compared by their time-mean fields over the window of
    `window` steps that follows, sampled every `every` steps, in both forms."""
    specs = WORKLOADS[workload]()
    if only:
        specs = [specs[k] for k in only]
    opts = dict(WORKLOAD_OPTIONS.get(workload, {}), kernel=kernel)
    s = _solver(specs, "fp64", **opts)
    steps, t0 = 0, time.time()
    hist64 = []
    while True:
        s.step(chunk)
        steps += chunk
        r64 = [float(row[2]) for row in s.residual()]
        hist64.append((steps, max(r64)))
        if max(r64) < tol or steps >= max_steps:
            break
    s.sync()
    f64 = _fields(s, len(specs))
    mean64 = _mean_fields(s, len(specs), window, every) if window else None
    w64 = time.time() - t0
    s.close()

    s = _solver(specs, "fp32dev", **opts)
    t0 = time.time()
    s.step(steps)
    f32 = _fields(s, len(specs))
    equal = [_errors(f32[k], f64[k]) for k in range(len(specs))]
    mean32 = _mean_fields(s, len(specs), window, every) if window else None
    s.step(max(0, (fp32_factor - 1) * steps - window))
    f32 = _fields(s, len(specs))
    w32 = time.time() - t0
    r32 = [float(row[2]) for row in s.residual()]
    s.close()
    rows = []
    for k, c in enumerate(specs):
        steady = r64[k] < tol
        rows.append({"grid": f"{c.nx}x{c.ny}", "theta": c.theta_deg, "n": c.n, "Re": c.Re,
                     "fp64_rinf": r64[k], "fp64_steady": steady, "fp32_rinf": r32[k],
                     "error_equal_steps": equal[k],
                     "error_steady": _errors(f32[k], f64[k]) if steady else None,
                     "error_time_mean": (_errors(mean32[k], mean64[k])
                                         if (window and (mean_all or not steady)) else None)})
    worst = {q: max(r["error_equal_steps"][q] for r in rows) for q in equal[0]}
    st = [r["error_steady"] for r in rows if r["error_steady"] is not None]
    worst_steady = {q: max(e[q] for e in st) for q in st[0]} if st else None
    return {"workload": workload, "tol": tol, "fp64_steps": steps,
            "fp32dev_steps": max(fp32_factor * steps, steps + window),
            "window": window, "every": every, "fp64_seconds": round(w64, 2),
            "fp32dev_seconds": round(w32, 2), "max_error_equal_steps": worst,
            "max_error_steady": worst_steady, "fp64_rinf_history": hist64[::10],
            "cavities": rows}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", default="sweep257", choices=sorted(WORKLOADS))
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--max-steps", type=int, default=200000)
    p.add_argument("--chunk", type=int, default=2000)
    p.add_argument("--kernel", default="auto", choices=["auto", "staged", "fused"])
    p.add_argument("--fp32-factor", type=int, default=3)
    p.add_argument("--window", type=int, default=0,
                   help="steps of the time-mean comparison of the cavities that do not settle")
    p.add_argument("--every", type=int, default=1000)
    p.add_argument("--save", default=None, help="also write the result to this JSON file")
    p.add_argument("--only", default=None, help="comma-separated indices of the cavities to run")
    p.add_argument("--mean-all", action="store_true",
                   help="compare the time-mean fields over the window for every cavity, "
                        "steady ones included (the FP32 form's steady state carries rounding "
                        "noise that the slow cavity modes integrate)")
    a = p.parse_args(argv)
    only = [int(k) for k in a.only.split(",")] if a.only else None
    out = compare(a.workload, a.tol, a.max_steps, a.chunk, a.kernel, a.fp32_factor, a.window,
                  a.every, only, a.mean_all)
    if a.save:
        with open(a.save, "w") as f:
            json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

"""Steady-state error of the FP32-deviation form against the FP64 form.

Runs every cavity of a workload from rest in FP64 until the max-norm
velocity residual of one step (max|u^n - u^(n-1)| / max|u^n|) is below
``tol`` for every cavity, or ``max_steps`` steps. The FP32-deviation form,
whose residual stalls at its rounding floor (~2e-7), then runs from rest for
``fp32_factor`` times as many steps: its trajectory relaxes towards its own
steady state along the slowest cavity mode, and the error against the FP64
fields is recorded at checkpoints until it levels off. Reported per cavity
and field (u, v, psi, and P minus its mean: the mean pressure is a neutral
mode of the scheme): max|a - b| / max|b|. Both runs use the library only;
the FP64 form is the one whose steps match the oracle to 1e-12.

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


def compare(workload="sweep257", tol=1e-8, max_steps=200000, chunk=2000, kernel="auto",
            fp32_factor=3, checkpoints=6):
    specs = WORKLOADS[workload]()
    opts = dict(WORKLOAD_OPTIONS.get(workload, {}), kernel=kernel)
    s = _solver(specs, "fp64", **opts)
    steps, t0 = 0, time.time()
    while True:
        s.step(chunk)
        steps += chunk
        r64 = [float(row[2]) for row in s.residual()]
        if max(r64) < tol or steps >= max_steps:
            break
    s.sync()
    w64 = time.time() - t0
    f64 = _fields(s, len(specs))
    s.close()

    s = _solver(specs, "fp32dev", **opts)
    total = fp32_factor * steps
    marks = sorted({max(chunk, total * (m + 1) // checkpoints) for m in range(checkpoints)})
    done, t0, history = 0, time.time(), []
    for mark in marks:
        s.step(mark - done)
        done = mark
        f32 = _fields(s, len(specs))
        history.append({"steps": done, "max_error": {
            q: max(_errors(f32[k], f64[k])[q] for k in range(len(specs)))
            for q in ("u", "v", "psi", "P - mean")}})
    w32 = time.time() - t0
    r32 = [float(row[2]) for row in s.residual()]
    s.close()
    rows = []
    for k, c in enumerate(specs):
        rows.append({"grid": f"{c.nx}x{c.ny}", "theta": c.theta_deg, "n": c.n, "Re": c.Re,
                     "fp64_rinf": r64[k], "fp32_rinf": r32[k], "error": _errors(f32[k], f64[k])})
    return {"workload": workload, "tol": tol, "fp64_steps": steps, "fp32dev_steps": done,
            "fp64_seconds": round(w64, 2), "fp32dev_seconds": round(w32, 2),
            "fp32_history": history, "cavities": rows}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", default="sweep257", choices=sorted(WORKLOADS))
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--max-steps", type=int, default=200000)
    p.add_argument("--chunk", type=int, default=2000)
    p.add_argument("--kernel", default="auto", choices=["auto", "staged", "fused"])
    p.add_argument("--fp32-factor", type=int, default=3)
    a = p.parse_args(argv)
    print(json.dumps(compare(a.workload, a.tol, a.max_steps, a.chunk, a.kernel, a.fp32_factor)))


if __name__ == "__main__":
    main()

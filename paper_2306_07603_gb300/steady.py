"""Steady-state error of the FP32-deviation form against the FP64 form.

Runs every cavity of a workload from rest in FP64 and in FP32-deviation
storage until the max-norm velocity residual of one step (Eq. 2.19's
companion, max|u^n - u^(n-1)| / max|u^n|) is below ``tol`` for every
cavity, or ``max_steps`` steps, and reports per cavity and field (u, v, P,
psi) max|a - b| / max|b| between the two forms. Both runs use the library
only; the FP64 form is the one whose steps match the oracle to 1e-12.

    python -m paper_2306_07603_gb300.steady --workload sweep257
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .solver import Solver, cavity
from .workloads import WORKLOAD_OPTIONS, WORKLOADS


def run_to_steady(specs, precision, tol, max_steps, chunk, **opts):
    s = Solver([cavity(c.nx, c.ny, c.Re, c.n, theta_deg=c.theta_deg, U_lid=c.U_lid, L=c.L, H=c.H)
                for c in specs], precision=precision, **opts)
    steps, t0 = 0, time.time()
    while True:
        s.step(chunk)
        steps += chunk
        r = s.residual()
        if max(row[2] for row in r) < tol or steps >= max_steps:
            break
    s.sync()
    wall = time.time() - t0
    fields = []
    for k, c in enumerate(specs):
        m = s.macros(k)
        m["P"] = (m["rho"] - 1.0) / 3.0   # rho = rho0 + P / c_s^2 with rho0 = 1, c = 1
        fields.append(m)
    s.close()
    return fields, steps, [float(row[2]) for row in r], wall


def compare(workload="sweep257", tol=1e-8, max_steps=200000, chunk=2000, kernel="auto"):
    specs = WORKLOADS[workload]()
    opts = dict(WORKLOAD_OPTIONS.get(workload, {}), kernel=kernel)
    f64, s64, r64, w64 = run_to_steady(specs, "fp64", tol, max_steps, chunk, **opts)
    f32, s32, r32, w32 = run_to_steady(specs, "fp32dev", tol, max_steps, chunk, **opts)
    rows = []
    for k, c in enumerate(specs):
        err = {q: float(np.abs(f32[k][q] - f64[k][q]).max() / np.abs(f64[k][q]).max())
               for q in ("u", "v", "P", "psi")}
        rows.append({"grid": f"{c.nx}x{c.ny}", "theta": c.theta_deg, "n": c.n, "Re": c.Re,
                     "fp64_rinf": r64[k], "fp32_rinf": r32[k], "error": err})
    return {"workload": workload, "tol": tol, "fp64_steps": s64, "fp32dev_steps": s32,
            "fp64_seconds": round(w64, 2), "fp32dev_seconds": round(w32, 2), "cavities": rows}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", default="sweep257", choices=sorted(WORKLOADS))
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--max-steps", type=int, default=200000)
    p.add_argument("--chunk", type=int, default=2000)
    p.add_argument("--kernel", default="auto", choices=["auto", "staged", "fused"])
    a = p.parse_args(argv)
    print(json.dumps(compare(a.workload, a.tol, a.max_steps, a.chunk, a.kernel)))


if __name__ == "__main__":
    main()

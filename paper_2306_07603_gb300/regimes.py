"""Unsteady cavity flows: probe and kinetic-energy time series and their statistics.

Sec. 5.3 of the paper follows the velocity (u, v) at the cavity centre, the
point (1.07735, 0.5) of the theta = 60 deg map (xi = eta = 0.5), and the
kinetic energy E(t) of Eq. (5.1), and calls a flow steady, periodic,
quasi-periodic or turbulent from the phase portrait of (u, v) and the power
spectrum of E(t). This module records those series on the GPU without
synchronising (``ifdlbm_probe_dev``, ``ifdlbm_residual_dev``, one sample every
``every`` steps) and reduces them on the host:

* mean and variance of E and of u, v at every probe;
* the power spectrum of E(t) - mean (Hann window), its principal frequency
  and period (in lattice time units, t = steps x dt), and its peaks;
* a regime label. The paper gives the regimes by inspection only; the rule
  used here (a reading) works on E(t) minus its linear trend over the record:
  steady if its relative standard deviation is below ``steady_tol``;
  drifting (the record is too short to tell: the flow is still settling) if
  the strongest spectral peak lies in the lowest ``drift_bins`` bins;
  turbulent if less than ``concentration`` of the fluctuation power lies
  within two bins of the ``max_discrete`` strongest peaks (a broadband
  spectrum); else periodic if every peak above ``peak_frac`` of the largest
  lies within one bin of a multiple of the principal frequency, and
  quasi-periodic if not. The relative drift of E over the record is
  reported beside the label.

The arithmetic of the step runs in libifdlbm.so; only the statistics of the
recorded series are formed here.

    python -m paper_2306_07603_gb300.regimes --cases theta60     # Sec. 5.3, theta = 60 deg
    python -m paper_2306_07603_gb300.regimes --case 257,60,1.5,4000 --precision fp64
    python -m paper_2306_07603_gb300.regimes --workload unsteady1025
    python -m paper_2306_07603_gb300.regimes --workload unsteady1025 --compare-precisions \
        --transient 50000 --steps 100000
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from .workloads import WORKLOAD_OPTIONS, WORKLOADS, CavitySpec

# Sec. 5.3, theta = 60 deg, 256^2 cells: the cases whose regime the paper states.
THETA60 = [CavitySpec(257, 257, Re, n, 60.0) for n, Re in
           ((1.5, 3000.0), (1.5, 4000.0), (1.5, 5000.0), (1.0, 2500.0), (1.0, 3000.0),
            (1.0, 4000.0), (0.5, 750.0), (0.5, 1000.0), (0.5, 2000.0))]

# probe points (xi, eta): the cavity centre first (the paper's probe), then the
# four quarter points
PROBES = ((0.5, 0.5), (0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75))


def record(specs, precision="fp32dev", transient=1_000_000, steps=1_000_000, every=100,
           probes=PROBES, **opts):
    """Advance all cavities `transient` steps, then record `steps` more, sampling
    E(t) and u, v at the probe nodes every `every` steps."""
    import torch

    from . import capi
    from .solver import Solver, cavity, quad_cavity
    s = Solver([quad_cavity(c.nx, c.ny, c.corners, c.Re, c.n, U_lid=c.U_lid, H=c.H)
                if hasattr(c, "corners") else
                cavity(c.nx, c.ny, c.Re, c.n, theta_deg=c.theta_deg, U_lid=c.U_lid, L=c.L, H=c.H)
                for c in specs], precision=precision, **opts)
    idx = [(k, int(round(xi * (c.nx - 1))), int(round(eta * (c.ny - 1))))
           for k, c in enumerate(specs) for (xi, eta) in probes]
    nsamp = steps // every
    with torch.cuda.stream(s.stream):
        pidx = torch.tensor(idx, dtype=torch.int32, device="cuda")
        pbuf = torch.empty((nsamp, len(idx), 3), dtype=torch.float64, device="cuda")
        rbuf = torch.empty((nsamp, len(specs), 4), dtype=torch.float64, device="cuda")
    t0 = time.time()
    done = 0
    while done < transient:
        k = min(100_000, transient - done)
        s.step(k)
        done += k
    for m in range(nsamp):
        s.step(every)
        capi.ifdlbm_probe_dev(s.h, pidx, pbuf[m])
        capi.ifdlbm_residual_dev(s.h, rbuf[m])
    s.sync()
    wall = time.time() - t0
    dts = [capi.ifdlbm_info(s.h, k).dt for k in range(len(specs))]
    out = {"probes": pbuf.cpu().numpy().reshape(nsamp, len(specs), len(probes), 3),
           "energy": rbuf.cpu().numpy()[:, :, 3], "dt": dts, "every": every,
           "transient": transient, "steps": steps, "seconds": wall,
           "lattice_updates": sum(c.nodes for c in specs) * (transient + steps)}
    s.close()
    return out


def spectrum(x, dt_sample):
    """One-sided power spectrum of x - mean with a Hann window."""
    y = (x - x.mean()) * np.hanning(len(x))
    p = np.abs(np.fft.rfft(y)) ** 2
    f = np.fft.rfftfreq(len(x), d=dt_sample)
    return f, p


def classify(E, dt_sample, steady_tol=1e-6, peak_frac=0.01, max_discrete=12, concentration=0.8,
             drift_bins=3):
    """Regime of an energy series (see the module docstring) and its spectrum facts."""
    E = np.asarray(E, dtype=float)
    t = np.arange(len(E), dtype=float)
    slope, icpt = np.polyfit(t, E, 1)
    r = E - (slope * t + icpt)
    mean, std = float(E.mean()), float(r.std())
    drift = float(slope * (len(E) - 1) / mean)
    facts = {"rel_std": std / abs(mean), "drift": drift}
    if std <= steady_tol * abs(mean):
        return {"regime": "steady", **facts, "f0": None, "period": None, "peaks": [],
                "concentration": None}
    f, p = spectrum(r, dt_sample)
    p[0] = 0.0
    df = f[1] - f[0]
    k0 = int(np.argmax(p))
    f0 = float(f[k0])
    # local maxima above peak_frac of the largest, strongest first
    pk = sorted((k for k in range(1, len(p) - 1)
                 if p[k] >= peak_frac * p[k0] and p[k] >= p[k - 1] and p[k] >= p[k + 1]),
                key=lambda k: -p[k])
    near = np.zeros(len(p), dtype=bool)
    for k in pk[:max_discrete]:
        near[max(k - 2, 0):k + 3] = True
    conc = float(p[near].sum() / p.sum())
    if k0 <= drift_bins:
        regime = "drifting"
    elif conc < concentration:
        regime = "turbulent"
    elif all(round(f[k] / f0) >= 1 and abs(f[k] - round(f[k] / f0) * f0) <= df for k in pk):
        regime = "periodic"
    else:
        regime = "quasi-periodic"
    return {"regime": regime, **facts, "f0": f0, "period": 1.0 / f0 if f0 > 0 else None,
            "peaks": [float(f[k]) for k in pk[:8]], "concentration": conc}


def summarize(specs, rec, probes=PROBES, **kw):
    rows = []
    for k, c in enumerate(specs):
        dts = rec["dt"][k] * rec["every"]
        E = rec["energy"][:, k]
        cl = classify(E, dts, **kw)
        pr = rec["probes"][:, k]
        rows.append({
            "grid": f"{c.nx}x{c.ny}", "theta": getattr(c, "theta_deg", None),
            "corners": getattr(c, "corners", None), "n": c.n, "Re": c.Re,
            "E_mean": float(E.mean()), "E_var": float(E.var()), **cl,
            "probes": [{"xi": xi, "eta": eta, "u_mean": float(pr[:, q, 0].mean()),
                        "u_var": float(pr[:, q, 0].var()), "v_mean": float(pr[:, q, 1].mean()),
                        "v_var": float(pr[:, q, 1].var())}
                       for q, (xi, eta) in enumerate(probes)]})
    return rows


def _rel(a, b):
    return float(abs(a - b) / abs(b)) if b != 0 else float(abs(a - b))


def compare_precisions(specs, transient, steps, every=100, **opts):
    """The same cavities and window in the FP64 form and the FP32-deviation
    form: per cavity, the mean, variance and principal period of E(t) and the
    mean and variance of u, v at every probe in both, and their relative
    differences (FP32 against FP64). Returns (rows, seconds per form)."""
    rec = {p: record(specs, p, transient, steps, every, **opts) for p in ("fp64", "fp32dev")}
    sm = {p: summarize(specs, rec[p]) for p in rec}
    rows = []
    for k, c in enumerate(specs):
        a, b = sm["fp32dev"][k], sm["fp64"][k]
        d = {"E_mean": _rel(a["E_mean"], b["E_mean"]), "E_var": _rel(a["E_var"], b["E_var"]),
             "period": (_rel(a["period"], b["period"])
                        if a["period"] and b["period"] else None)}
        e64 = rec["fp64"]["energy"][:, k]
        e32 = rec["fp32dev"]["energy"][:, k]
        d["E_series_max"] = float(np.abs(e32 - e64).max() / np.abs(e64).max())
        pr = []
        for q in range(len(a["probes"])):
            pa, pb = a["probes"][q], b["probes"][q]
            scale = max(abs(pb["u_mean"]), abs(pb["v_mean"]), 1e-30)
            pr.append({"xi": pb["xi"], "eta": pb["eta"],
                       "u_mean": abs(pa["u_mean"] - pb["u_mean"]) / scale,
                       "v_mean": abs(pa["v_mean"] - pb["v_mean"]) / scale,
                       "u_std": _rel(pa["u_var"] ** 0.5, pb["u_var"] ** 0.5),
                       "v_std": _rel(pa["v_var"] ** 0.5, pb["v_var"] ** 0.5)})
        d["probes"] = pr
        rows.append({"grid": f"{c.nx}x{c.ny}", "theta": getattr(c, "theta_deg", None), "n": c.n,
                     "Re": c.Re, "fp64": b, "fp32dev": a, "difference": d})
    return rows, {p: round(rec[p]["seconds"], 1) for p in rec}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--cases", choices=["theta60"], default=None)
    p.add_argument("--workload", choices=sorted(WORKLOADS), default=None)
    p.add_argument("--case", default=None, help="one cavity: N,theta_deg,n,Re (e.g. 257,60,1.5,4000)")
    p.add_argument("--precision", default="fp32dev", choices=["fp32dev", "fp64"])
    p.add_argument("--transient", type=int, default=1_000_000)
    p.add_argument("--steps", type=int, default=1_000_000)
    p.add_argument("--every", type=int, default=100)
    p.add_argument("--save", default=None, help="write the raw series to this .npz")
    p.add_argument("--eta-b", type=float, default=None, help="blend of Eq. 2.5 (default 0.5)")
    p.add_argument("--dt-mode", choices=["contravariant", "grid"], default=None,
                   help="time-step rule (default contravariant)")
    p.add_argument("--cfl", type=float, default=None, help="Courant number (default 0.5)")
    p.add_argument("--wall-pressure", choices=["zeroth", "first"], default=None,
                   help="pressure of the wall rule (default zeroth; first runs on the staged "
                        "kernels)")
    p.add_argument("--kernel", choices=["auto", "staged", "fused"], default=None)
    p.add_argument("--only", default=None,
                   help="with --cases: comma-separated indices of the cases to run")
    p.add_argument("--compare-precisions", action="store_true",
                   help="run the window in FP64 and in the FP32-deviation form and report "
                        "the differences of the statistics")
    a = p.parse_args(argv)
    if a.case:
        N, th, n, Re = (float(v) for v in a.case.split(","))
        specs, opts = [CavitySpec(int(N), int(N), Re, n, th)], {}
    elif a.workload:
        specs, opts = WORKLOADS[a.workload](), dict(WORKLOAD_OPTIONS.get(a.workload, {}))
    else:
        specs, opts = THETA60, {}
        if a.only:
            specs = [specs[int(k)] for k in a.only.split(",")]
    if a.eta_b is not None:
        opts["eta_b"] = a.eta_b
    if a.dt_mode is not None:
        opts["dt_mode"] = a.dt_mode
    if a.cfl is not None:
        opts["cfl"] = a.cfl
    if a.wall_pressure is not None:
        opts["wall_pressure"] = a.wall_pressure
    if a.kernel is not None:
        opts["kernel"] = a.kernel
    if a.compare_precisions:
        rows, secs = compare_precisions(specs, a.transient, a.steps, a.every, **opts)
        print(json.dumps({"compare": "fp32dev vs fp64", "eta_b": opts.get("eta_b", 0.5),
                          "transient": a.transient, "steps": a.steps, "every": a.every,
                          "seconds": secs, "cases": rows}))
        return
    rec = record(specs, a.precision, a.transient, a.steps, a.every, **opts)
    if a.save:
        np.savez_compressed(a.save, probes=rec["probes"], energy=rec["energy"],
                            dt=np.array(rec["dt"]), every=a.every)
    print(json.dumps({"precision": a.precision, "eta_b": opts.get("eta_b", 0.5),
                      "dt_mode": opts.get("dt_mode", "contravariant"), "cfl": opts.get("cfl", 0.5),
                      "wall_pressure": opts.get("wall_pressure", "zeroth"),
                      "transient": a.transient, "steps": a.steps,
                      "every": a.every, "seconds": round(rec["seconds"], 1),
                      "mlups": round(rec["lattice_updates"] / rec["seconds"] / 1e6, 1),
                      "cases": summarize(specs, rec)}))


if __name__ == "__main__":
    main()

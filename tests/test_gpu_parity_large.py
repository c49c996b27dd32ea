"""GPU parity at the layouts and sizes the product runs (one step against the oracle).

The autotuner picks wide CTAs with long row segments on large cavities
(256 threads x 64 or 128 rows on a 2049^2 cavity; 64 threads x 32 rows on the
257^2 sweep; DYNAMIC schedules with 128-row tasks on the 64-cavity batch of
grids up to 513^2). These tests run exactly those layouts on cavities large
enough for several strips and several row segments per cavity, and compare
one step with the FP64 oracle: FP64 at the 1e-12 bars of
``test_gpu_parity.compare_state``; the FP32-deviation form with u, v within
1e-5 of the largest speed, P within 1e-4, and lambda within its FP32
conditioning bound (``lam_bound32``).

Inputs are seeded smooth synthetic states (equilibria of random smooth P, u, v
plus a random smooth non-equilibrium part, and a smooth positive lambda), so
that every node of every strip and segment carries gradients and shear; one
case is a state the oracle developed from rest.
"""
import numpy as np
import pytest

import oracle as O
from paper_2306_07603_gb300.workloads import smooth_noise
from test_gpu_parity import cav, compare_state, lam_bound, oracle_run, rel, solver

pytestmark = pytest.mark.gpu


def synthetic_state(run, seed):
    """A non-trivial state on the run's grid (seeded; no GPU input)."""
    ny, nx = run.g.ny, run.g.nx
    P = 1e-3 * smooth_noise((ny, nx), seed)
    u = 0.05 * smooth_noise((ny, nx), seed + 1)
    v = 0.05 * smooth_noise((ny, nx), seed + 2)
    f = O.equilibrium(P, u, v) + 2e-4 * smooth_noise((9, ny, nx), seed + 3)
    lam = run.lam * (1.0 + 0.3 * smooth_noise((ny, nx), seed + 4))
    return f, lam


def lam_bound32(f_in, lam_in, prm, lam_out):
    """Pointwise bound on |lambda_fp32 - lambda_oracle| after one step of the
    FP32-deviation form. Its strain rate (Eqs. 2.12-2.13) comes from FP32
    differences g - g^eq of the stored deviations g = f-hat - w rho0: their
    rounding, ~eps32 max|g| per population, is a fraction
    16 eps32 max|g| / (lambda_prev c_s^2 gamma-dot) of the strain rate, which
    Eq. (1.4) passes to lambda times |n - 1| (as lam_bound does for FP64,
    with the FP32 epsilon). On top: 1e-6 of max lambda for the FP32 rounding
    of lambda itself and of the collision arithmetic."""
    ux, uy, P = O.macros(f_in)
    feq = O.equilibrium(P, ux, uy)
    f = O.f_from_fhat(f_in, feq, lam_in, prm.dt)
    gd = O.shear_rate(*O.strain_rate(f, feq, lam_in))
    cs2 = prm.c ** 2 / 3.0
    g = f_in - O.OMEGA[:, None, None] * prm.rho0
    dfne = 16.0 * np.finfo(np.float32).eps * np.abs(g).max()
    cond = abs(prm.n - 1.0) * lam_out * dfne / (lam_in * cs2 * np.maximum(gd, prm.gamma_min))
    return 1e-6 * np.abs(lam_out).max() + cond


def check_fp32(fg, lg, fo, lo, f0, l0, prm):
    ug, vg, Pg = O.macros(fg)
    uo, vo, Po = O.macros(fo)
    umax = np.sqrt(uo ** 2 + vo ** 2).max()
    assert np.abs(ug - uo).max() <= 1e-5 * umax and np.abs(vg - vo).max() <= 1e-5 * umax
    assert rel(Pg, Po) < 1e-4
    assert np.all(np.abs(lg - lo) <= lam_bound32(f0, l0, prm, lo))
    assert rel(lg, lo) < 1e-4


# (name, cavities [(nx, ny, Re, n, theta)], library options)
LAYOUTS = [
    ("300x260 NT256 rows64 grid", [(300, 260, 1000.0, 0.75, 60.0)],
     dict(kernel="fused", fused_threads=256, fused_rows=64, schedule="grid")),
    ("300x260 NT256 rows128 dynamic", [(300, 260, 1000.0, 0.75, 60.0)],
     dict(kernel="fused", fused_threads=256, fused_rows=128, schedule="dynamic")),
    ("257^2 NT64 rows32 static", [(257, 257, 100.0, 1.25, 60.0)],
     dict(kernel="fused", fused_threads=64, fused_rows=32, schedule="static")),
    ("385^2 + 513^2 + 129^2 NT128 rows128 dynamic",
     [(385, 385, 400.0, 0.6, 30.0), (513, 513, 1000.0, 1.4, 75.0), (129, 129, 100.0, 1.0, 90.0)],
     dict(kernel="fused", fused_threads=128, fused_rows=128, schedule="dynamic")),
    ("385^2 + 513^2 NT64 rows128 dynamic",
     [(385, 385, 400.0, 0.6, 45.0), (513, 513, 1000.0, 1.4, 60.0)],
     dict(kernel="fused", fused_threads=64, fused_rows=128, schedule="dynamic")),
]


def _set_and_step(specs, opts, precision, seed0):
    runs, states = [], []
    s = solver([cav(*sp) for sp in specs], precision=precision, **opts)
    for k, sp in enumerate(specs):
        r = oracle_run(*sp)
        f0, l0 = synthetic_state(r, seed0 + 10 * k)
        s.set_state(k, f0, l0)
        runs.append(r)
        states.append((f0, l0))
    info = [s.info(k) for k in range(len(specs))]
    s.step(1)
    return s, runs, states, info


@pytest.mark.parametrize("name,specs,opts", LAYOUTS, ids=[l[0] for l in LAYOUTS])
def test_one_step_fp64_at_product_layouts(name, specs, opts):
    s, runs, states, info = _set_and_step(specs, opts, "fp64", 100)
    # the layout asked for is the one in use, with several tasks per cavity
    assert info[0].fused_threads == opts["fused_threads"] and info[0].fused_rows == opts["fused_rows"]
    assert info[0].ntasks >= 2 * len(specs)
    for k, (r, (f0, l0)) in enumerate(zip(runs, states)):
        fo, lo = O.step(f0, l0, r.g, r.prm)
        fg, lg = s.get_state(k)
        compare_state(fg, lg, fo, lo, lam_tol=lam_bound(f0, l0, r.prm, lo))
        # residual of Eq. (2.19) and kinetic energy of Eq. (5.1), per cavity
        res = s.residual()[k]
        Eu, EP, Rinf = O.global_relative_error(*O.macros(fo), *O.macros(f0))
        assert abs(res[0] - Eu) <= 1e-9 * Eu and abs(res[1] - EP) <= 1e-9 * EP
        assert abs(res[2] - Rinf) <= 1e-9 * Rinf
        Ek = O.kinetic_energy(*O.macros(fo)[:2], r.g)
        assert abs(res[3] - Ek) <= 1e-12 * Ek
    s.close()


@pytest.mark.parametrize("name,specs,opts", LAYOUTS, ids=[l[0] for l in LAYOUTS])
def test_one_step_fp32dev_at_product_layouts(name, specs, opts):
    s, runs, states, _ = _set_and_step(specs, opts, "fp32dev", 200)
    for k, (r, (f0, l0)) in enumerate(zip(runs, states)):
        fo, lo = O.step(f0, l0, r.g, r.prm)
        fg, lg = s.get_state(k)
        check_fp32(fg, lg, fo, lo, f0, l0, r.prm)
    s.close()


def test_staged_fp64_on_a_large_developed_cavity():
    """The FP64 default (staged kernels) on a 300 x 260 cavity the oracle
    developed from rest, one step."""
    r = oracle_run(300, 260, 1000.0, 0.75, 60.0)
    r.advance(12)
    f0, l0 = r.fhat.copy(), r.lam.copy()
    fo, lo = O.step(f0, l0, r.g, r.prm)
    s = solver([cav(300, 260, 1000.0, 0.75, 60.0)], kernel="staged")
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, fo, lo, lam_tol=lam_bound(f0, l0, r.prm, lo))
    s.close()

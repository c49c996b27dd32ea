"""The first-order wall-pressure reading (wall_pressure = "first") against the oracle.

The wall rule of Sec. 4 with P_b = 2 P_nb - P_nnb (the oracle's
Params.wall_pressure = 1), on the staged kernels: one FP64 step from states the
oracle developed with the same reading, at the 1e-12 bars; FP32 at its bars;
and a batch under kernel AUTO, which must pick the staged kernels.
"""
import numpy as np
import pytest

import oracle as O
from test_gpu_parity import cav, compare_state, lam_bound, rel, solver

pytestmark = pytest.mark.gpu

CASES = [(67, 45, 100.0, 0.75, 60.0, 30), (33, 29, 1000.0, 0.5, 45.0, 20),
         (9, 70, 100.0, 1.5, 75.0, 15), (5, 5, 100.0, 1.0, 90.0, 10)]


def developed(nx, ny, Re, n, th, k0):
    run = O.cavity_run(nx, Re, n, theta_deg=th, ny=ny, wall_pressure=1)
    run.advance(k0)
    return run


@pytest.mark.parametrize("nx,ny,Re,n,th,k0", CASES)
def test_one_step_fp64_first_order_wall_pressure(nx, ny, Re, n, th, k0):
    run = developed(nx, ny, Re, n, th, k0)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    fo, lo = O.step(f0, l0, run.g, run.prm)
    # the reading changes the result: the zeroth-order step differs
    prm0 = O.cavity_params(nx, ny, Re, n, grid=run.g)
    fz, _ = O.step(f0, l0, run.g, prm0)
    assert np.abs(fz - fo).max() > 1e-10
    s = solver([cav(nx, ny, Re, n, th)], kernel="staged", wall_pressure="first")
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, fo, lo, lam_tol=lam_bound(f0, l0, run.prm, lo))
    s.close()


def test_fp32_first_order_wall_pressure_and_auto_kernel():
    specs = [(67, 45, 100.0, 0.75, 60.0), (33, 29, 1000.0, 0.5, 45.0)]
    s = solver([cav(*sp) for sp in specs], precision="fp32dev", wall_pressure="first")
    from paper_2306_07603_gb300 import capi
    assert s.info(0).kernel == capi.IFDLBM_KERNEL_STAGED
    runs = []
    for k, sp in enumerate(specs):
        r = developed(*sp, 40)
        s.set_state(k, r.fhat, r.lam)
        runs.append(r)
    s.step(1)
    for k, r in enumerate(runs):
        fo, lo = O.step(r.fhat, r.lam, r.g, r.prm)
        fg, lg = s.get_state(k)
        ug, vg, Pg = O.macros(fg)
        uo, vo, Po = O.macros(fo)
        umax = np.sqrt(uo ** 2 + vo ** 2).max()
        assert np.abs(ug - uo).max() <= 1e-5 * umax and np.abs(vg - vo).max() <= 1e-5 * umax
        assert rel(Pg, Po) < 1e-4
    s.close()

"""GPU parity on general quadrilaterals (per-node metrics of the bilinear map):
ifdlbm_create_quad_batch against the oracle's quad_grid / quad_run.

* The trapezoid's own corners give the trapezoid handle's time step,
  Courant number and trajectory (to rounding of the metrics).
* One FP64 step from an oracle-developed state on skewed quadrilaterals
  (eta_x != 0, a lid that is not horizontal) matches the oracle to the
  1e-12 bars of the trapezoid parity tests, on the staged kernels, with the
  lagged and the implicit relaxation time; the Eq. (2.19) residuals and the
  kinetic energy of Eq. (5.1) (the Jacobian of the node) too.
* A batch of two different quadrilaterals, several steps from rest; the
  macroscopic fields with the stream function of the general map.
* FP32 deviation storage: one step within 1e-5 of the oracle.
* Eddy centres of a developed flow, located in (xi, eta) and mapped
  through the corners, equal the oracle finder's.
"""
import math

import numpy as np
import pytest

import oracle as O
from test_gpu_parity import compare_state, lam_bound, rel

pytestmark = pytest.mark.gpu

SKEW = ((0.1, -0.05), (1.3, 0.12), (-0.2, 0.9), (1.05, 1.1))
KITE = ((0.0, 0.0), (1.0, 0.3), (0.2, 1.0), (1.1, 1.4))


def _trapezoid_corners(theta=60.0, L=1.0, H=1.0):
    ct = 1.0 / math.tan(math.radians(theta))
    return ((H * ct, 0.0), (L + H * ct, 0.0), (0.0, H), (L + 2 * H * ct, H))


def quad_solver(specs, **kw):
    """specs: (nx, ny, corners, Re, n)."""
    from paper_2306_07603_gb300.solver import Solver, quad_cavity
    return Solver([quad_cavity(nx, ny, cr, Re, n) for nx, ny, cr, Re, n in specs], **kw)


def test_trapezoid_corners_equal_the_trapezoid_handle():
    from paper_2306_07603_gb300.solver import Solver, cavity
    a = quad_solver([(33, 29, _trapezoid_corners(), 400.0, 0.75)])
    b = Solver([cavity(33, 29, 400.0, 0.75, theta_deg=60.0)], kernel="staged")
    ia, ib = a.info(0), b.info(0)
    assert abs(ia.dt - ib.dt) <= 1e-15 * ib.dt
    assert abs(ia.courant_max - ib.courant_max) <= 1e-14 * ib.courant_max
    assert ia.kernel == ib.kernel
    a.step(20)
    b.step(20)
    fa, la = a.get_state(0)
    fb, lb = b.get_state(0)
    assert np.abs(fa - fb).max() <= 1e-13
    assert rel(la, lb) <= 1e-12


QCASES = [
    # nx, ny, corners, Re, n, developed steps
    (37, 29, SKEW, 400.0, 0.75, 30),
    (41, 33, KITE, 100.0, 1.5, 30),
    (70, 9, SKEW, 100.0, 0.5, 20),
    (5, 5, KITE, 100.0, 1.0, 10),
]


@pytest.mark.parametrize("lambda_mode", ["lagged", "implicit"])
@pytest.mark.parametrize("nx,ny,corners,Re,n,k0", QCASES)
def test_one_step_fp64_parity_on_a_quadrilateral(nx, ny, corners, Re, n, k0, lambda_mode):
    impl = lambda_mode == "implicit"
    run = O.quad_run(nx, ny, corners, Re, n, implicit_lambda=impl)
    run.advance(k0)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    fo, lo = O.step(f0, l0, run.g, run.prm)
    s = quad_solver([(nx, ny, corners, Re, n)], lambda_mode=lambda_mode)
    assert abs(s.info(0).dt - run.prm.dt) <= 1e-15 * run.prm.dt
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, fo, lo, lam_tol=lam_bound(f0, l0, run.prm, lo))
    r = s.residual()[0]
    ux0, uy0, P0 = O.macros(f0)
    ux1, uy1, P1 = O.macros(fo)
    Eu, EP, Rinf = O.global_relative_error(ux1, uy1, P1, ux0, uy0, P0)
    assert abs(r[0] - Eu) <= 1e-9 * Eu and abs(r[1] - EP) <= 1e-9 * EP
    assert abs(r[2] - Rinf) <= 1e-9 * Rinf
    Ek = O.kinetic_energy(ux1, uy1, run.g)
    assert abs(r[3] - Ek) <= 1e-12 * Ek


def test_batch_of_two_quadrilaterals_from_rest_with_fields():
    specs = [(37, 29, SKEW, 400.0, 0.75), (23, 31, KITE, 100.0, 1.25)]
    s = quad_solver(specs)
    steps = 40
    s.step(steps)
    for k, (nx, ny, cr, Re, n) in enumerate(specs):
        run = O.quad_run(nx, ny, cr, Re, n)
        run.advance(steps - 1)
        f_in, l_in = run.fhat.copy(), run.lam.copy()
        run.advance(1)
        fg, lg = s.get_state(k)
        compare_state(fg, lg, run.fhat, run.lam, lam_tol=lam_bound(f_in, l_in, run.prm, run.lam))
        m, d = s.macros(k), run.fields()
        for key in ("u", "v", "psi"):
            assert rel(m[key], d[key]) <= 1e-12, key
        P = (m["rho"] - 1.0) * (1.0 / 3.0)
        assert np.abs(P - d["P"]).max() <= 1e-12 * max(np.abs(d["P"]).max(), 1e-3)


FP32_KERNELS = {
    "staged": dict(kernel="staged"),
    "fused64x8": dict(kernel="fused", fused_threads=64, fused_rows=8),
    "fused128": dict(kernel="fused", fused_threads=128),
    "fused256x16": dict(kernel="fused", fused_threads=256, fused_rows=16),
}


@pytest.mark.parametrize("power_fp32", [False, True])
@pytest.mark.parametrize("kname", list(FP32_KERNELS))
@pytest.mark.parametrize("nx,ny,corners,Re,n", [(37, 29, SKEW, 400.0, 0.75),
                                                (70, 9, KITE, 100.0, 1.5)])
def test_fp32_deviation_one_step_error_on_a_quadrilateral(nx, ny, corners, Re, n, kname,
                                                         power_fp32):
    """FP32 deviation storage on a quadrilateral, staged and fused (the fused
    kernel's general variant: metrics of the bilinear map per node in FP32)."""
    run = O.quad_run(nx, ny, corners, Re, n)
    run.advance(200)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    fo, lo = O.step(f0, l0, run.g, run.prm)
    s = quad_solver([(nx, ny, corners, Re, n)], precision="fp32dev", power_fp32=power_fp32,
                    **FP32_KERNELS[kname])
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    ug, vg, Pg = O.macros(fg)
    uo, vo, Po = O.macros(fo)
    assert rel(ug, uo) < 1e-5 and rel(vg, vo) < 1e-5 and rel(Pg, Po) < 1e-4
    assert rel(lg, lo) < 1e-5
    r = s.residual()[0]
    Ek = O.kinetic_energy(*O.macros(fo)[:2], run.g)
    assert abs(r[3] - Ek) <= 1e-5 * Ek


def test_kernel_choice_for_quadrilaterals():
    from paper_2306_07603_gb300 import capi
    spec = [(17, 17, SKEW, 100.0, 0.75)]
    assert quad_solver(spec, precision="fp32dev").info(0).kernel == capi.IFDLBM_KERNEL_FUSED
    assert quad_solver(spec).info(0).kernel == capi.IFDLBM_KERNEL_STAGED            # FP64
    assert (quad_solver(spec, precision="fp32dev", lambda_mode="implicit").info(0).kernel
            == capi.IFDLBM_KERNEL_STAGED)


def test_fused_fp32_tracks_staged_fp32_over_many_steps():
    """A batch of three quadrilaterals (ragged tails, a 9-row grid) from an
    oracle state, 300 steps in FP32 on the fused and on the staged kernels:
    the two FP32 trajectories stay within FP32 rounding of each other."""
    specs = [(37, 29, SKEW, 400.0, 0.75), (41, 33, KITE, 100.0, 1.5), (70, 9, SKEW, 100.0, 0.5)]
    runs = []
    for nx, ny, cr, Re, n in specs:
        r = O.quad_run(nx, ny, cr, Re, n)
        r.advance(40)
        runs.append(r)
    out = {}
    for kname in ("staged", "fused64x8"):
        s = quad_solver(specs, precision="fp32dev", **FP32_KERNELS[kname])
        for k, r in enumerate(runs):
            s.set_state(k, r.fhat, r.lam)
        s.step(300)
        out[kname] = [s.macros(k) for k in range(len(specs))]
        s.close()
    for k in range(len(specs)):
        a, b = out["staged"][k], out["fused64x8"][k]
        umax = np.sqrt(a["u"] ** 2 + a["v"] ** 2).max()
        for key in ("u", "v"):
            assert np.abs(a[key] - b[key]).max() <= 1e-5 * umax, (k, key)
        assert rel(b["psi"], a["psi"]) <= 1e-5, k


def test_trapezoid_corners_fused_fp32_equal_the_trapezoid_handle():
    from paper_2306_07603_gb300.solver import Solver, cavity
    a = quad_solver([(65, 49, _trapezoid_corners(), 400.0, 0.75)], precision="fp32dev",
                    kernel="fused", fused_threads=128)
    b = Solver([cavity(65, 49, 400.0, 0.75, theta_deg=60.0)], precision="fp32dev",
               kernel="fused", fused_threads=128)
    a.step(100)
    b.step(100)
    ma, mb = a.macros(0), b.macros(0)
    umax = np.sqrt(mb["u"] ** 2 + mb["v"] ** 2).max()
    for key in ("u", "v"):
        assert np.abs(ma[key] - mb[key]).max() <= 1e-5 * umax, key


def test_eddies_of_a_developed_flow_are_mapped_through_the_corners():
    nx = ny = 33
    run = O.quad_run(nx, ny, SKEW, 100.0, 0.75)
    run.advance(1500)
    s = quad_solver([(nx, ny, SKEW, 100.0, 0.75)])
    s.set_state(0, run.fhat, run.lam)
    lib = s.eddies(0)
    orc = O.eddy_centres(run.fields()["psi"], 1.0, 1.0, 90.0)   # unit square: x = xi, y = eta
    assert orc[0] is not None and lib[0].found
    for a, b in zip(lib, orc):
        assert bool(a.found) == (b is not None)
        if b is None:
            continue
        assert (a.i, a.j) == (b["i"], b["j"])
        assert abs(a.xi - b["xi"]) <= 1e-9 and abs(a.eta - b["eta"]) <= 1e-9
        x, y = O.quad_xy(b["xi"], b["eta"], SKEW)
        assert abs(a.x - x) <= 1e-9 and abs(a.y - y) <= 1e-9


def test_adjoint_rejects_a_quadrilateral_handle():
    import torch

    from paper_2306_07603_gb300 import capi
    s = quad_solver([(17, 17, SKEW, 100.0, 0.75)])
    buf = torch.zeros(capi.ifdlbm_state_bytes(s.h) // 8, dtype=torch.float64, device="cuda")
    dp = torch.zeros(3, dtype=torch.float64, device="cuda")
    capi.ifdlbm_save_state_dev(s.h, buf)
    with pytest.raises(capi.IfdlbmError) as e:
        capi.ifdlbm_adjoint_seed_energy(s.h, buf, torch.zeros_like(buf), dp)
    assert e.value.code == capi.IFDLBM_ERR_INVALID_ARG
    s.close()

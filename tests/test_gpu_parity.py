"""GPU parity: the sm_103a library (through its C ABI) against the FP64 oracle.

FP64 bar: max|gpu - oracle| / max|oracle| <= 1e-12 per field (each f-hat
plane, lambda, u, v, P), on grids that span several 32x8 tiles with ragged
tails, edge cases (5x5, theta = 90 and 30 deg, n = 1) and batches of
uneven cavities. Inputs are oracle states (rest, or developed by the
oracle); no expected value comes from the GPU.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def solver(cavs, **kw):
    from paper_2306_07603_gb300.solver import Solver
    return Solver(cavs, **kw)


def cav(nx, ny, Re, n, th, U=0.1, L=1.0, H=1.0):
    from paper_2306_07603_gb300.solver import cavity
    return cavity(nx, ny, Re, n, theta_deg=th, U_lid=U, L=L, H=H)


def oracle_run(nx, ny, Re, n, th, U=0.1, L=1.0, H=1.0, eta_b=0.5):
    return O.cavity_run(nx, Re, n, theta_deg=th, U=U, L=L, H=H, ny=ny, eta_b=eta_b)


def lam_bound(f_in, lam_in, prm, lam_out):
    """Pointwise bound on |lam_gpu - lam_oracle| after a step from (f_in, lam_in).

    The strain rate of Eqs. (2.12)-(2.13) is formed from f - f^eq, a
    difference of O(w_i) numbers, so in FP64 its absolute rounding is about
    eps * max|f|; through Eq. (1.4) lam = K |gamma-dot|^(n-1) / c_s^2 takes a
    relative error |n - 1| * delta(gamma-dot) / gamma-dot with
    delta(gamma-dot) ~ sum |c c| delta(f^ne) / (lam_prev c_s^2). Near the
    zero-shear clamp this exceeds 1e-12 on either side; elsewhere the 1e-12
    relative bar applies."""
    ux, uy, P = O.macros(f_in)
    feq = O.equilibrium(P, ux, uy)
    f = O.f_from_fhat(f_in, feq, lam_in, prm.dt)
    gd = O.shear_rate(*O.strain_rate(f, feq, lam_in))
    cs2 = prm.c ** 2 / 3.0
    dfne = 16.0 * np.finfo(float).eps * np.abs(f_in).max()
    cond = abs(prm.n - 1.0) * lam_out * dfne / (lam_in * cs2 * np.maximum(gd, prm.gamma_min))
    return TOL64 * np.abs(lam_out).max() + cond


def p_scale(fo, c=1.0):
    """Magnitude of the terms Eq. (2.11) forms P from: c_s^2/|wbar_0| max sum_{i>0} |f_i|.
    P is a small difference of O(w_i) numbers, so its rounding is relative to this."""
    return (c * c / 3.0) / abs(O.OMEGA_BAR[0]) * np.abs(fo[1:]).sum(axis=0).max()


def compare_state(fg, lg, fo, lo, tol=TOL64, lam_tol=None):
    """f-hat planes to `tol` relative (max-norm); u and v to `tol` of the
    largest velocity magnitude (they are components of one vector, formed
    from the same populations, so a component much smaller than the other has
    no relative accuracy of its own); P to `tol` of the magnitude of its
    Eq. (2.11) terms; lambda pointwise to `lam_tol` (an array from lam_bound)
    or to `tol` relative."""
    for q in range(9):
        assert rel(fg[q], fo[q]) <= tol, (q, rel(fg[q], fo[q]))
    ug, vg, Pg = O.macros(fg)
    uo, vo, Po = O.macros(fo)
    umax = max(np.sqrt(uo ** 2 + vo ** 2).max(), 1e-300)
    du, dv = np.abs(ug - uo).max() / umax, np.abs(vg - vo).max() / umax
    assert du <= tol and dv <= tol, (du, dv)
    assert np.abs(Pg - Po).max() <= tol * p_scale(fo), np.abs(Pg - Po).max() / p_scale(fo)
    if lam_tol is None:
        assert rel(lg, lo) <= tol, rel(lg, lo)
    else:
        assert np.all(np.abs(lg - lo) <= lam_tol), np.max(np.abs(lg - lo) / lam_tol)


CASES = [
    # nx, ny, Re, n, theta, developed steps
    (67, 45, 100.0, 0.75, 60.0, 40),
    (33, 29, 1000.0, 0.5, 45.0, 30),
    (41, 37, 400.0, 1.5, 75.0, 30),
    (37, 35, 100.0, 1.0, 90.0, 30),
    (35, 33, 100.0, 1.25, 30.0, 30),
    (5, 5, 100.0, 0.75, 60.0, 10),
    (9, 70, 100.0, 0.75, 60.0, 20),
    (70, 9, 100.0, 0.75, 60.0, 20),
]


# kernel organisations: staged; fused with several CTA widths and row segments
# (small segments put task boundaries inside the grid)
KERNELS = {
    "staged": dict(kernel="staged"),
    "fused64x8": dict(kernel="fused", fused_threads=64, fused_rows=8),
    "fused128": dict(kernel="fused", fused_threads=128),
    "fused256x16": dict(kernel="fused", fused_threads=256, fused_rows=16),
}


@pytest.mark.parametrize("kname", list(KERNELS))
@pytest.mark.parametrize("nx,ny,Re,n,th,k0", CASES)
def test_one_step_fp64_parity(nx, ny, Re, n, th, k0, kname):
    run = oracle_run(nx, ny, Re, n, th)
    run.advance(k0)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    fo, lo = O.step(f0, l0, run.g, run.prm)
    s = solver([cav(nx, ny, Re, n, th)], **KERNELS[kname])
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, fo, lo, lam_tol=lam_bound(f0, l0, run.prm, lo))
    # residuals of Eq. (2.19) and the kinetic energy of Eq. (5.1)
    r = s.residual()[0]
    ux0, uy0, P0 = O.macros(f0)
    ux1, uy1, P1 = O.macros(fo)
    Eu, EP, Rinf = O.global_relative_error(ux1, uy1, P1, ux0, uy0, P0)
    assert abs(r[0] - Eu) <= 1e-9 * Eu and abs(r[1] - EP) <= 1e-9 * EP
    assert abs(r[2] - Rinf) <= 1e-9 * Rinf
    Ek = O.kinetic_energy(ux1, uy1, run.g)
    assert abs(r[3] - Ek) <= 1e-12 * Ek


def test_rest_start_matches_oracle_initial_state():
    run = oracle_run(33, 29, 100.0, 0.75, 60.0)
    s = solver([cav(33, 29, 100.0, 0.75, 60.0)])
    fg, lg = s.get_state(0)
    compare_state(fg, lg, run.fhat, run.lam, tol=1e-15)


@pytest.mark.parametrize("kname", ["staged", "fused64x8"])
def test_config1_4000_steps_fields_and_residual_history(kname):
    """65^2, theta = 60 deg, n = 0.75, Re = 100, 4000 steps from rest:
    rho, u, v, psi and the residual every 500 steps."""
    run = oracle_run(65, 65, 100.0, 0.75, 60.0)
    s = solver([cav(65, 65, 100.0, 0.75, 60.0)], **KERNELS[kname])
    for k in range(8):
        run.advance(499)
        f_in, l_in = run.fhat.copy(), run.lam.copy()
        run.advance(1, record=True)
        s.step(500)
        r = s.residual()[0]
        Eu, EP, Rinf = run.history[-1]
        assert abs(r[0] - Eu) <= 1e-6 * Eu, (r[0], Eu)
        assert abs(r[1] - EP) <= 1e-6 * EP, (r[1], EP)
        assert abs(r[2] - Rinf) <= 1e-6 * Rinf, (r[2], Rinf)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, run.fhat, run.lam, lam_tol=lam_bound(f_in, l_in, run.prm, run.lam))
    mg = s.macros(0)
    mo = run.fields()
    for k in ("rho", "u", "v", "psi"):
        assert np.abs(mg[k] - mo[k]).max() <= TOL64 * np.abs(mo[k]).max(), k


@pytest.mark.parametrize("kname", list(KERNELS))
def test_batch_of_uneven_cavities_matches_each_oracle(kname):
    specs = [(67, 45, 100.0, 0.75, 60.0), (33, 29, 1000.0, 0.5, 45.0), (41, 57, 400.0, 1.5, 75.0),
             (5, 5, 100.0, 1.0, 90.0)]
    s = solver([cav(*sp) for sp in specs], **KERNELS[kname])
    runs = []
    for k, sp in enumerate(specs):
        r = oracle_run(*sp)
        r.advance(15)
        s.set_state(k, r.fhat, r.lam)
        runs.append(r)
    s.step(7)
    for k, r in enumerate(runs):
        r.advance(6)
        f_in, l_in = r.fhat.copy(), r.lam.copy()
        r.advance(1)
        fg, lg = s.get_state(k)
        compare_state(fg, lg, r.fhat, r.lam, lam_tol=lam_bound(f_in, l_in, r.prm, r.lam))


def test_graph_chunks_equal_eager_steps():
    """Steps replayed from captured CUDA graphs give the oracle's result too
    (graph_chunk = 4 over 21 steps: 5 graph replays + eager remainder)."""
    run = oracle_run(34, 30, 400.0, 0.75, 60.0)
    s = solver([cav(34, 30, 400.0, 0.75, 60.0)], graph_chunk=4)
    s.step(21)
    run.advance(20)
    f_in, l_in = run.fhat.copy(), run.lam.copy()
    run.advance(1)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, run.fhat, run.lam, lam_tol=lam_bound(f_in, l_in, run.prm, run.lam))


def test_eta_b_and_dt_options_reach_the_kernel():
    run = O.cavity_run(33, 100.0, 0.75, theta_deg=60.0, eta_b=0.9, dt=0.01)
    s = solver([cav(33, 33, 100.0, 0.75, 60.0)], eta_b=0.9, dt=0.01)
    run.advance(11)
    f_in, l_in = run.fhat.copy(), run.lam.copy()
    run.advance(1)
    s.step(12)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, run.fhat, run.lam, lam_tol=lam_bound(f_in, l_in, run.prm, run.lam))


@pytest.mark.parametrize("power_fp32", [False, True])
@pytest.mark.parametrize("kname", list(KERNELS))
def test_fp32_deviation_one_step_error(kname, power_fp32):
    """FP32 deviation storage: one step from an oracle state stays within
    1e-5 relative of the FP64 oracle on every field (FP64 power law, and the
    FP32-power opt-in)."""
    run = oracle_run(67, 45, 100.0, 0.75, 60.0)
    run.advance(200)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    fo, lo = O.step(f0, l0, run.g, run.prm)
    s = solver([cav(67, 45, 100.0, 0.75, 60.0)], precision="fp32dev", power_fp32=power_fp32,
               **KERNELS[kname])
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    ug, vg, Pg = O.macros(fg)
    uo, vo, Po = O.macros(fo)
    assert rel(ug, uo) < 1e-5 and rel(vg, vo) < 1e-5 and rel(Pg, Po) < 1e-4
    assert rel(lg, lo) < 1e-5


def test_divergence_is_reported_not_hidden():
    """A state with a non-finite population makes the next synchronising call
    return IFDLBM_ERR_DIVERGED (the status word, no device fault)."""
    from paper_2306_07603_gb300 import capi
    run = oracle_run(17, 17, 100.0, 0.75, 60.0)
    f = run.fhat.copy()
    f[1, 8, 8] = np.inf
    s = solver([cav(17, 17, 100.0, 0.75, 60.0)])
    s.set_state(0, f, run.lam)
    s.step(2)
    with pytest.raises(capi.IfdlbmError) as e:
        s.residual()
    assert e.value.code == capi.IFDLBM_ERR_DIVERGED


def test_async_residual_read_equals_the_synchronous_one():
    """ifdlbm_batch_residual_async: the residuals and the divergence word land
    in page-locked host memory once the stream reaches the copy."""
    import torch

    from paper_2306_07603_gb300 import capi
    s = solver([cav(33, 29, 400.0, 0.75, 60.0), cav(17, 21, 100.0, 1.5, 75.0)], kernel="fused")
    res = torch.full((2, 4), np.nan, dtype=torch.float64, pin_memory=True)
    st = torch.full((1,), 7, dtype=torch.int32, pin_memory=True)
    s.step(5)
    capi.ifdlbm_batch_residual_async(s.h, res, st)
    ev = torch.cuda.Event()
    ev.record(s.stream)
    ev.synchronize()
    assert int(st[0]) == 0
    assert np.array_equal(res.numpy(), s.residual())
    # a non-finite state sets bit 0 of the word
    run = oracle_run(17, 21, 100.0, 1.5, 75.0)
    f = run.fhat.copy()
    f[2, 9, 9] = np.nan
    s.set_state(1, f, run.lam)
    s.step(1)
    capi.ifdlbm_batch_residual_async(s.h, res, st)
    ev.record(s.stream)
    ev.synchronize()
    assert int(st[0]) & 1
    with pytest.raises(capi.IfdlbmError):
        s.sync()
    s.close()


@pytest.mark.parametrize("schedule", ["grid", "static", "dynamic"])
def test_fused_schedules_match_oracle_on_uneven_batch(schedule):
    """Persistent schedules (static largest-first, dynamic atomic counter) give
    every cavity of an uneven batch the oracle's step (FP64 fused kernel)."""
    specs = [(67, 45, 100.0, 0.75, 60.0), (33, 29, 1000.0, 0.5, 45.0), (41, 57, 400.0, 1.5, 75.0),
             (9, 70, 100.0, 1.0, 90.0), (70, 9, 100.0, 1.25, 30.0)]
    s = solver([cav(*sp) for sp in specs], kernel="fused", fused_threads=64, fused_rows=16,
               schedule=schedule)
    runs = []
    for k, sp in enumerate(specs):
        r = oracle_run(*sp)
        r.advance(12)
        s.set_state(k, r.fhat, r.lam)
        runs.append(r)
    s.step(3)
    for k, r in enumerate(runs):
        r.advance(2)
        f_in, l_in = r.fhat.copy(), r.lam.copy()
        r.advance(1)
        fg, lg = s.get_state(k)
        compare_state(fg, lg, r.fhat, r.lam, lam_tol=lam_bound(f_in, l_in, r.prm, r.lam))


def test_autotune_keeps_state_and_result():
    """The autotuner times layouts from a saved state and restores it: the
    state is unchanged and later steps still equal the oracle's."""
    specs = [(67, 45, 100.0, 0.75, 60.0), (41, 57, 400.0, 1.5, 75.0)]
    s = solver([cav(*sp) for sp in specs], kernel="fused")
    runs = []
    for k, sp in enumerate(specs):
        r = oracle_run(*sp)
        r.advance(10)
        s.set_state(k, r.fhat, r.lam)
        runs.append(r)
    before = [s.get_state(k) for k in range(2)]
    t = s.autotune(trial_steps=2)
    assert t.candidates == 45 and t.fused_threads in (64, 128, 256) and t.schedule in (0, 1, 2)
    info = s.info(0)
    assert (info.fused_threads, info.fused_rows, info.schedule) == (t.fused_threads, t.fused_rows,
                                                                     t.schedule)
    for k in range(2):
        f, l = s.get_state(k)
        assert np.array_equal(f, before[k][0]) and np.array_equal(l, before[k][1])
    s.step(2)
    for k, r in enumerate(runs):
        r.advance(1)
        f_in, l_in = r.fhat.copy(), r.lam.copy()
        r.advance(1)
        fg, lg = s.get_state(k)
        compare_state(fg, lg, r.fhat, r.lam, lam_tol=lam_bound(f_in, l_in, r.prm, r.lam))


@pytest.mark.parametrize("kname", ["staged", "fused64x8"])
def test_contravariant_time_step_theta30(kname):
    """dt_mode 'contravariant' (dt = CFL min(dxi/max|c_xi|, deta/max|c_eta|)) gives
    the oracle's dt and step at theta = 30 deg, where the default rule is unstable."""
    from paper_2306_07603_gb300 import capi
    nx, ny = 41, 37
    run = O.cavity_run(nx, 400.0, 0.75, theta_deg=30.0, ny=ny, dt_mode="contravariant")
    s = solver([cav(nx, ny, 400.0, 0.75, 30.0)], dt_mode="contravariant", **KERNELS[kname])
    assert abs(capi.ifdlbm_info(s.h, 0).dt - run.prm.dt) <= 1e-15 * run.prm.dt
    run.advance(30)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    s.set_state(0, f0, l0)
    s.step(1)
    fo, lo = O.step(f0, l0, run.g, run.prm)
    fg, lg = s.get_state(0)
    compare_state(fg, lg, fo, lo, lam_tol=lam_bound(f0, l0, run.prm, lo))


def test_fp32_rebasing_keeps_the_state():
    """FP32 storage re-bases its deviations on the mean pressure every 1024
    steps (the state f-hat is unchanged but for one FP32 rounding of g): the
    exported f-hat, rho and the save/load round trip all carry the reference
    pressure. Checked across a re-basing against an FP32 handle whose
    re-basing has not happened yet (same steps, set to the same state)."""
    import torch

    from paper_2306_07603_gb300 import capi
    run = oracle_run(41, 37, 100.0, 0.75, 60.0)
    run.advance(300)
    s = solver([cav(41, 37, 100.0, 0.75, 60.0)], precision="fp32dev", graph_chunk=0)
    s.set_state(0, run.fhat, run.lam)
    s.step(1030)                        # one re-basing after step 1024
    f1, l1 = s.get_state(0)
    m = s.macros(0)
    # rho of the ABI and the pressure of the exported f-hat (Eq. 2.11) agree
    _, _, P = O.macros(f1)
    assert np.abs(m["rho"] - (1.0 + 3.0 * P)).max() <= 1e-6 * np.abs(P).max()
    # a fresh FP32 handle set to the exported state continues identically to
    # FP32 rounding of the state
    t = solver([cav(41, 37, 100.0, 0.75, 60.0)], precision="fp32dev", graph_chunk=0)
    t.set_state(0, f1, l1)
    s.step(20)
    t.step(20)
    fa, _ = s.get_state(0)
    fb, _ = t.get_state(0)
    assert np.abs(fa - fb).max() <= 1e-6
    # save / load carries the reference pressure
    buf = torch.empty(capi.ifdlbm_state_bytes(s.h) // 8, dtype=torch.float64, device="cuda")
    capi.ifdlbm_save_state_dev(s.h, buf)
    s.step(2000)                         # two more re-basings
    capi.ifdlbm_load_state_dev(s.h, buf)
    fc, _ = s.get_state(0)
    assert np.array_equal(fc, fa)
    s.close()
    t.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_probes_and_device_residual_match_the_host_outputs(precision):
    """ifdlbm_probe_dev gives u, v and P of ifdlbm_macros at the probe nodes
    (NaN outside the cavity); ifdlbm_residual_dev copies the residual array."""
    import torch

    from paper_2306_07603_gb300 import capi
    specs = [(41, 37, 400.0, 0.75, 60.0), (33, 29, 100.0, 1.5, 45.0)]
    s = solver([cav(*sp) for sp in specs], precision=precision)
    s.step(1500)                       # FP32: past one re-basing of the pressure reference
    probes = [(0, 20, 18), (0, 0, 36), (1, 32, 0), (1, 7, 11), (1, 33, 5), (2, 1, 1)]
    idx = torch.tensor(probes, dtype=torch.int32, device="cuda")
    out = torch.zeros((len(probes), 3), dtype=torch.float64, device="cuda")
    res = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    capi.ifdlbm_probe_dev(s.h, idx, out)
    capi.ifdlbm_residual_dev(s.h, res)
    s.sync()
    out, res = out.cpu().numpy(), res.cpu().numpy()
    m = [s.macros(k) for k in range(2)]
    for k, (c, i, j) in enumerate(probes):
        if c > 1 or i >= specs[c][0] or j >= specs[c][1]:
            assert np.all(np.isnan(out[k]))
            continue
        assert out[k, 0] == m[c]["u"][j, i] and out[k, 1] == m[c]["v"][j, i]
        assert abs(1.0 + 3.0 * out[k, 2] - m[c]["rho"][j, i]) <= 1e-15
    assert np.array_equal(res, np.array(s.residual()))
    s.close()


IMPLICIT_CASES = [(67, 45, 100.0, 0.75, 60.0, 40), (33, 29, 1000.0, 0.5, 45.0, 30),
                  (41, 37, 400.0, 1.5, 75.0, 30), (35, 33, 100.0, 1.0, 30.0, 30)]


@pytest.mark.parametrize("kname", ["staged", "fused64x8", "fused256x16"])
@pytest.mark.parametrize("nx,ny,Re,n,th,k0", IMPLICIT_CASES)
def test_implicit_lambda_one_step_fp64_parity(nx, ny, Re, n, th, k0, kname):
    """lambda_mode 'implicit' (Eq. 2.14 at the current lambda; the oracle
    bisects, the library runs a bracketed Newton iteration): one step from an
    oracle state. lambda is held pointwise to 1e-12 max|lambda| plus
    |n - 1| lambda da / a, da = 32 eps max|f-hat| / c_s^2 the rounding of a
    (it is formed from f-hat - f^eq, a difference of O(w_i) numbers)."""
    run = oracle_run(nx, ny, Re, n, th)
    run.advance(k0)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    prm = O.cavity_params(nx, ny, Re, n, grid=run.g, implicit_lambda=True)
    fo, lo = O.step(f0, l0, run.g, prm)
    s = solver([cav(nx, ny, Re, n, th)], lambda_mode="implicit", **KERNELS[kname])
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    ux, uy, P = O.macros(f0)
    feq = O.equilibrium(P, ux, uy)
    d = f0 - feq
    pxx = (O.EX[:, None, None] ** 2 * d).sum(0)
    pxy = (O.EX[:, None, None] * O.EY[:, None, None] * d).sum(0)
    pyy = (O.EY[:, None, None] ** 2 * d).sum(0)
    a = 6.0 * np.sqrt(0.5 * (pxx ** 2 + 2 * pxy ** 2 + pyy ** 2))
    da = 32 * np.finfo(float).eps * np.abs(f0).max() * 3.0
    lam_tol = TOL64 * np.abs(lo).max() + abs(n - 1.0) * lo * da / np.maximum(a, 1e-300)
    compare_state(fg, lg, fo, lo, lam_tol=lam_tol)


@pytest.mark.parametrize("power_fp32", [False, True])
@pytest.mark.parametrize("kname", ["staged", "fused64x8", "fused128"])
@pytest.mark.parametrize("nx,ny,Re,n,th", [(67, 45, 100.0, 0.75, 60.0), (41, 37, 400.0, 1.5, 75.0)])
def test_implicit_lambda_fp32_one_step_error(nx, ny, Re, n, th, kname, power_fp32):
    """FP32 form: the implicit relaxation time (solved in FP64, or in FP32
    with the FP32-power opt-in), one step within the FP32 bars of the FP64
    oracle."""
    run = oracle_run(nx, ny, Re, n, th)
    run.advance(200)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    prm = O.cavity_params(nx, ny, Re, n, grid=run.g, implicit_lambda=True)
    fo, lo = O.step(f0, l0, run.g, prm)
    s = solver([cav(nx, ny, Re, n, th)], precision="fp32dev", lambda_mode="implicit",
               power_fp32=power_fp32, **KERNELS[kname])
    s.set_state(0, f0, l0)
    s.step(1)
    fg, lg = s.get_state(0)
    ug, vg, Pg = O.macros(fg)
    uo, vo, Po = O.macros(fo)
    assert rel(ug, uo) < 1e-5 and rel(vg, vo) < 1e-5 and rel(Pg, Po) < 1e-4
    assert rel(lg, lo) < 1e-5


def test_adjoint_rejects_the_implicit_form():
    import torch

    from paper_2306_07603_gb300 import capi
    s = solver([cav(17, 17, 100.0, 0.75, 60.0)], precision="fp64", kernel="staged",
               lambda_mode="implicit")
    buf = torch.zeros(capi.ifdlbm_state_bytes(s.h) // 8, dtype=torch.float64, device="cuda")
    dp = torch.zeros(3, dtype=torch.float64, device="cuda")
    capi.ifdlbm_save_state_dev(s.h, buf)
    with pytest.raises(capi.IfdlbmError):
        capi.ifdlbm_adjoint_seed_energy(s.h, buf, torch.zeros_like(buf), dp)
    s.close()

"""GPU adjoint (ifdlbm_adjoint_step) against independent derivatives.

* one reverse step: <w, J v> = <J^T w, v> with J v from central differences
  of the GPU forward step (the state Jacobian part);
* d E(T)/d(n, Re, theta) through KineticEnergy.backward against central
  differences of the GPU forward and against the oracle's complex-step
  gradient (exact derivative of the oracle's discrete map);
* the config-size case (257^2, theta = 60, n = 0.75, Re = 400, 2000 steps,
  checkpoints every 100) against central differences.
Spec tolerance for the gradient: 1e-4 relative.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def _dev_state(s, fhat, lam):
    """Library (opaque-layout) device state holding (fhat, lam)."""
    import torch

    from paper_2306_07603_gb300 import capi
    s.set_state(0, fhat, lam)
    buf = torch.empty(capi.ifdlbm_state_bytes(s.h) // 8, dtype=torch.float64, device="cuda")
    capi.ifdlbm_save_state_dev(s.h, buf)
    s.sync()
    return buf


@pytest.mark.parametrize("n", [1.0, 0.75, 1.5])
def test_adjoint_step_dot_product(n):
    """<w, J v> = <J^T w, v> for one step from an oracle-developed state.
    lambda(t) is a pointwise function of a node's own state, with a kink at
    the zero-shear clamp; the perturbation v is kept off the nodes whose
    shear rate is within a factor 10 of the clamp, so that no difference
    straddles it. For n != 1 the strain rate is formed from f^ne, which is
    ~1e-7 at weakly sheared nodes, so the central difference uses a
    perturbation of ~1e-9 (well inside the linear range; FP64 roundoff of the
    difference stays ~1e-9 relative)."""
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import Solver, cavity
    from paper_2306_07603_gb300.workloads import smooth_noise

    nx, ny = 33, 29
    run = O.cavity_run(nx, 400.0, n, theta_deg=60.0, ny=ny, dt_mode="grid")
    run.advance(60)
    f0, l0 = run.fhat.copy(), run.lam.copy()
    ux, uy, P = O.macros(f0)
    feq = O.equilibrium(P, ux, uy)
    gd = O.shear_rate(*O.strain_rate(O.f_from_fhat(f0, feq, l0, run.prm.dt), feq, l0))
    away = gd > 10.0 * run.prm.gamma_min
    s = Solver([cavity(nx, ny, 400.0, n, theta_deg=60.0)], precision="fp64", kernel="staged",
               dt_mode="grid")
    vf = smooth_noise((9, ny, nx), seed=1) * 1e-3 * away[None]
    vl = smooth_noise((ny, nx), seed=2) * 1e-2 * l0 * away
    wf = smooth_noise((9, ny, nx), seed=3)
    wl = smooth_noise((ny, nx), seed=4)
    w_rest = O.OMEGA[:, None, None]          # set_state stores fhat - w_i rho0
    W = _dev_state(s, wf + w_rest, wl)
    V = _dev_state(s, vf + w_rest, vl)

    def forward(fh, lm):
        _dev_state(s, fh, lm)
        s.step(1)
        out = torch.empty_like(W)
        capi.ifdlbm_save_state_dev(s.h, out)
        s.sync()
        return out

    eps = 1e-3 if n == 1.0 else 1e-6
    Jv = (forward(f0 + eps * vf, l0 + eps * vl) - forward(f0 - eps * vf, l0 - eps * vl)) / (2 * eps)
    S0 = _dev_state(s, f0, l0)
    adj = W.clone()
    dparams = torch.zeros(3, dtype=torch.float64, device="cuda")
    capi.ifdlbm_adjoint_step(s.h, S0, adj, dparams)
    s.sync()
    lhs = float(torch.dot(W, Jv))
    rhs = float(torch.dot(adj, V))
    assert abs(lhs - rhs) <= (1e-9 if n == 1.0 else 1e-6) * abs(lhs), (lhs, rhs)


def _gpu_energy(n, Re, th, nx, ny, T):
    from paper_2306_07603_gb300.solver import Solver, cavity
    s = Solver([cavity(nx, ny, Re, n, theta_deg=th)], precision="fp64", kernel="staged",
               dt_mode="grid")
    s.step(T)
    e = float(s.residual()[0][3])
    s.close()
    return e


@pytest.mark.parametrize("every", [1, 7, 40])
def test_energy_gradient_matches_central_differences(every):
    from paper_2306_07603_gb300.adjoint import energy_and_gradient
    x = [0.75, 400.0, 60.0]
    nx, ny, T = 33, 29, 40
    J, *g = energy_and_gradient(*x, nx, ny, T, every=every)
    assert abs(J - _gpu_energy(*x, nx, ny, T)) <= 1e-14 * J
    for k in range(3):
        h = 1e-6 * abs(x[k])
        xp, xm = list(x), list(x)
        xp[k] += h
        xm[k] -= h
        fd = (_gpu_energy(*xp, nx, ny, T) - _gpu_energy(*xm, nx, ny, T)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * abs(g[k]), (k, g[k], fd)


def test_energy_gradient_matches_oracle_complex_step():
    from paper_2306_07603_gb300.adjoint import energy_and_gradient

    def energy(n, Re, theta):
        run = O.cavity_run(33, Re, n, theta_deg=theta, dt_mode="grid")
        run.advance(40)
        ux, uy, _ = O.macros(run.fhat)
        return O.kinetic_energy(ux, uy, run.g)

    x = [0.75, 400.0, 60.0]
    J, *g = energy_and_gradient(*x, 33, 33, 40, every=10)
    for k in range(3):
        xs = [complex(v) for v in x]
        xs[k] += 1e-30j
        ref = np.imag(energy(*xs)) / 1e-30
        assert abs(g[k] - ref) <= 1e-8 * abs(ref), (k, g[k], ref)


def test_config5_gradient_against_central_differences():
    """257^2, theta = 60 deg, n = 0.75, Re = 400, FP64, 2000 steps from rest,
    checkpoints every 100 steps (the adjoint configuration)."""
    from paper_2306_07603_gb300.adjoint import energy_and_gradient
    x = [0.75, 400.0, 60.0]
    J, *g = energy_and_gradient(*x, 257, 257, 2000, every=100)
    for k in range(3):
        h = 1e-6 * abs(x[k])
        xp, xm = list(x), list(x)
        xp[k] += h
        xm[k] -= h
        fd = (_gpu_energy(*xp, 257, 257, 2000) - _gpu_energy(*xm, 257, 257, 2000)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-4 * abs(g[k]), (k, g[k], fd)


def _gpu_psimin(n, Re, th, nx, ny, T):
    """min over interior nodes of psi after T steps (the library's forward run)."""
    from paper_2306_07603_gb300.solver import Solver, cavity
    s = Solver([cavity(nx, ny, Re, n, theta_deg=th)], precision="fp64", kernel="staged",
               dt_mode="grid")
    s.step(T)
    psi = s.macros(0)["psi"]
    s.close()
    return float(psi[1:-1, 1:-1].min())


@pytest.mark.parametrize("every", [1, 7, 40])
def test_psi_min_gradient_matches_central_differences(every):
    from paper_2306_07603_gb300.adjoint import objective_and_gradient
    x = [0.75, 400.0, 60.0]
    nx, ny, T = 33, 29, 40
    J, *g = objective_and_gradient("psi_min", *x, nx, ny, T, every=every)
    assert J < 0 and abs(J - _gpu_psimin(*x, nx, ny, T)) <= 1e-14 * abs(J)
    for k in range(3):
        h = 1e-6 * abs(x[k])
        xp, xm = list(x), list(x)
        xp[k] += h
        xm[k] -= h
        fd = (_gpu_psimin(*xp, nx, ny, T) - _gpu_psimin(*xm, nx, ny, T)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * abs(g[k]), (k, g[k], fd)


def test_psi_min_gradient_matches_oracle_complex_step():
    """psi at the primary eddy's node, complex-step differentiated through the
    oracle (the node is chosen on the real parts)."""
    from paper_2306_07603_gb300.adjoint import objective_and_gradient

    def psi_at(n, Re, theta, node=None):
        run = O.cavity_run(33, Re, n, theta_deg=theta, dt_mode="grid")
        run.advance(40)
        ux, uy, _ = O.macros(run.fhat)
        psi = O.stream_function(ux, uy, run.g)
        if node is None:
            inner = np.real(psi)[1:-1, 1:-1]
            j, i = np.unravel_index(np.argmin(inner), inner.shape)
            node = (j + 1, i + 1)
        return psi[node], node

    x = [0.75, 400.0, 60.0]
    J, *g = objective_and_gradient("psi_min", *x, 33, 33, 40, every=10)
    J0, node = psi_at(*x)
    assert abs(J - J0) <= 1e-12 * abs(J0)
    for k in range(3):
        xs = [complex(v) for v in x]
        xs[k] += 1e-30j
        ref = np.imag(psi_at(*xs, node=node)[0]) / 1e-30
        assert abs(g[k] - ref) <= 1e-8 * abs(ref), (k, g[k], ref)


def test_adjoint_seed_psi_rejects_nodes_outside_the_cavity():
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import Solver, cavity
    s = Solver([cavity(17, 17, 100.0, 0.75)], precision="fp64", kernel="staged")
    buf = torch.zeros(capi.ifdlbm_state_bytes(s.h) // 8, dtype=torch.float64, device="cuda")
    adj = torch.zeros_like(buf)
    dp = torch.zeros(3, dtype=torch.float64, device="cuda")
    capi.ifdlbm_save_state_dev(s.h, buf)
    with pytest.raises(capi.IfdlbmError):
        capi.ifdlbm_adjoint_seed_psi(s.h, buf, [(17, 3)], adj, dp)
    s.close()


def test_adjoint_step_saved_equals_recomputing_step():
    """ifdlbm_adjoint_step_saved, fed the state after each step and the step's
    intermediates as ifdlbm_step left them, gives the adjoint and the parameter
    terms of ifdlbm_adjoint_step (which forms the step again) bit for bit, over
    a reverse sweep of five steps from an oracle-developed state."""
    import torch

    from paper_2306_07603_gb300 import capi
    from paper_2306_07603_gb300.solver import Solver, cavity
    from paper_2306_07603_gb300.workloads import smooth_noise

    nx, ny, n = 37, 29, 0.75
    run = O.cavity_run(nx, 400.0, n, theta_deg=60.0, ny=ny, dt_mode="grid")
    run.advance(40)
    s = Solver([cavity(nx, ny, 400.0, n, theta_deg=60.0)], precision="fp64", kernel="staged",
               dt_mode="grid")
    states = [_dev_state(s, run.fhat.copy(), run.lam.copy())]
    nb = capi.ifdlbm_intermediate_bytes(s.h)
    assert nb == 27 * (capi.ifdlbm_state_bytes(s.h) - 8) // 10
    inter = []
    for _ in range(5):
        s.step(1)
        st = torch.empty_like(states[0])
        it = torch.empty(nb // 8, dtype=torch.float64, device="cuda")
        capi.ifdlbm_save_state_dev(s.h, st)
        capi.ifdlbm_save_intermediates_dev(s.h, it)
        states.append(st)
        inter.append(it)
    seed = smooth_noise((9, ny, nx), seed=5)
    w = _dev_state(s, seed + O.OMEGA[:, None, None], smooth_noise((ny, nx), seed=6))
    a_re, a_sv = w.clone(), w.clone()
    d_re = torch.zeros(3, dtype=torch.float64, device="cuda")
    d_sv = torch.zeros(3, dtype=torch.float64, device="cuda")
    for k in range(4, -1, -1):
        capi.ifdlbm_adjoint_step(s.h, states[k], a_re, d_re)
        capi.ifdlbm_adjoint_step_saved(s.h, states[k], states[k + 1], inter[k], a_sv, d_sv)
    s.sync()
    assert torch.equal(a_re, a_sv)
    assert torch.equal(d_re, d_sv)
    assert float(d_re.abs().sum()) > 0.0
    with pytest.raises(capi.IfdlbmError):
        capi.ifdlbm_adjoint_step_saved(s.h, states[0], None, inter[0], a_sv, d_sv)
    with pytest.raises(capi.IfdlbmError):
        capi.ifdlbm_save_intermediates_dev(s.h, None)
    s.close()


def test_gradient_does_not_depend_on_the_checkpoint_interval():
    """Every checkpointing of the sweep feeds the adjoint the same states and
    intermediates (recomputed from checkpoints, or kept by the forward pass
    with every = 1), so the gradients agree bit for bit."""
    from paper_2306_07603_gb300.adjoint import energy_and_gradient
    x = [0.75, 400.0, 60.0]
    ref = energy_and_gradient(*x, 33, 29, 40, every=1)
    for every in (3, 40, 100):
        assert energy_and_gradient(*x, 33, 29, 40, every=every) == ref

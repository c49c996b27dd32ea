"""Whole-step pins of the oracle against analytic flows and the paper's tables.

* free-stream preservation on the skewed theta = 60 deg mesh;
* steady power-law Poiseuille flow (textbook closed form), n < 1, = 1, > 1;
* plane Couette flow under a moving lid (the moving-wall branch of the wall rule);
* Taylor-Green vortex decay rate for n = 1 (exact Navier-Stokes solution);
* second-order grid convergence of that decay rate;
* the primary-eddy centre of the paper's Table 2 (slow; loose tolerance).
"""
import math
import os

import numpy as np
import pytest

import oracle as O


def test_free_stream_preserved_on_skewed_mesh():
    """Uniform (u, P) with walls moving at that velocity is a fixed point:
    every difference of a constant vanishes and the boundary rule returns
    the state itself (Eqs. (3.6)-(3.7), Sec. 4 boundary)."""
    g = O.cavity_grid(17, 15, 1.0, 1.0, 60.0)
    u0, v0, p0 = 0.04, -0.03, 2e-3
    for side in g.wall_u:
        n = len(g.wall_u[side][0])
        g.wall_u[side] = (np.full(n, u0), np.full(n, v0))
    prm = O.Params(dt=0.5 / 16, K=0.002, n=0.75, gamma_min=1e-4, eta_b=0.5)
    shape = (g.ny, g.nx)
    fhat, lam = O.initial_state(g, prm, np.full(shape, p0), np.full(shape, u0), np.full(shape, v0))
    f0 = fhat.copy()
    for _ in range(100):
        fhat, lam = O.step(fhat, lam, g, prm)
    assert np.abs(fhat - f0).max() < 1e-14


def _poiseuille(n, ny, mu_wall=0.005, umax=0.05, ntau=2.0, eta_b=0.5):
    """Channel periodic in x with a pressure drop, walls at y = 0 and y = H = 1.

    Steady power-law solution (textbook): with G = -dP/dx,
    u(y) = U_max [1 - |2 y / H - 1|^((n+1)/n)],
    U_max = n/(n+1) (G/K)^(1/n) (H/2)^((n+1)/n).

    K is set so that the apparent viscosity at the wall is mu_wall; the
    kinetic model recovers the Navier-Stokes limit only while the mean free
    path lam c = 3 mu / c stays well below H, so mu is kept small (the
    zero-shear clamp caps it at the centreline for n < 1). The run starts
    from the analytic profile and advances two viscous time constants
    H^2 / (pi^2 mu_wall): a wrong viscosity, exponent or stress would drift
    the profile away by tens of percent over that time.
    Returns (max error / U_max, last GRE(u)).
    """
    H = 1.0
    gdot_wall = umax * (n + 1) / n * 2.0 / H
    K = mu_wall / gdot_wall ** (n - 1.0)
    G = K * (umax * (n + 1) / n) ** n / (H / 2) ** (n + 1)
    nx = 5
    deta = H / (ny - 1)
    Lx = nx * deta                      # square cells
    g = O.periodic_grid(nx, ny, Lx, H, periodic_eta=False)
    g.jump_P = -G * Lx
    prm = O.Params(dt=0.5 * deta, K=K, n=n, gamma_min=0.01 * gdot_wall, eta_b=eta_b)
    exact = umax * (1.0 - np.abs(2 * g.y / H - 1.0) ** ((n + 1) / n))
    fhat, lam = O.initial_state(g, prm, P0=-G * g.x, ux0=exact)
    nsteps = int(ntau * H * H / (np.pi ** 2 * mu_wall) / prm.dt)
    run = O.Run(g=g, prm=prm, fhat=fhat, lam=lam)
    run.advance(nsteps - 1)
    run.advance(1, record=True)
    ux, uy, _ = O.macros(run.fhat)
    return np.abs(ux - exact).max() / umax, np.abs(uy).max(), run.history[-1][0]


@pytest.mark.parametrize("n,tol33", [(0.5, 2.5e-2), (1.0, 5e-3), (1.5, 1e-2)])
def test_power_law_poiseuille_profile_and_convergence(n, tol33):
    e17, _, _ = _poiseuille(n, 17)
    e33, v33, gre = _poiseuille(n, 33)
    assert e33 < tol33, (e17, e33)
    assert e17 / e33 > 2.5, (e17, e33)
    assert v33 < 1e-6 * 0.05
    assert gre < 1e-6


def _couette(n, ny, U, mu=0.01, nx=4):
    """Channel periodic in x, bottom wall at rest, top wall (the lid) moving at
    (U, 0). The steady Navier-Stokes solution is u = U y / H for every power-law
    index: the shear rate U / H is uniform, so is mu = K (U/H)^(n-1), and the
    momentum balance reduces to d^2u/dy^2 = 0. K is set so that mu is the given
    value. The run starts from that profile with f-hat = f^eq and advances until
    the max-norm velocity residual is below 1e-14; the lid enters only through
    the moving-wall branch of the non-equilibrium extrapolation (Sec. 4).
    Returns (max |u - U y/H| / U, max |v| / U)."""
    H = 1.0
    K = mu / (U / H) ** (n - 1.0)
    deta = H / (ny - 1)
    g = O.periodic_grid(nx, ny, nx * deta, H, periodic_eta=False)
    z = np.zeros(nx)
    g.wall_u = dict(bottom=(z, z), top=(np.full(nx, U), z))
    prm = O.Params(dt=0.5 * deta, K=K, n=n, gamma_min=1e-3 * U / H, eta_b=0.5)
    exact = U * g.y / H
    fhat, lam = O.initial_state(g, prm, ux0=exact)
    run = O.Run(g=g, prm=prm, fhat=fhat, lam=lam)
    for _ in range(100):
        run.advance(199)
        run.advance(1, record=True)
        if run.history[-1][2] < 1e-14:
            break
    assert run.history[-1][2] < 1e-14, run.history[-1]
    ux, uy, _ = O.macros(run.fhat)
    return np.abs(ux - exact).max() / U, np.abs(uy).max() / U


def test_plane_couette_newtonian_exact():
    """n = 1: the kinetic scheme holds the linear profile to rounding."""
    du, dv = _couette(1.0, 17, U=0.05)
    assert du < 1e-12 and dv < 1e-12, (du, dv)


@pytest.mark.parametrize("n", [0.5, 0.75, 1.5])
def test_plane_couette_power_law(n):
    """n != 1: the profile is U y / H up to the O(Ma^2) term by which the strain
    rate of Eqs. (2.12)-(2.13) (from f^ne) departs from the velocity gradient;
    through mu(gamma-dot) it bends the profile slightly. That term falls as U^2:
    halving U divides the relative deviation by 4. A wrong lid velocity, a lid
    rule that drops the wall term, or a non-uniform viscosity from a wrong
    exponent would leave an O(1) error instead."""
    d1, v1 = _couette(n, 9, U=0.02)
    d2, v2 = _couette(n, 9, U=0.01)
    assert d2 < 2e-9 and v2 < 1e-10, (d2, v2)
    assert 3.9 < d1 / d2 < 4.1, (d1, d2)


def _taylor_green(N, nu=0.002, U0=0.01, t_end=1.0, t_start=0.25, eta_b=0.5):
    """Doubly periodic Taylor-Green vortex on [0, 1)^2 with k = 2 pi, n = 1:
    u = -U0 cos(kx) sin(ky) e^{-2 nu k^2 t}, v = U0 sin(kx) cos(ky) e^{...},
    P = -U0^2/4 (cos 2kx + cos 2ky) e^{-4 nu k^2 t} (exact NSE solution).

    The viscosity is small enough that the kinetic correction (lam c k)^2
    stays below 0.2 %. Returns the measured and the exact decay rate of the
    velocity amplitude over [t_start, t_end]."""
    k = 2 * np.pi
    g = O.periodic_grid(N, N, 1.0, 1.0, periodic_eta=True)
    dt = 0.5 / N
    prm = O.Params(dt=dt, K=nu, n=1.0, gamma_min=1e-8, eta_b=eta_b)
    x, y = g.x, g.y
    mode_u = -np.cos(k * x) * np.sin(k * y)
    mode_v = np.sin(k * x) * np.cos(k * y)
    P0 = -U0 ** 2 / 4 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    fhat, lam = O.initial_state(g, prm, P0, U0 * mode_u, U0 * mode_v)

    def amp(f):
        ux, uy, _ = O.macros(f)
        return np.sum(ux * mode_u + uy * mode_v) / np.sum(mode_u ** 2 + mode_v ** 2)

    n1, n2 = int(round(t_start / dt)), int(round(t_end / dt))
    for s in range(n2):
        if s == n1:
            a1 = amp(fhat)
        fhat, lam = O.step(fhat, lam, g, prm)
    measured = math.log(a1 / amp(fhat)) / ((n2 - n1) * dt)
    return measured, 2 * nu * k * k


def test_taylor_green_decay_rate_newtonian():
    """Viscous decay rate 2 nu k^2 with nu = lam c_s^2 = K (Eq. (2.14), n = 1)."""
    measured, exact = _taylor_green(64)
    assert abs(measured / exact - 1) < 0.015, (measured, exact)


@pytest.mark.parametrize("eta_b", [0.5, 1.0])
def test_taylor_green_second_order_convergence(eta_b):
    """The decay-rate error falls by at least 3x per halving of h (2nd order)."""
    e = [abs(m / x - 1) for m, x in (_taylor_green(N, eta_b=eta_b) for N in (32, 64))]
    assert e[0] / e[1] > 3.0, e


@pytest.mark.slow
def test_primary_eddy_centre_table2(golden_dir):
    """Table 2 (theta = 60 deg, n = 0.75, Re = 100): primary eddy at
    (1.4292, 0.6872). On a 33^2 grid the psi-minimum node must lie within
    1.5 grid spacings (physical) of the printed centre."""
    rows = np.loadtxt(os.path.join(golden_dir, "eddy_centres_re100.txt"))
    row = rows[(rows[:, 0] == 60) & (rows[:, 1] == 0.75)][0]
    run = O.cavity_run(33, 100.0, 0.75, theta_deg=60.0)
    while run.steps < 40000:
        run.advance(500, record=True)
        if run.history[-1][0] < 1e-8:
            break
    psi = run.fields()["psi"]
    j, i = np.unravel_index(np.argmin(psi), psi.shape)
    x, y = run.g.x[j, i], run.g.y[j, i]
    h = 1.0 / 32
    assert abs(x - row[2]) < 1.5 * h * (1 + 2 / math.sqrt(3)) and abs(y - row[3]) < 1.5 * h


@pytest.mark.parametrize("theta,corners", [(90.0, True), (60.0, False)])
def test_wall_rule_first_order_pressure_is_exact_for_linear_pressure(theta, corners):
    """The alternative wall reading (first-order pressure, P_b = 2 P_nb - P_nnb):
    on an equilibrium state with a pressure linear in (x, y) and no flow, the
    wall rule must give every wall node f^eq of the exact linear pressure
    there (linear extrapolation along a grid line is exact for a linear
    function of the line parameter). On the theta = 60 deg map the diagonal
    corner lines are not straight in (x, y), so only the edges are checked
    there. The zeroth-order reading (P_b = P_nb) misses by the pressure step."""
    g = O.cavity_grid(9, 11, 1.0, 1.0, theta)
    for side in g.wall_u:
        nn = len(g.wall_u[side][0])
        g.wall_u[side] = (np.zeros(nn), np.zeros(nn))
    P = 1e-3 + 2e-3 * g.x - 3e-3 * g.y
    F0 = O.equilibrium(P, 0.0 * P, 0.0 * P)
    expect = O.equilibrium(P, 0.0 * P, 0.0 * P)
    mask = np.zeros((g.ny, g.nx), dtype=bool)
    mask[0, 1:-1] = mask[-1, 1:-1] = True
    mask[1:-1, 0] = mask[1:-1, -1] = True
    if corners:
        mask[0, 0] = mask[0, -1] = mask[-1, 0] = mask[-1, -1] = True
    for wp, exact in ((1, True), (0, False)):
        prm = O.Params(dt=0.01, K=0.01, n=1.0, gamma_min=1e-4, eta_b=0.5, wall_pressure=wp)
        F = O.nee_boundary(F0.copy(), g, prm)
        err = np.abs(F - expect)[:, mask].max()
        assert (err < 1e-14) == exact, (wp, err)


def test_free_stream_preserved_with_first_order_wall_pressure():
    g = O.cavity_grid(17, 15, 1.0, 1.0, 60.0)
    u0, v0, p0 = 0.04, -0.03, 2e-3
    for side in g.wall_u:
        nn = len(g.wall_u[side][0])
        g.wall_u[side] = (np.full(nn, u0), np.full(nn, v0))
    prm = O.Params(dt=0.5 / 16, K=0.002, n=0.75, gamma_min=1e-4, eta_b=0.5, wall_pressure=1)
    shape = (g.ny, g.nx)
    fhat, lam = O.initial_state(g, prm, np.full(shape, p0), np.full(shape, u0), np.full(shape, v0))
    f0 = fhat.copy()
    for _ in range(100):
        fhat, lam = O.step(fhat, lam, g, prm)
    assert np.abs(fhat - f0).max() < 1e-14

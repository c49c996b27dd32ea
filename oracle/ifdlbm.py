"""Plain, slow FP64 CPU oracle of the IFDLBM time step (test infrastructure).

This module is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may import it. It shares no code, table or
constant with the CUDA library, and the CUDA library never calls it.

It restates, step by step and in the paper's order and notation, the
incompressible finite-difference lattice Boltzmann method (IFDLBM) of
Chen, Chai, Zhao and Shi (arXiv 2306.07603) for a power-law fluid in a
lid-driven isosceles trapezoidal cavity mapped to the unit square:

* D2Q9 lattice and weights ............................ Eq. (2.9)
* designed equilibrium ................................ Eq. (2.8), moments Eq. (A1)
* macroscopic velocity and pressure ................... Eqs. (2.10), (2.11)
* strain rate from the non-equilibrium part ........... Eqs. (2.12), (2.13)
* power-law apparent viscosity, relaxation time ....... Eqs. (1.4), (2.14), (2.15.1)
* closed-form transforms of the two-stage scheme ...... Eqs. (2.15)-(2.18)
* mixed central / 2nd-order upwind differences ........ Eqs. (2.5)-(2.7)
* curvilinear metrics and contravariant velocities .... Eqs. (3.1)-(3.5), (3.8)
* transformed evolution equations ..................... Eqs. (3.6), (3.7)
* non-equilibrium extrapolation boundary .............. Sec. 4 (boundary scheme)
* calculation process Steps (1)-(8) ................... Sec. 4
* global relative error ............................... Eq. (2.19)
* kinetic energy ...................................... Eq. (5.1)
* eddy centres of Tables 1-3 .......................... Sec. 5.1 (a READING)
* implicit relaxation time (Eq. 2.14 at the current
  lambda, solved by bisection) ........................ Eq. (2.14), (2.18)
* general convex quadrilaterals (bilinear map,
  per-node metrics) ................................... Eqs. (3.2)-(3.4) (a READING)

Where the paper is silent, garbled or self-contradictory, one explicit
reading is taken; each is marked ``READING`` below. The same readings bind
the CUDA path.

Every function works on NumPy arrays and is written so that complex inputs
(complex-step differentiation) flow through: branch decisions (upwind side,
clamps) are taken on real parts only.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, analytic solutions or the paper's printed
numbers; none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# D2Q9 lattice, Eq. (2.9).  Column j of the velocity matrix is e_j; the
# physical velocity is c_j = c * e_j.
# ---------------------------------------------------------------------------
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.float64)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.float64)
OMEGA = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
# The pressure weights: omega_bar_0 = -5/9, the others equal omega_j.
OMEGA_BAR = np.array([-5 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
Q = 9


def _re(x):
    """Real part, used for every branch decision (complex-step safety)."""
    return np.real(x)


def sound_speed_sq(c=1.0):
    """c_s^2 = c^2 / 3 for D2Q9."""
    return c * c / 3.0


def _bcast(w, like):
    """Reshape a length-9 lattice vector to broadcast against (9, ...)."""
    return np.asarray(w).reshape((Q,) + (1,) * (np.ndim(like)))


# ---------------------------------------------------------------------------
# Equilibrium and moments
# ---------------------------------------------------------------------------
def equilibrium(P, ux, uy, rho0=1.0, c=1.0):
    """Designed incompressible equilibrium f_i^eq(P, u), Eq. (2.8).

    f_i^eq = wbar_i P / c_s^2 + w_i rho0
             + w_i [ c_i.u / c_s^2 + u u : (c_i c_i - c_s^2 I) / (2 c_s^4) ]

    READING: the printed denominator of the quadratic term is 2 c_s^2; only
    2 c_s^4 gives the second moment of Eq. (A1), (P + c_s^2 rho0) I + u u.
    Returns an array of shape (9,) + shape(P).
    """
    P = np.asarray(P)
    cs2 = sound_speed_sq(c)
    ex, ey = _bcast(EX * c, P), _bcast(EY * c, P)
    w, wb = _bcast(OMEGA, P), _bcast(OMEGA_BAR, P)
    cu = ex * ux + ey * uy
    uu = ux * ux + uy * uy
    # u u : (c_i c_i - c_s^2 I) = (c_i.u)^2 - c_s^2 |u|^2
    quad = (cu * cu - cs2 * uu) / (2.0 * cs2 * cs2)
    return wb * P / cs2 + w * rho0 + w * (cu / cs2 + quad)


def macros(F, rho0=1.0, c=1.0):
    """Velocity and pressure from f, f-hat or f-bar, Eqs. (2.10)-(2.11).

    u = sum_i c_i F_i
    P = c_s^2 / wbar_0 * ( -sum_{i!=0} F_i + (1 - w_0) rho0 + w_0 |u|^2 / (2 c_s^2) )

    READING: the "u u" of Eq. (2.11) is the scalar |u|^2 (it equals the
    inversion of Eq. (2.8) for f_0^eq).
    Returns (ux, uy, P).
    """
    cs2 = sound_speed_sq(c)
    ex, ey = _bcast(EX * c, F[0]), _bcast(EY * c, F[0])
    ux = np.sum(ex * F, axis=0)
    uy = np.sum(ey * F, axis=0)
    s = np.sum(F[1:], axis=0)
    uu = ux * ux + uy * uy
    P = cs2 / OMEGA_BAR[0] * (-s + (1.0 - OMEGA[0]) * rho0 + OMEGA[0] * uu / (2.0 * cs2))
    return ux, uy, P


# ---------------------------------------------------------------------------
# Closed-form transforms of the two-stage scheme, Eqs. (2.15)-(2.18)
#
# READING: Eqs. (2.3)-(2.4) print the collision as "-lambda (f - f^eq)";
# the BGK operator of Eq. (2.0) is -(f - f^eq)/lambda, and only that form
# reproduces the closed forms (2.15)-(2.18) that the algorithm uses. The
# oracle codes (2.15)-(2.18) directly; the tests check them against
# (2.3)-(2.4) with the BGK operator.
# ---------------------------------------------------------------------------
def f_from_fhat(fhat, feq, lam, dt):
    """f = 2 lam / (2 lam + dt) f-hat + dt / (2 lam + dt) f^eq, Eq. (2.18)."""
    return (2.0 * lam / (2.0 * lam + dt)) * fhat + (dt / (2.0 * lam + dt)) * feq


def fhat_plus(fhat, feq, lam, dt):
    """f-hat^+ = (2 lam - dt)/(2 lam + dt) f-hat + 2 dt/(2 lam + dt) f^eq, Eq. (2.15)."""
    return ((2.0 * lam - dt) / (2.0 * lam + dt)) * fhat + (2.0 * dt / (2.0 * lam + dt)) * feq


def fbar_plus(fhat, feq, lam, dt):
    """f-bar^+ = (4 lam - dt)/(4 lam + 2 dt) f-hat + 3 dt/(4 lam + 2 dt) f^eq, Eq. (2.16)."""
    return ((4.0 * lam - dt) / (4.0 * lam + 2.0 * dt)) * fhat + (3.0 * dt / (4.0 * lam + 2.0 * dt)) * feq


def f_from_fbar(fbar, feq, lam, dt):
    """f = 4 lam/(4 lam + dt) f-bar + dt/(4 lam + dt) f^eq, Eq. (2.17)."""
    return (4.0 * lam / (4.0 * lam + dt)) * fbar + (dt / (4.0 * lam + dt)) * feq


# ---------------------------------------------------------------------------
# Power-law rheology
# ---------------------------------------------------------------------------
def consistency_coefficient(Re, n, U, H):
    """K from the power-law Reynolds number Re = U^(2-n) H^n / K, Eq. (2.15.1).

    READING: the "mu" of Eq. (2.15.1) is the consistency coefficient K of
    Eq. (1.4), and the length is the cavity height H.
    """
    return U ** (2.0 - n) * H ** n / Re


def strain_rate(f, feq, lam, c=1.0):
    """S = grad u + grad u^T = -sum_i c_i c_i f_i^ne / (lam c_s^2), Eqs. (2.12)-(2.13).

    Returns (S_xx, S_xy, S_yy).
    """
    cs2 = sound_speed_sq(c)
    fne = f - feq
    ex, ey = _bcast(EX * c, fne[0]), _bcast(EY * c, fne[0])
    pxx = np.sum(ex * ex * fne, axis=0)
    pxy = np.sum(ex * ey * fne, axis=0)
    pyy = np.sum(ey * ey * fne, axis=0)
    k = -1.0 / (lam * cs2)
    return k * pxx, k * pxy, k * pyy


def shear_rate(Sxx, Sxy, Syy):
    """|gamma-dot| = sqrt(2 D:D) with D = S/2, Eqs. (1.3.1), (1.4).

    2 D:D = (1/2) (S_xx^2 + 2 S_xy^2 + S_yy^2).
    """
    return np.sqrt(0.5 * (Sxx * Sxx + 2.0 * Sxy * Sxy + Syy * Syy))


def relaxation_time(gdot, K, n, gamma_min, c=1.0):
    """lam = mu / c_s^2 with mu = K |gamma-dot|^(n-1), Eqs. (1.4), (2.14).

    READING: the paper does not say how mu behaves at zero shear, where
    |gamma-dot|^(n-1) diverges for n < 1 and vanishes for n > 1. The shear
    rate is clamped from below: mu = K max(|gamma-dot|, gamma_min)^(n-1).
    """
    g = np.where(_re(gdot) > _re(gamma_min), gdot, gamma_min + 0.0 * gdot)
    return K * g ** (n - 1.0) / sound_speed_sq(c)


def relaxation_time_implicit(fhat, feq, dt, K, n, gamma_min, c=1.0, iters=200):
    """lam solving lam = K max(gamma-dot(lam), gamma_min)^(n-1) / c_s^2 node by node.

    The implicit form of Eq. (2.14), which the paper lags (the text after
    Eq. 2.14 takes the strain rate with the previous step's lam). With f from
    f-hat by Eq. (2.18) at the same lam, f^ne = 2 lam / (2 lam + dt) (f-hat -
    f^eq), and Eqs. (2.12)-(2.13) give gamma-dot(lam) = a / (2 lam + dt),
    a = 2 sqrt((Pi_xx^2 + 2 Pi_xy^2 + Pi_yy^2) / 2) / c_s^2 with
    Pi = sum_i c_i c_i (f-hat_i - f^eq_i), which does not depend on lam.
    F(lam) = lam - K max(gamma-dot(lam), gamma_min)^(n-1) / c_s^2 increases
    strictly with lam, is negative at lam = 0 and non-negative at
    lam_hi = K/c_s^2 max over gamma in [gamma_min, max(a/dt, gamma_min)] of
    gamma^(n-1); its root is found by bisection (real arithmetic only).
    """
    cs2 = sound_speed_sq(c)
    d = fhat - feq
    ex, ey = _bcast(EX * c, d[0]), _bcast(EY * c, d[0])
    pxx, pxy, pyy = (np.sum(w * d, axis=0) for w in (ex * ex, ex * ey, ey * ey))
    a = 2.0 * np.sqrt(0.5 * (pxx * pxx + 2.0 * pxy * pxy + pyy * pyy)) / cs2
    C = K / cs2
    gmax = np.maximum(a / dt, gamma_min)
    lo = np.zeros_like(a)
    hi = C * np.maximum(gmax ** (n - 1.0), gamma_min ** (n - 1.0))

    def F(lam):
        g = np.maximum(a / (2.0 * lam + dt), gamma_min)
        return lam - C * g ** (n - 1.0)

    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        pos = F(mid) >= 0.0
        hi = np.where(pos, mid, hi)
        lo = np.where(pos, lo, mid)
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------------------
# Geometry: isosceles trapezoid mapped to the unit square, Eqs. (3.1)-(3.8)
# ---------------------------------------------------------------------------
def cot_deg(theta_deg):
    """cot(theta) for theta in degrees; exactly 0 at theta = 90 (the square)."""
    t = np.asarray(theta_deg) * (math.pi / 180.0)
    ct = np.cos(t) / np.sin(t)
    if float(_re(theta_deg)) == 90.0:
        ct = ct - _re(ct)  # keep only the complex-step part
    return ct


def trapezoid_xy(xi, eta, L=1.0, H=1.0, theta_deg=60.0):
    """Physical point (x, y) of computational point (xi, eta), Eq. (3.8.1).

    General {L, H}: x = L xi + H cot(theta) (1 - eta + 2 xi eta), y = H eta.
    At L = H = 1 this is Eq. (3.8.1) term by term. The bottom edge spans
    x in [H cot, L + H cot], the lid (eta = 1) spans x in [0, L + 2 H cot].
    """
    ct = cot_deg(theta_deg)
    x = L * xi + H * ct * (1.0 - eta + 2.0 * xi * eta)
    y = H * eta + 0.0 * xi
    return x, y


def trapezoid_metrics(xi, eta, L=1.0, H=1.0, theta_deg=60.0):
    """Analytic derivatives of the map, Eq. (3.8.2), Jacobian Eq. (3.3) and
    inverse metrics Eq. (3.2).

    Returns a dict with x_xi, x_eta, y_xi, y_eta, J, xi_x, xi_y, eta_x, eta_y.
    """
    ct = cot_deg(theta_deg)
    x_xi = L + 2.0 * H * ct * eta + 0.0 * xi
    x_eta = H * ct * (2.0 * xi - 1.0) + 0.0 * eta
    y_xi = 0.0 * (xi + eta)
    y_eta = H + 0.0 * (xi + eta)
    return inverse_metrics(x_xi, x_eta, y_xi, y_eta)


def inverse_metrics(x_xi, x_eta, y_xi, y_eta):
    """[xi_x xi_y; eta_x eta_y] = (1/J) [y_eta -x_eta; -y_xi x_xi], Eqs. (3.2)-(3.3)."""
    J = x_xi * y_eta - x_eta * y_xi
    return dict(x_xi=x_xi, x_eta=x_eta, y_xi=y_xi, y_eta=y_eta, J=J,
                xi_x=y_eta / J, xi_y=-x_eta / J, eta_x=-y_xi / J, eta_y=x_xi / J)


def contravariant_velocities(met, c=1.0):
    """c_{i xi} = c_ix xi_x + c_iy xi_y, c_{i eta} = c_ix eta_x + c_iy eta_y, Eq. (3.4).

    Returns two arrays of shape (9,) + grid shape.
    """
    ex, ey = _bcast(EX * c, met["J"]), _bcast(EY * c, met["J"])
    cxi = ex * met["xi_x"] + ey * met["xi_y"]
    ceta = ex * met["eta_x"] + ey * met["eta_y"]
    return cxi, ceta


# ---------------------------------------------------------------------------
# Mixed difference scheme, Eqs. (2.5)-(2.7)
# ---------------------------------------------------------------------------
def mixed_derivative(F, cvel, d, eta_b, axis, periodic=False, jump=None):
    """dPi/dchi|_m = eta_b * central + (1 - eta_b) * 2nd-order upwind, Eqs. (2.5)-(2.7).

    F and cvel have the grid shape (ny, nx); ``axis`` is 1 for xi, 0 for eta;
    d is the grid spacing along that axis.

    * central, Eq. (2.6): (F[k+1] - F[k-1]) / (2 d)
    * upwind, Eq. (2.7), c >= 0: (3 F[k] - 4 F[k-1] + F[k-2]) / (2 d)
                         c <  0: -(3 F[k] - 4 F[k+1] + F[k+2]) / (2 d)
      READING: the printed c < 0 branch repeats F[k+1] as its third term;
      the second-order stencil that differentiates linear functions exactly
      uses F[k+2].
    * READING (upwind side): the side is chosen per node by the sign of the
      contravariant velocity component along that axis; c = 0 takes the
      c >= 0 branch.
    * READING (near-wall nodes, non-periodic axis): where the upwind stencil
      would reach beyond the grid (k = 1 with c >= 0, k = N-2 with c < 0),
      the first-order upwind difference is used. The derivative is only
      formed at interior nodes 1..N-2; boundary entries are returned as 0.

    For a periodic axis, ``jump`` (same leading shape as F broadcast) is the
    value added to F when it is carried one period forward (test-only
    periodic-with-pressure-jump condition).
    """
    F = np.moveaxis(F, axis, 0)
    cv = np.moveaxis(np.broadcast_to(cvel, np.shape(cvel)), axis, 0)
    N = F.shape[0]
    out = np.zeros(F.shape, dtype=np.result_type(F, cv, 1.0))
    if periodic:
        jmp = 0.0 if jump is None else jump
        ext = np.concatenate([F[N - 2:] - jmp, F, F[:2] + jmp], axis=0)
        k = np.arange(N) + 2
        central = (ext[k + 1] - ext[k - 1]) / (2.0 * d)
        up_pos = (3.0 * ext[k] - 4.0 * ext[k - 1] + ext[k - 2]) / (2.0 * d)
        up_neg = -(3.0 * ext[k] - 4.0 * ext[k + 1] + ext[k + 2]) / (2.0 * d)
        upwind = np.where(_re(cv) >= 0.0, up_pos, up_neg)
        out[:] = eta_b * central + (1.0 - eta_b) * upwind
    else:
        # interior nodes k = 1..N-2, all at once
        central = (F[2:] - F[:-2]) / (2.0 * d)
        up_pos = np.empty_like(central)
        up_pos[1:] = (3.0 * F[2:N - 1] - 4.0 * F[1:N - 2] + F[0:N - 3]) / (2.0 * d)
        up_pos[0] = (F[1] - F[0]) / d                      # k = 1, first order
        up_neg = np.empty_like(central)
        up_neg[:-1] = -(3.0 * F[1:N - 2] - 4.0 * F[2:N - 1] + F[3:N]) / (2.0 * d)
        up_neg[-1] = (F[N - 1] - F[N - 2]) / d             # k = N-2, first order
        upwind = np.where(_re(cv[1:N - 1]) >= 0.0, up_pos, up_neg)
        out[1:N - 1] = eta_b * central + (1.0 - eta_b) * upwind
    return np.moveaxis(out, 0, axis)


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------
@dataclass
class Grid:
    """A computational grid with its contravariant velocities and boundaries.

    nx, ny     nodes along xi (contiguous) and eta
    dxi, deta  computational spacings
    cxi, ceta  contravariant velocities, shape (9, ny, nx), Eq. (3.4)
    J          Jacobian per node, Eq. (3.3) (area weight of Eq. (5.1))
    x_eta, y_eta  metric terms used by the stream function
    periodic_xi, periodic_eta   axis boundary kind (False = walls)
    wall_u     dict side -> (ux, uy) wall velocity arrays along that side
               (sides: 'bottom', 'top' of length nx; 'left', 'right' of length ny)
    jump_P     pressure change over one period along xi (test-only)
    """
    nx: int
    ny: int
    dxi: float
    deta: float
    cxi: np.ndarray
    ceta: np.ndarray
    J: np.ndarray
    x_eta: np.ndarray
    y_eta: np.ndarray
    periodic_xi: bool = False
    periodic_eta: bool = False
    wall_u: dict = field(default_factory=dict)
    jump_P: float = 0.0
    x: np.ndarray | None = None
    y: np.ndarray | None = None


@dataclass
class Params:
    """Run parameters (Sec. 5.1: c = 1, CFL = 0.5, lid speed U = 0.1)."""
    dt: float
    K: complex | float
    n: complex | float
    gamma_min: float
    eta_b: float
    rho0: float = 1.0
    c: float = 1.0
    implicit_lambda: bool = False   # solve Eq. (2.14) at the current lam instead of lagging
    wall_pressure: int = 0          # wall-rule pressure: 0 zeroth-order, 1 first-order extrapolation


def cavity_grid(nx, ny, L=1.0, H=1.0, theta_deg=60.0, U=0.1, c=1.0):
    """The lid-driven trapezoidal cavity of Sec. 2 on an nx x ny node grid.

    Nodes: xi_i = i / (nx - 1), eta_j = j / (ny - 1); j = 0 is the bottom
    wall, j = ny - 1 the lid. Boundary conditions, Eq. (1.5): no slip on
    the bottom and the two inclined side walls, u = (U, 0) on the lid.
    READING: the two top corner nodes belong to the stationary side walls.
    """
    xi = np.linspace(0.0, 1.0, nx)[None, :]
    eta = np.linspace(0.0, 1.0, ny)[:, None]
    met = trapezoid_metrics(xi, eta, L, H, theta_deg)
    cxi, ceta = contravariant_velocities(met, c)
    x, y = trapezoid_xy(xi, eta, L, H, theta_deg)
    lid = np.zeros(nx, dtype=np.result_type(U, 1.0))
    lid[1:-1] = U
    z_x = np.zeros(nx)
    z_y = np.zeros(ny)
    wall_u = dict(bottom=(z_x, z_x), top=(lid, z_x), left=(z_y, z_y), right=(z_y, z_y))
    return Grid(nx=nx, ny=ny, dxi=1.0 / (nx - 1), deta=1.0 / (ny - 1), cxi=cxi, ceta=ceta,
                J=met["J"] + 0.0 * xi, x_eta=met["x_eta"] + 0.0 * eta,
                y_eta=met["y_eta"] + 0.0 * (xi + eta), wall_u=wall_u, x=x, y=y)


def quad_xy(xi, eta, corners):
    """Bilinear (Coons) map of the unit square onto the quadrilateral with
    corners ((x0, y0) bottom-left, (x1, y1) bottom-right, (x2, y2) top-left,
    (x3, y3) top-right): xi runs along the bottom and lid, eta up the sides."""
    (x0, y0), (x1, y1), (x2, y2), (x3, y3) = corners
    w = ((1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta)
    x = w[0] * x0 + w[1] * x1 + w[2] * x2 + w[3] * x3
    y = w[0] * y0 + w[1] * y1 + w[2] * y2 + w[3] * y3
    return x, y


def quad_metrics(xi, eta, corners):
    """Analytic derivatives of the bilinear map, the Jacobian (Eq. 3.3) and the
    inverse metrics (Eq. 3.2); eta_x need not vanish here."""
    (x0, y0), (x1, y1), (x2, y2), (x3, y3) = corners
    x_xi = (1 - eta) * (x1 - x0) + eta * (x3 - x2) + 0.0 * xi
    y_xi = (1 - eta) * (y1 - y0) + eta * (y3 - y2) + 0.0 * xi
    x_eta = (1 - xi) * (x2 - x0) + xi * (x3 - x1) + 0.0 * eta
    y_eta = (1 - xi) * (y2 - y0) + xi * (y3 - y1) + 0.0 * eta
    return inverse_metrics(x_xi, x_eta, y_xi, y_eta)


def quad_grid(nx, ny, corners, U=0.1, c=1.0):
    """A lid-driven cavity on a general convex quadrilateral (per-node metrics).

    READING (the paper's cavities are trapezoids; this generalises them): the
    lid is the top edge (corner 2 to corner 3) and moves along itself at speed
    U, u_lid = U (x3 - x2, y3 - y2) / |...|; the other walls are at rest, the
    two top corner nodes too. With the trapezoid's corners this is
    cavity_grid exactly.
    """
    xi = np.linspace(0.0, 1.0, nx)[None, :]
    eta = np.linspace(0.0, 1.0, ny)[:, None]
    met = quad_metrics(xi, eta, corners)
    if np.any(met["J"] <= 0):
        raise ValueError("corners must make a convex, counter-clockwise quadrilateral")
    cxi, ceta = contravariant_velocities(met, c)
    x, y = quad_xy(xi, eta, corners)
    (x0, y0), (x1, y1), (x2, y2), (x3, y3) = corners
    tl = math.hypot(x3 - x2, y3 - y2)
    lid_x, lid_y = np.zeros(nx), np.zeros(nx)
    lid_x[1:-1] = U * (x3 - x2) / tl
    lid_y[1:-1] = U * (y3 - y2) / tl
    z_x, z_y = np.zeros(nx), np.zeros(ny)
    wall_u = dict(bottom=(z_x, z_x), top=(lid_x, lid_y), left=(z_y, z_y), right=(z_y, z_y))
    return Grid(nx=nx, ny=ny, dxi=1.0 / (nx - 1), deta=1.0 / (ny - 1), cxi=cxi, ceta=ceta,
                J=met["J"] + 0.0 * (xi + eta), x_eta=met["x_eta"] + 0.0 * (xi + eta),
                y_eta=met["y_eta"] + 0.0 * (xi + eta), wall_u=wall_u, x=x + 0.0 * eta,
                y=y + 0.0 * xi)


def quad_run(nx, ny, corners, Re, n, H=1.0, U=0.1, **kw):
    """Rest-state lid-driven cavity on a general quadrilateral; K from Eq.
    (2.15.1) with the reference length H."""
    g = quad_grid(nx, ny, corners, U)
    prm = cavity_params(nx, ny, Re, n, U=U, H=H, grid=g, **kw)
    fhat, lam = initial_state(g, prm)
    return Run(g=g, prm=prm, fhat=fhat, lam=lam)


def periodic_grid(nx, ny, Lx=1.0, Ly=1.0, periodic_eta=True, c=1.0):
    """Identity-map test domain (x = Lx xi, y = Ly eta) used by the oracle's pins.

    Periodic along xi (node spacing Lx / nx); along eta either periodic
    (spacing Ly / ny) or bounded by two stationary walls at eta = 0 and
    eta = 1 (spacing Ly / (ny - 1)). It is not part of the cavity problem;
    it hosts the analytic flows (Taylor-Green, power-law Poiseuille).
    """
    dxi = 1.0 / nx
    deta = 1.0 / ny if periodic_eta else 1.0 / (ny - 1)
    xi = (np.arange(nx) * dxi)[None, :]
    eta = (np.arange(ny) * deta)[:, None]
    one = np.ones((ny, nx))
    met = inverse_metrics(Lx * one, 0.0 * one, 0.0 * one, Ly * one)
    cxi, ceta = contravariant_velocities(met, c)
    z = np.zeros(nx)
    wall_u = {} if periodic_eta else dict(bottom=(z, z), top=(z, z))
    return Grid(nx=nx, ny=ny, dxi=dxi, deta=deta, cxi=cxi, ceta=ceta, J=met["J"],
                x_eta=0.0 * one, y_eta=Ly * one, periodic_xi=True,
                periodic_eta=periodic_eta, wall_u=wall_u, x=Lx * xi * one, y=Ly * eta * one)


def cavity_params(nx, ny, Re, n, U=0.1, H=1.0, L=1.0, cfl=0.5, c=1.0, eta_b=None,
                  gamma_min=None, dt=None, dt_mode="contravariant", grid=None,
                  implicit_lambda=False, wall_pressure=0):
    """Parameters of a cavity run.

    * K from Re, Eq. (2.15.1).
    * READING (time step, c = 1 and CFL = 0.5 of Sec. 5.1): the Courant
      number applies to the contravariant speeds of Eq. (3.4), the speeds
      the finite differences of the computational grid see:
      dt = CFL * min(dxi / max|c_xi|, deta / max|c_eta|), taken over all
      nodes and directions (dt_mode "contravariant", needs the cavity's
      Grid). On the skewed grid these speeds exceed c, and the rule
      dt = CFL * min(L dxi, H deta) / c (dt_mode "grid") lets the two-stage
      scheme amplify the diagonal populations (von Neumann factor up to
      1.75 per step at theta = 60 deg); the 256^2, Re = 100, n >= 1
      cavities of Tables 1-3 then diverge. At theta = 90 deg both rules
      agree.
    * READING (blend): eta_b, which the paper leaves free in [0, 1], defaults
      to DEFAULT_ETA_B.
    * READING (zero-shear clamp): gamma_min defaults to 1e-3 U / H.
    * implicit_lambda: solve Eq. (2.14) with the strain rate of the current
      lam (relaxation_time_implicit) instead of the paper's lagged lam.
    """
    K = consistency_coefficient(Re, n, U, H)
    if dt is None and dt_mode == "contravariant":
        if grid is None:
            raise ValueError("dt_mode 'contravariant' needs the cavity's Grid")
        mxi = float(np.max(np.abs(_re(grid.cxi))))
        meta = float(np.max(np.abs(_re(grid.ceta))))
        dt = cfl * min(grid.dxi / mxi, grid.deta / meta)
    elif dt is None:
        dt = cfl * min(L / (nx - 1), H / (ny - 1)) / c
    if eta_b is None:
        eta_b = DEFAULT_ETA_B
    if gamma_min is None:
        gamma_min = 1e-3 * U / H
    return Params(dt=dt, K=K, n=n, gamma_min=gamma_min, eta_b=eta_b, c=c,
                  implicit_lambda=implicit_lambda, wall_pressure=wall_pressure)


DEFAULT_ETA_B = 0.5


# ---------------------------------------------------------------------------
# Non-equilibrium extrapolation boundary (Sec. 4)
# ---------------------------------------------------------------------------
def _boundary_nodes(g: Grid):
    """List of (side, index along side, (jb, ib), (jn, in)) for every wall node.

    READING: the neighbour is the adjacent interior node along the
    computational-grid normal; a corner uses its diagonal interior node.
    A corner shared by two walls is listed once, with the side whose wall
    velocity it takes (the vertical walls for the cavity corners).
    """
    nx, ny = g.nx, g.ny
    out = []
    walls_eta = not g.periodic_eta
    walls_xi = not g.periodic_xi
    if walls_eta:
        i_range = range(1, nx - 1) if walls_xi else range(nx)
        for i in i_range:
            out.append(("bottom", i, (0, i), (1, i)))
            out.append(("top", i, (ny - 1, i), (ny - 2, i)))
    if walls_xi:
        j_range = range(1, ny - 1) if walls_eta else range(ny)
        for j in j_range:
            out.append(("left", j, (j, 0), (j, 1)))
            out.append(("right", j, (j, nx - 1), (j, nx - 2)))
    if walls_xi and walls_eta:
        out.append(("left", 0, (0, 0), (1, 1)))
        out.append(("right", 0, (0, nx - 1), (1, nx - 2)))
        out.append(("left", ny - 1, (ny - 1, 0), (ny - 2, 1)))
        out.append(("right", ny - 1, (ny - 1, nx - 1), (ny - 2, nx - 2)))
    return out


def nee_boundary(F, g: Grid, prm: Params):
    """Non-equilibrium extrapolation on every wall node, in place.

    F_b = f^eq(P_nb, u_wall) + [F_nb - f^eq(P_nb, u_nb)]

    READING: the pressure is extrapolated at zeroth order (P_b = P_nb); the
    same rule is applied to f at t + dt/2 (needed by the full-step stencil)
    and to f-hat at t + dt (Step 6). The alternative reading
    prm.wall_pressure = 1 extrapolates it at first order along the same grid
    line, P_b = 2 P_nb - P_nnb, nnb the next node beyond nb (the diagonal one
    at corners); the non-equilibrium part is taken from nb as before.
    """
    nodes = _boundary_nodes(g)
    if not nodes:
        return F
    jb = np.array([b[2][0] for b in nodes])
    ib = np.array([b[2][1] for b in nodes])
    jn = np.array([b[3][0] for b in nodes])
    inn = np.array([b[3][1] for b in nodes])
    uw_x = np.array([g.wall_u[b[0]][0][b[1]] for b in nodes])
    uw_y = np.array([g.wall_u[b[0]][1][b[1]] for b in nodes])
    Fn = F[:, jn, inn]                                   # (9, n_boundary)
    ux_n, uy_n, P_n = macros(Fn, prm.rho0, prm.c)
    P_b = P_n
    if getattr(prm, "wall_pressure", 0) == 1:
        P_nn = macros(F[:, 2 * jn - jb, 2 * inn - ib], prm.rho0, prm.c)[2]
        P_b = 2.0 * P_n - P_nn
    fe_w = equilibrium(P_b, uw_x + 0.0 * P_n, uw_y + 0.0 * P_n, prm.rho0, prm.c)
    fe_n = equilibrium(P_n, ux_n, uy_n, prm.rho0, prm.c)
    F[:, jb, ib] = fe_w + (Fn - fe_n)
    return F


def _interior_mask(g: Grid):
    m = np.ones((g.ny, g.nx), dtype=bool)
    if not g.periodic_eta:
        m[0, :] = False
        m[-1, :] = False
    if not g.periodic_xi:
        m[:, 0] = False
        m[:, -1] = False
    return m


def advection(F, g: Grid, prm: Params, P_jump_per_dir=None):
    """(c_{i xi} d/dxi + c_{i eta} d/deta) F_i at interior nodes, Eqs. (3.4)-(3.5)."""
    out = np.zeros(F.shape, dtype=np.result_type(F, g.cxi, 1.0))
    for i in range(1, Q):  # c_0 = 0: no advection of the rest population
        jump = None
        if g.periodic_xi and P_jump_per_dir is not None:
            jump = P_jump_per_dir[i]
        dxi = mixed_derivative(F[i], g.cxi[i], g.dxi, prm.eta_b, axis=1,
                               periodic=g.periodic_xi, jump=jump)
        deta = mixed_derivative(F[i], g.ceta[i], g.deta, prm.eta_b, axis=0,
                                periodic=g.periodic_eta)
        out[i] = g.cxi[i] * dxi + g.ceta[i] * deta
    return out


# ---------------------------------------------------------------------------
# One time step, Steps (2)-(7) of Sec. 4
# ---------------------------------------------------------------------------
def step(fhat, lam_prev, g: Grid, prm: Params, return_stages=False):
    """Advance f-hat from t to t + dt.

    fhat      (9, ny, nx) f-hat(t), boundary nodes included
    lam_prev  (ny, nx) relaxation time used by the previous step's Eq. (2.18)

    READING (lagged relaxation time, text after Eq. (2.14)): Step (2) forms
    f(t) from f-hat(t) with lam_prev (Eq. (2.18)), takes f^ne and the strain
    rate (Eqs. (2.12)-(2.13)) with lam_prev, and gets lam(t) from Eq. (2.14);
    lam(t) is then used in Eqs. (2.15), (2.16), (2.17) and is returned as
    the next step's lam_prev (it is the lam of Step (7)'s Eq. (2.18)).
    READING (half step): the half-step uses lam(t); the half-step macros
    come from f-bar at interior nodes; f(t + dt/2) on wall nodes comes from
    the non-equilibrium extrapolation.

    Returns (fhat_new, lam) or, with return_stages, also a dict of stages.
    """
    dt, rho0, c = prm.dt, prm.rho0, prm.c
    cs2 = sound_speed_sq(c)
    interior = _interior_mask(g)
    jump = None
    if g.periodic_xi and g.jump_P != 0.0:
        jump = OMEGA_BAR * g.jump_P / cs2  # f^eq shift for a pressure shift

    # Step (2): moments, equilibrium, lam from f^(1) = f - f^eq
    ux, uy, P = macros(fhat, rho0, c)                       # Eqs. (2.10)-(2.11)
    feq = equilibrium(P, ux, uy, rho0, c)                  # Eq. (2.8)
    f = f_from_fhat(fhat, feq, lam_prev, dt)               # Eq. (2.18), lam_prev
    Sxx, Sxy, Syy = strain_rate(f, feq, lam_prev, c)       # Eqs. (2.12)-(2.13)
    gdot = shear_rate(Sxx, Sxy, Syy)                       # Eq. (1.4)
    lam = relaxation_time(gdot, prm.K, prm.n, prm.gamma_min, c)  # Eq. (2.14)
    if prm.implicit_lambda:                                # Eq. (2.14) at the current lam
        lam = relaxation_time_implicit(fhat, feq, dt, prm.K, prm.n, prm.gamma_min, c)

    # Step (3): f-hat^+
    fhp = fhat_plus(fhat, feq, lam, dt)                    # Eq. (2.15)

    # Step (4): f-bar^+, half step, f(t + dt/2)
    fbp = fbar_plus(fhat, feq, lam, dt)                    # Eq. (2.16)
    fbar = fbp - 0.5 * dt * advection(fbp, g, prm, jump)   # Eq. (3.7)
    uxh, uyh, Ph = macros(fbar, rho0, c)                   # Eqs. (2.10)-(2.11) on f-bar
    feqh = equilibrium(Ph, uxh, uyh, rho0, c)
    fhalf = f_from_fbar(fbar, feqh, lam, dt)               # Eq. (2.17)
    fhalf = np.where(interior[None], fhalf, 0.0)
    nee_boundary(fhalf, g, prm)                            # boundary f(t + dt/2)

    # Step (5): f-hat(t + dt) at interior nodes
    fnew = fhp - dt * advection(fhalf, g, prm, jump)       # Eq. (3.6)
    fnew = np.where(interior[None], fnew, 0.0)

    # Step (6): boundary populations of f-hat(t + dt)
    nee_boundary(fnew, g, prm)

    if return_stages:
        return fnew, lam, dict(ux=ux, uy=uy, P=P, feq=feq, f=f, gdot=gdot, lam=lam,
                               fhat_plus=fhp, fbar_plus=fbp, fbar_half=fbar,
                               f_half=fhalf)
    return fnew, lam


# ---------------------------------------------------------------------------
# Initial state, Step (1)
# ---------------------------------------------------------------------------
def initial_state(g: Grid, prm: Params, P0=None, ux0=None, uy0=None):
    """f-hat(0) = f(0) = f^eq(P0, u0) (Step (1)); rest state by default.

    READING: wall nodes start at their wall velocity (impulsively started
    lid). lam_prev(0) is Eq. (2.14) at zero shear (the clamp value); at t = 0
    f^ne = 0, so it does not enter the first step's strain rate.
    """
    shape = (g.ny, g.nx)
    P0 = np.zeros(shape) if P0 is None else P0
    ux0 = np.zeros(shape) if ux0 is None else np.array(ux0, dtype=np.result_type(ux0, 1.0))
    uy0 = np.zeros(shape) if uy0 is None else np.array(uy0, dtype=np.result_type(uy0, 1.0))
    ux0 = ux0.astype(np.result_type(ux0, *[v[0] for v in g.wall_u.values()]), copy=True)
    uy0 = uy0.astype(np.result_type(uy0, 1.0), copy=True)
    for side, k, (jb, ib), _ in _boundary_nodes(g):
        ux0[jb, ib] = g.wall_u[side][0][k]
        uy0[jb, ib] = g.wall_u[side][1][k]
    fhat = equilibrium(P0, ux0, uy0, prm.rho0, prm.c)
    lam0 = relaxation_time(np.zeros(shape), prm.K, prm.n, prm.gamma_min, prm.c) + 0.0 * P0
    return fhat, lam0


# ---------------------------------------------------------------------------
# Diagnostics: Eq. (2.19), Eq. (5.1), stream function
# ---------------------------------------------------------------------------
def global_relative_error(ux, uy, P, ux_prev, uy_prev, P_prev):
    """GRE of u and P between consecutive steps, Eq. (2.19).

    E(u) = sqrt(sum |u^n - u^{n-1}|^2) / sqrt(sum |u^n|^2),
    E(P) = sqrt(sum (P^n - P^{n-1})^2) / sqrt(sum (P^n)^2).
    Also returns R_inf = max |u^n - u^{n-1}| / max |u^n| (Euclidean norm per
    node, max over nodes), the max-norm velocity residual.
    """
    du2 = (ux - ux_prev) ** 2 + (uy - uy_prev) ** 2
    u2 = ux ** 2 + uy ** 2
    Eu = np.sqrt(np.sum(du2)) / np.sqrt(np.sum(u2))
    EP = np.sqrt(np.sum((P - P_prev) ** 2)) / np.sqrt(np.sum(P ** 2))
    Rinf = np.sqrt(np.max(du2)) / np.sqrt(np.max(u2))
    return Eu, EP, Rinf


def trapezoid_weights(nx, ny):
    """Composite trapezoidal-rule weights over the unit square (dxi deta included)."""
    wx = np.full(nx, 1.0 / (nx - 1))
    wx[0] = wx[-1] = 0.5 / (nx - 1)
    wy = np.full(ny, 1.0 / (ny - 1))
    wy[0] = wy[-1] = 0.5 / (ny - 1)
    return wy[:, None] * wx[None, :]


def kinetic_energy(ux, uy, g: Grid):
    """E = 1/2 sum_Omega |u|^2 dx, Eq. (5.1).

    READING: the physical area element is dx = J dxi deta; the sum over
    nodes uses the composite trapezoidal rule in (xi, eta).
    """
    w = trapezoid_weights(g.nx, g.ny)
    return 0.5 * np.sum(w * g.J * (ux * ux + uy * uy))


def stream_function(ux, uy, g: Grid):
    """psi with psi = 0 on the bottom wall, integrated along xi = const lines.

    READING (the paper plots streamlines without stating how psi is formed):
    d psi = u dy - v dx = (u y_eta - v x_eta) d eta along a line of constant
    xi, integrated by the trapezoidal rule in eta from eta = 0.
    """
    integrand = ux * g.y_eta - uy * g.x_eta
    psi = np.zeros_like(integrand)
    psi[1:] = np.cumsum(0.5 * (integrand[1:] + integrand[:-1]) * g.deta, axis=0)
    return psi


def eddy_centres(psi, L=1.0, H=1.0, theta_deg=60.0):
    """Centres of the primary and the two bottom-corner eddies (Tables 1-3).

    READING (the paper tabulates the centres without saying how they were
    located): the primary eddy is the interior node of smallest psi (the
    clockwise eddy of a lid moving in +x); a corner eddy is, among interior
    nodes with eta <= 1/2 and xi < 1/2 (left) or xi >= 1/2 (right), the strict
    local maximum of psi (above its 8 neighbours) with the largest psi > 0.
    Each node is refined by the least-squares quadratic
    psi ~ a + b s + c t + d s^2 + e s t + f t^2 on its 3 x 3 neighbourhood
    (s, t node offsets): its stationary point is taken when the Hessian has
    the extremum's sign and the point lies within one node, else the node.
    Returns [primary, left, right], each a dict (x, y, xi, eta, psi, i, j,
    refined) or None.
    """
    psi = np.asarray(psi, dtype=float)
    ny, nx = psi.shape
    s_off, t_off = np.meshgrid([-1.0, 0.0, 1.0], [-1.0, 0.0, 1.0])
    s_off, t_off = s_off.ravel(), t_off.ravel()
    A = np.stack([np.ones(9), s_off, t_off, s_off ** 2, s_off * t_off, t_off ** 2], axis=1)

    def refine(i, j, minimum):
        patch = psi[j - 1:j + 2, i - 1:i + 2].ravel()
        a, b, c, d, e, f = np.linalg.lstsq(A, patch, rcond=None)[0]
        Hm = np.array([[2 * d, e], [e, 2 * f]])
        s = t = 0.0
        refined = False
        det = np.linalg.det(Hm)
        if det > 0 and ((2 * d > 0) if minimum else (2 * d < 0)):
            st = np.linalg.solve(Hm, -np.array([b, c]))
            if np.all(np.abs(st) <= 1.0):
                s, t = st
                refined = True
        val = a + b * s + c * t + d * s * s + e * s * t + f * t * t if refined else psi[j, i]
        xi_c, eta_c = (i + s) / (nx - 1), (j + t) / (ny - 1)
        x, y = trapezoid_xy(xi_c, eta_c, L, H, theta_deg)
        return dict(x=float(x), y=float(y), xi=xi_c, eta=eta_c, psi=float(val), i=i, j=j,
                    refined=refined)

    inner = psi[1:-1, 1:-1]
    j0, i0 = np.unravel_index(np.argmin(inner), inner.shape)
    out = [refine(i0 + 1, j0 + 1, True), None, None]
    best = [None, None]
    for j in range(1, ny - 1):
        if 2 * j > ny - 1:
            break
        for i in range(1, nx - 1):
            p = psi[j, i]
            nb = psi[j - 1:j + 2, i - 1:i + 2].copy()
            nb[1, 1] = -np.inf
            if p > 0 and p > nb.max():
                side = 0 if 2 * i < nx - 1 else 1
                if best[side] is None or p > psi[best[side][1], best[side][0]]:
                    best[side] = (i, j)
    for side in (0, 1):
        if best[side] is not None:
            out[1 + side] = refine(best[side][0], best[side][1], False)
    return out


# ---------------------------------------------------------------------------
# Driver
# ---------------------------------------------------------------------------
@dataclass
class Run:
    g: Grid
    prm: Params
    fhat: np.ndarray
    lam: np.ndarray
    steps: int = 0
    history: list = field(default_factory=list)

    def advance(self, nsteps, record=False):
        for _ in range(nsteps):
            ux0, uy0, P0 = macros(self.fhat, self.prm.rho0, self.prm.c)
            self.fhat, self.lam = step(self.fhat, self.lam, self.g, self.prm)
            self.steps += 1
            if record:
                ux1, uy1, P1 = macros(self.fhat, self.prm.rho0, self.prm.c)
                self.history.append(global_relative_error(ux1, uy1, P1, ux0, uy0, P0))
        return self

    def fields(self):
        ux, uy, P = macros(self.fhat, self.prm.rho0, self.prm.c)
        rho = self.prm.rho0 + P / sound_speed_sq(self.prm.c)
        return dict(rho=rho, u=ux, v=uy, P=P, psi=stream_function(ux, uy, self.g))


def cavity_run(n_nodes, Re, n, theta_deg=60.0, U=0.1, L=1.0, H=1.0, ny=None, **kw):
    """Rest-state lid-driven trapezoidal cavity ready to advance."""
    nx = n_nodes
    ny = n_nodes if ny is None else ny
    g = cavity_grid(nx, ny, L, H, theta_deg, U)
    prm = cavity_params(nx, ny, Re, n, U=U, H=H, L=L, grid=g, **kw)
    fhat, lam = initial_state(g, prm)
    return Run(g=g, prm=prm, fhat=fhat, lam=lam)

"""Cartesian restatement of the IFDLBM step for the square cavity (test infrastructure).

This module is test infrastructure, like ``oracle/ifdlbm.py``: only
``tests/`` may import it. It exists to pin the general oracle: at theta = 90
deg the trapezoid of Eq. (3.8.1) is the unit square, the map is the identity,
and the transformed equations (3.6)-(3.7) reduce to the Cartesian ones,

    f-bar(t + dt/2) = f-bar^+ - dt/2 (c_ix d_x + c_iy d_y) f-bar^+,
    f-hat(t + dt)   = f-hat^+ - dt   (c_ix d_x + c_iy d_y) f(t + dt/2),

so ``oracle.step`` on the theta = 90 deg grid must equal this step to
rounding. The two share no function: everything the step needs (lattice,
equilibrium, moments, power law, differences, wall rule) is written again
here, node by node along each grid line, in plain Python loops over
directions and rows, on the physical (x, y) grid with spacing h = 1/(N-1).

The readings are those of the general oracle (the same method): BGK sign of
Eqs. (2.3)-(2.4), Eq. (2.8) over 2 c_s^4, Eq. (2.11) with |u|^2, the c < 0
branch of Eq. (2.7) with the +2 node, the upwind side by the sign of c_ix or
c_iy (zero counts as positive), first-order upwind next to the walls, the
lagged relaxation time with the zero-shear clamp, non-equilibrium
extrapolation from the inner neighbour (the diagonal one at corners) with the
pressure taken from that neighbour, a lid that moves at (U, 0) between the
two top corners, which are at rest.
"""
from __future__ import annotations

import numpy as np

# D2Q9, Eq. (2.9): (e_x, e_y, w, wbar) per direction
LATTICE = [
    (0, 0, 4.0 / 9.0, -5.0 / 9.0),
    (1, 0, 1.0 / 9.0, 1.0 / 9.0),
    (0, 1, 1.0 / 9.0, 1.0 / 9.0),
    (-1, 0, 1.0 / 9.0, 1.0 / 9.0),
    (0, -1, 1.0 / 9.0, 1.0 / 9.0),
    (1, 1, 1.0 / 36.0, 1.0 / 36.0),
    (-1, 1, 1.0 / 36.0, 1.0 / 36.0),
    (-1, -1, 1.0 / 36.0, 1.0 / 36.0),
    (1, -1, 1.0 / 36.0, 1.0 / 36.0),
]


def feq_cart(P, ux, uy, c=1.0, rho0=1.0):
    """Eq. (2.8), direction by direction (list of 9 arrays)."""
    cs2 = c * c / 3.0
    out = []
    for exi, eyi, w, wb in LATTICE:
        cu = c * (exi * ux + eyi * uy)
        out.append(wb * P / cs2 + w * rho0
                   + w * (cu / cs2 + (cu * cu - cs2 * (ux * ux + uy * uy)) / (2.0 * cs2 * cs2)))
    return out


def moments_cart(F, c=1.0, rho0=1.0):
    """u = sum c_i F_i, P from Eq. (2.11) (wbar_0 = -5/9, w_0 = 4/9)."""
    cs2 = c * c / 3.0
    ux = sum(c * LATTICE[i][0] * F[i] for i in range(9))
    uy = sum(c * LATTICE[i][1] * F[i] for i in range(9))
    rest = sum(F[i] for i in range(1, 9))
    P = cs2 / (-5.0 / 9.0) * (-rest + (5.0 / 9.0) * rho0
                              + (4.0 / 9.0) * (ux * ux + uy * uy) / (2.0 * cs2))
    return ux, uy, P


def _d_line(v, cvel, h, eta_b):
    """Mixed difference of Eqs. (2.5)-(2.7) along one grid line v[0..N-1] at
    nodes 1..N-2 (0 elsewhere), with a constant particle speed cvel."""
    N = len(v)
    out = np.zeros(N)
    for k in range(1, N - 1):
        central = (v[k + 1] - v[k - 1]) / (2.0 * h)
        if cvel >= 0.0:
            up = (v[k] - v[k - 1]) / h if k == 1 else (3 * v[k] - 4 * v[k - 1] + v[k - 2]) / (2.0 * h)
        else:
            up = (v[k + 1] - v[k]) / h if k == N - 2 else -(3 * v[k] - 4 * v[k + 1] + v[k + 2]) / (2.0 * h)
        out[k] = eta_b * central + (1.0 - eta_b) * up
    return out


def advect_cart(F, h, eta_b, c=1.0):
    """(c_ix d_x + c_iy d_y) F_i on the interior of the square, per direction."""
    ny, nx = F[0].shape
    out = [np.zeros((ny, nx)) for _ in range(9)]
    for i in range(1, 9):
        cx, cy = c * LATTICE[i][0], c * LATTICE[i][1]
        a = np.zeros((ny, nx))
        if cx != 0.0:
            for j in range(ny):
                a[j] += cx * _d_line(F[i][j], cx, h, eta_b)
        if cy != 0.0:
            for k in range(nx):
                a[:, k] += cy * _d_line(F[i][:, k], cy, h, eta_b)
        a[0, :] = a[-1, :] = 0.0
        a[:, 0] = a[:, -1] = 0.0
        out[i] = a
    return out


def _walls_cart(F, U, c=1.0):
    """Non-equilibrium extrapolation on the square's walls, in place:
    F_b = f^eq(P_nb, u_w) + F_nb - f^eq(P_nb, u_nb)."""
    ny, nx = F[0].shape
    jobs = []
    for i in range(1, nx - 1):
        jobs.append((0, i, 1, i, 0.0))
        jobs.append((ny - 1, i, ny - 2, i, U))
    for j in range(1, ny - 1):
        jobs.append((j, 0, j, 1, 0.0))
        jobs.append((j, nx - 1, j, nx - 2, 0.0))
    jobs += [(0, 0, 1, 1, 0.0), (0, nx - 1, 1, nx - 2, 0.0),
             (ny - 1, 0, ny - 2, 1, 0.0), (ny - 1, nx - 1, ny - 2, nx - 2, 0.0)]
    new = []
    for jb, ib, jn, inn, uw in jobs:
        Fn = [F[q][jn, inn] for q in range(9)]
        ux, uy, P = moments_cart(Fn, c)
        fw = feq_cart(P, uw, 0.0, c)
        fn = feq_cart(P, ux, uy, c)
        new.append((jb, ib, [fw[q] + Fn[q] - fn[q] for q in range(9)]))
    for jb, ib, vals in new:
        for q in range(9):
            F[q][jb, ib] = vals[q]


def step_cart(fhat, lam_prev, U, K, n, dt, eta_b, gamma_min, c=1.0):
    """One step on the N x N square (Steps (2)-(6) of Sec. 4, Cartesian form).

    fhat: array (9, N, N), lam_prev: (N, N). Returns (fhat_new, lam)."""
    F = [np.array(fhat[q], dtype=float) for q in range(9)]
    N = F[0].shape[0]
    h = 1.0 / (N - 1)
    cs2 = c * c / 3.0
    ux, uy, P = moments_cart(F, c)
    fe = feq_cart(P, ux, uy, c)
    # Eq. (2.18) with lam_prev, then Eqs. (2.12)-(2.13), (1.4), (2.14)
    a = 2.0 * lam_prev / (2.0 * lam_prev + dt)
    fne = [a * (F[q] - fe[q]) for q in range(9)]
    sxx = sum((c * LATTICE[q][0]) ** 2 * fne[q] for q in range(9)) * (-1.0 / (lam_prev * cs2))
    sxy = sum(c * c * LATTICE[q][0] * LATTICE[q][1] * fne[q] for q in range(9)) * (-1.0 / (lam_prev * cs2))
    syy = sum((c * LATTICE[q][1]) ** 2 * fne[q] for q in range(9)) * (-1.0 / (lam_prev * cs2))
    gdot = np.sqrt(0.5 * (sxx ** 2 + 2.0 * sxy ** 2 + syy ** 2))
    lam = K * np.maximum(gdot, gamma_min) ** (n - 1.0) / cs2
    # Eqs. (2.15), (2.16)
    fhp = [((2 * lam - dt) * F[q] + 2 * dt * fe[q]) / (2 * lam + dt) for q in range(9)]
    fbp = [((4 * lam - dt) * F[q] + 3 * dt * fe[q]) / (4 * lam + 2 * dt) for q in range(9)]
    # half step, Eq. (3.7) at theta = 90 deg, then Eq. (2.17)
    adv = advect_cart(fbp, h, eta_b, c)
    fbar = [fbp[q] - 0.5 * dt * adv[q] for q in range(9)]
    uxh, uyh, Ph = moments_cart(fbar, c)
    feh = feq_cart(Ph, uxh, uyh, c)
    fhalf = [(4 * lam * fbar[q] + dt * feh[q]) / (4 * lam + dt) for q in range(9)]
    _walls_cart(fhalf, U, c)
    # full step, Eq. (3.6) at theta = 90 deg, then the walls of f-hat(t + dt)
    adv = advect_cart(fhalf, h, eta_b, c)
    fnew = [fhp[q] - dt * adv[q] for q in range(9)]
    _walls_cart(fnew, U, c)
    return np.stack(fnew), lam

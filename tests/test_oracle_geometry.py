"""Pins of the oracle's geometry, difference operators and diagnostics.

* the map is the bilinear (Coons) interpolation of the trapezoid's corners
  and reproduces the paper's printed Eq. (3.8.1) and probe point;
* analytic metrics equal exact finite differences of the bilinear map and
  invert the Jacobian matrix (library inverse);
* the mixed scheme differentiates polynomials exactly where its order says;
* the transformed advection operator c_i . grad reproduces physical
  gradients of linear / quadratic fields (pins metrics + contravariant
  velocities + stencils together);
* diagnostics reduce to closed forms (area, uniform flows, library norms).
"""
import math
import os

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(7603)


def _corners(L, H, th):
    ct = 1.0 / math.tan(math.radians(th)) if th != 90 else 0.0
    return (H * ct, 0.0), (L + H * ct, 0.0), (0.0, H), (L + 2 * H * ct, H)


@pytest.mark.parametrize("L,H,th", [(1, 1, 60), (1, 1, 45), (1.3, 0.8, 75), (2, 1, 30), (1, 1, 90)])
def test_map_is_bilinear_coons_of_corners(L, H, th):
    (x00, y00), (x10, y10), (x01, y01), (x11, y11) = _corners(L, H, th)
    xi, eta = RNG.random(100), RNG.random(100)
    x, y = O.trapezoid_xy(xi, eta, L, H, th)
    xb = (1 - xi) * (1 - eta) * x00 + xi * (1 - eta) * x10 + (1 - xi) * eta * x01 + xi * eta * x11
    yb = (1 - xi) * (1 - eta) * y00 + xi * (1 - eta) * y10 + (1 - xi) * eta * y01 + xi * eta * y11
    np.testing.assert_allclose(x, xb, atol=1e-14)
    np.testing.assert_allclose(y, yb, atol=1e-14)


@pytest.mark.parametrize("th", [75, 60, 45])
def test_map_matches_printed_eq381(th):
    """Eq. (3.8.1) as printed (L = H = 1): x = 2/tan(t) xi eta + xi - eta/tan(t) + 1/tan(t)."""
    t = math.tan(math.radians(th))
    xi, eta = RNG.random(50), RNG.random(50)
    x, y = O.trapezoid_xy(xi, eta, 1.0, 1.0, th)
    np.testing.assert_allclose(x, 2 / t * xi * eta + xi - eta / t + 1 / t, atol=1e-14)
    np.testing.assert_allclose(y, eta, atol=0)


def test_probe_point_golden(golden_dir):
    """The paper's theta = 60 deg probe [1.07735, 0.5] is the image of (0.5, 0.5)."""
    rows = np.loadtxt(os.path.join(golden_dir, "probe_point.txt"))
    th, xi, eta, xp, yp = rows
    x, y = O.trapezoid_xy(xi, eta, 1.0, 1.0, th)
    assert abs(x - xp) < 5e-6 and abs(y - yp) < 1e-15


def test_square_is_identity_map():
    """theta = 90 deg: cot is exactly 0 and the map is the identity."""
    assert O.cot_deg(90.0) == 0.0
    xi, eta = RNG.random(10), RNG.random(10)
    x, y = O.trapezoid_xy(xi, eta, 1.0, 1.0, 90.0)
    assert np.array_equal(x, xi) and np.array_equal(y, eta)


@pytest.mark.parametrize("L,H,th", [(1, 1, 60), (1.5, 0.7, 45)])
def test_metrics_equal_exact_differences_and_invert(L, H, th):
    """Eq. (3.8.2): central differences of a bilinear map are exact; Eq. (3.2):
    [xi_x xi_y; eta_x eta_y] is the inverse of [x_xi x_eta; y_xi y_eta]."""
    xi, eta = RNG.random(30), RNG.random(30)
    h = 1e-3
    m = O.trapezoid_metrics(xi, eta, L, H, th)
    xp, _ = O.trapezoid_xy(xi + h, eta, L, H, th)
    xm, _ = O.trapezoid_xy(xi - h, eta, L, H, th)
    np.testing.assert_allclose(m["x_xi"], (xp - xm) / (2 * h), rtol=1e-10)
    xp, yp = O.trapezoid_xy(xi, eta + h, L, H, th)
    xm, ym = O.trapezoid_xy(xi, eta - h, L, H, th)
    np.testing.assert_allclose(m["x_eta"], (xp - xm) / (2 * h), atol=1e-10)
    np.testing.assert_allclose(m["y_eta"], (yp - ym) / (2 * h), rtol=1e-10)
    for k in range(30):
        A = np.array([[m["x_xi"][k], m["x_eta"][k]], [m["y_xi"][k], m["y_eta"][k]]])
        Ainv = np.linalg.inv(A)
        B = np.array([[m["xi_x"][k], m["xi_y"][k]], [m["eta_x"][k], m["eta_y"][k]]])
        np.testing.assert_allclose(B, Ainv, rtol=1e-13, atol=1e-15)
        assert abs(m["J"][k] - np.linalg.det(A)) < 1e-13


@pytest.mark.parametrize("eta_b", [1.0, 0.5, 0.0])
def test_mixed_derivative_polynomial_exactness(eta_b):
    """Eqs. (2.5)-(2.7): central and 2nd-order upwind differentiate quadratics
    exactly (both upwind sides); the first-order near-wall stencil is exact
    for linear functions."""
    N, d = 12, 0.1
    s = np.arange(N) * d
    quad = (1.3 - 0.7 * s + 2.1 * s * s)[:, None] * np.ones((1, 3))
    dquad = (-0.7 + 4.2 * s)[:, None] * np.ones((1, 3))
    for sign in (+1.0, -1.0):
        cv = sign * np.ones((N, 3))
        D = O.mixed_derivative(quad, cv, d, eta_b, axis=0)
        inner = slice(2, N - 2)
        np.testing.assert_allclose(D[inner], dquad[inner], rtol=1e-12)
        lin = (0.4 - 1.9 * s)[:, None] * np.ones((1, 3))
        D = O.mixed_derivative(lin, cv, d, eta_b, axis=0)
        np.testing.assert_allclose(D[1:N - 1], -1.9, rtol=1e-12)
        assert np.all(D[0] == 0) and np.all(D[-1] == 0)
    # along axis 1 as well
    D = O.mixed_derivative(quad.T.copy(), np.ones((3, N)), d, eta_b, axis=1)
    np.testing.assert_allclose(D[:, 2:N - 2], dquad.T[:, 2:N - 2], rtol=1e-12)


def test_mixed_derivative_upwind_side_matters():
    """The two upwind branches differ on a cubic (so a swapped branch is caught):
    the c >= 0 branch uses points k-2..k, the c < 0 branch k..k+2."""
    N, d = 10, 1.0
    s = np.arange(N, dtype=float)
    F = (s ** 3)[:, None]
    k = 5
    Dp = O.mixed_derivative(F, np.ones((N, 1)), d, 0.0, axis=0)[k, 0]
    Dn = O.mixed_derivative(F, -np.ones((N, 1)), d, 0.0, axis=0)[k, 0]
    assert Dp == (3 * k ** 3 - 4 * (k - 1) ** 3 + (k - 2) ** 3) / 2
    assert Dn == -(3 * k ** 3 - 4 * (k + 1) ** 3 + (k + 2) ** 3) / 2


def test_mixed_derivative_periodic_second_order():
    """Periodic axis: error on sin(2 pi s) falls by ~4x per halving of d."""
    errs = []
    for N in (32, 64):
        d = 1.0 / N
        s = np.arange(N) * d
        F = np.sin(2 * np.pi * s)[:, None]
        D = O.mixed_derivative(F, np.ones((N, 1)), d, 0.5, axis=0, periodic=True)
        errs.append(np.abs(D[:, 0] - 2 * np.pi * np.cos(2 * np.pi * s)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("th", [60, 45, 30, 90])
@pytest.mark.parametrize("eta_b", [0.5, 1.0])
def test_advection_operator_reproduces_physical_gradients(th, eta_b):
    """Eqs. (3.4)-(3.5): c_{i xi} d_xi F + c_{i eta} d_eta F equals c_i . grad F
    for F linear in (x, y) at every interior node, and for F = x^2 + x y at
    nodes where the 2nd-order stencils apply (exact for these polynomials)."""
    g = O.cavity_grid(13, 11, 1.0, 1.0, th)
    prm = O.Params(dt=0.01, K=0.01, n=1.0, gamma_min=1e-4, eta_b=eta_b)
    x, y = g.x, g.y
    F = np.broadcast_to(0.3 * x - 1.7 * y + 0.2, (9,) + x.shape).copy()
    A = O.advection(F, g, prm)
    for i in range(1, 9):
        np.testing.assert_allclose(A[i][1:-1, 1:-1], O.EX[i] * 0.3 - O.EY[i] * 1.7, atol=1e-12)
    F = np.broadcast_to(x * x + x * y, (9,) + x.shape).copy()
    A = O.advection(F, g, prm)
    for i in range(1, 9):
        exact = O.EX[i] * (2 * x + y) + O.EY[i] * x
        np.testing.assert_allclose(A[i][2:-2, 2:-2], exact[2:-2, 2:-2], atol=1e-11)


@pytest.mark.parametrize("th,L,H", [(60, 1, 1), (45, 1.2, 0.9), (90, 1, 1)])
def test_area_and_kinetic_energy_closed_forms(th, L, H):
    """Eq. (5.1) weights integrate the Jacobian to the trapezoid's area
    H (L + H cot) exactly; a uniform flow has E = |U|^2 area / 2."""
    g = O.cavity_grid(9, 7, L, H, th)
    ct = 0.0 if th == 90 else 1 / math.tan(math.radians(th))
    area = H * (L + H * ct)
    assert abs(np.sum(O.trapezoid_weights(9, 7) * g.J) - area) < 1e-14
    ux = np.full((7, 9), 0.03)
    uy = np.full((7, 9), -0.04)
    assert abs(O.kinetic_energy(ux, uy, g) - 0.5 * 0.05 ** 2 * area) < 1e-16


def test_stream_function_closed_forms():
    """psi of uniform flows is exact; a smooth solenoidal field converges at 2nd order."""
    g = O.cavity_grid(11, 9, 1.0, 1.0, 60)
    psi = O.stream_function(np.full((9, 11), 0.1), np.zeros((9, 11)), g)
    np.testing.assert_allclose(psi, 0.1 * g.y, atol=1e-15)
    psi = O.stream_function(np.zeros((9, 11)), np.full((9, 11), 0.2), g)
    np.testing.assert_allclose(psi, -0.2 * (g.x - g.x[0:1, :]), atol=1e-15)
    errs = []
    for N in (17, 33):
        g = O.cavity_grid(N, N, 1.0, 1.0, 60)
        x, y = g.x, g.y
        ux, uy = 2 * np.sin(x) * y, -np.cos(x) * y * y      # psi = sin(x) y^2
        errs.append(np.abs(O.stream_function(ux, uy, g) - np.sin(x) * y * y).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_global_relative_error_library_norms():
    """Eq. (2.19) equals ratios of library 2-norms; a field from rest gives 1."""
    ux, uy, P = RNG.standard_normal((3, 5, 6))
    u0, v0, p0 = RNG.standard_normal((3, 5, 6))
    Eu, EP, Rinf = O.global_relative_error(ux, uy, P, u0, v0, p0)
    du = np.stack([ux - u0, uy - v0]).ravel()
    assert abs(Eu - np.linalg.norm(du) / np.linalg.norm(np.stack([ux, uy]).ravel())) < 1e-14
    assert abs(EP - np.linalg.norm(P - p0) / np.linalg.norm(P)) < 1e-14
    z = np.zeros_like(ux)
    assert O.global_relative_error(ux, uy, P, z, z, z)[:2] == (1.0, 1.0)
    assert abs(Rinf - np.hypot(ux - u0, uy - v0).max() / np.hypot(ux, uy).max()) < 1e-14


@pytest.mark.parametrize("th", [45.0, 60.0, 75.0, 90.0])
@pytest.mark.parametrize("nx,ny", [(33, 33), (65, 65), (41, 29)])
def test_contravariant_time_step_closed_form(th, nx, ny):
    """Default time step (c = 1, CFL = 0.5 of Sec. 5.1 applied to the
    contravariant speeds of Eq. 3.4). On the L = H = 1 trapezoid,
    c_xi = (e_x - e_y x_eta) / x_xi with x_xi = 1 + 2 cot(theta) eta >= 1 and
    |x_eta| = cot(theta) |2 xi - 1| <= cot(theta), so max |c_xi| = 1 + cot(theta),
    reached by the diagonal directions at the two bottom corners, and
    c_eta = e_y gives max |c_eta| = 1. Hence
    dt = CFL min(dxi / (1 + cot(theta)), deta); at 90 deg, CFL min(dxi, deta)."""
    cot = 0.0 if th == 90.0 else math.cos(math.radians(th)) / math.sin(math.radians(th))
    g = O.cavity_grid(nx, ny, 1.0, 1.0, th)
    prm = O.cavity_params(nx, ny, 100.0, 0.75, grid=g)
    dxi, deta = 1.0 / (nx - 1), 1.0 / (ny - 1)
    expect = 0.5 * min(dxi / (1.0 + cot), deta)
    assert prm.dt == pytest.approx(expect, rel=1e-14)
    # the grid rule of the same paragraph: CFL min(L dxi, H deta) / c
    prm_g = O.cavity_params(nx, ny, 100.0, 0.75, grid=g, dt_mode="grid")
    assert prm_g.dt == pytest.approx(0.5 * min(dxi, deta), rel=1e-14)
    # CFL scales it linearly
    prm_c = O.cavity_params(nx, ny, 100.0, 0.75, grid=g, cfl=0.25)
    assert prm_c.dt == pytest.approx(0.5 * expect, rel=1e-14)

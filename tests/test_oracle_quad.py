"""Pins of the oracle's general quadrilateral cavity (per-node metrics, the
second half of the implicit-lambda / general-metrics extension).

* With the trapezoid's corners the bilinear map is the map of Eq. (3.8.1):
  the grid (metrics, contravariant velocities, Jacobian, walls) and a run
  equal the trapezoid ones.
* Central differences of the bilinear map equal its analytic metrics (the
  map is linear along each grid line).
* The composite trapezoidal rule integrates the Jacobian to the polygon's
  shoelace area (J is bilinear).
* A uniform flow with walls moving at that velocity stays uniform on a
  skewed quadrilateral whose eta_x does not vanish (free-stream
  preservation with general metrics).
"""
import math

import numpy as np

import oracle as O

SKEW = ((0.1, -0.05), (1.3, 0.12), (-0.2, 0.9), (1.05, 1.1))


def _trapezoid_corners(theta=60.0, L=1.0, H=1.0):
    ct = 1.0 / math.tan(math.radians(theta))
    return ((H * ct, 0.0), (L + H * ct, 0.0), (0.0, H), (L + 2 * H * ct, H))


def test_trapezoid_corners_reproduce_the_trapezoid_grid_and_run():
    ga = O.quad_grid(23, 19, _trapezoid_corners())
    gb = O.cavity_grid(23, 19, 1.0, 1.0, 60.0)
    for k in ("cxi", "ceta", "J", "x_eta", "y_eta", "x", "y"):
        a, b = getattr(ga, k), getattr(gb, k)
        assert np.abs(a - b).max() <= 1e-14 * max(np.abs(b).max(), 1.0), k
    for side in gb.wall_u:
        for q in (0, 1):
            assert np.abs(ga.wall_u[side][q] - gb.wall_u[side][q]).max() <= 1e-16
    ra = O.quad_run(23, 19, _trapezoid_corners(), 400.0, 0.75, H=1.0)
    rb = O.cavity_run(23, 400.0, 0.75, theta_deg=60.0, ny=19)
    assert abs(ra.prm.dt - rb.prm.dt) <= 1e-15 * rb.prm.dt
    ra.advance(20)
    rb.advance(20)
    assert np.abs(ra.fhat - rb.fhat).max() <= 1e-13


def test_metrics_equal_central_differences_of_the_map():
    nx, ny = 21, 17
    xi = np.linspace(0, 1, nx)[None, :]
    eta = np.linspace(0, 1, ny)[:, None]
    x, y = O.quad_xy(xi + 0 * eta, eta + 0 * xi, SKEW)
    met = O.quad_metrics(xi, eta, SKEW)
    dxi, deta = 1.0 / (nx - 1), 1.0 / (ny - 1)
    assert np.allclose((x[:, 2:] - x[:, :-2]) / (2 * dxi), met["x_xi"][:, 1:-1] + 0 * x[:, 1:-1],
                       rtol=0, atol=1e-13)
    assert np.allclose((y[2:] - y[:-2]) / (2 * deta), met["y_eta"][1:-1] + 0 * y[1:-1],
                       rtol=0, atol=1e-13)
    assert np.allclose((x[2:] - x[:-2]) / (2 * deta), met["x_eta"][1:-1] + 0 * x[1:-1],
                       rtol=0, atol=1e-13)
    assert np.abs(met["eta_x"]).max() > 1e-2       # a genuinely general mesh


def test_jacobian_integrates_to_the_shoelace_area():
    nx, ny = 13, 11
    g = O.quad_grid(nx, ny, SKEW)
    w = O.trapezoid_weights(nx, ny)
    area = float((w * g.J).sum())          # the weights include dxi deta
    (x0, y0), (x1, y1), (x2, y2), (x3, y3) = SKEW
    poly = [(x0, y0), (x1, y1), (x3, y3), (x2, y2)]
    shoe = 0.5 * abs(sum(poly[k][0] * poly[k - 1][1] - poly[k - 1][0] * poly[k][1]
                         for k in range(4)))
    assert abs(area - shoe) <= 1e-14


def test_free_stream_preserved_on_a_general_quadrilateral():
    g = O.quad_grid(17, 15, SKEW)
    u0, v0, p0 = 0.04, -0.03, 2e-3
    for side in g.wall_u:
        n = len(g.wall_u[side][0])
        g.wall_u[side] = (np.full(n, u0), np.full(n, v0))
    prm = O.Params(dt=0.25 / 16, K=0.002, n=0.75, gamma_min=1e-4, eta_b=0.5)
    shape = (g.ny, g.nx)
    fhat, lam = O.initial_state(g, prm, np.full(shape, p0), np.full(shape, u0), np.full(shape, v0))
    f0 = fhat.copy()
    for _ in range(100):
        fhat, lam = O.step(fhat, lam, g, prm)
    assert np.abs(fhat - f0).max() < 1e-14


def test_lid_moves_along_the_top_edge():
    g = O.quad_grid(9, 7, SKEW)
    ux, uy = g.wall_u["top"]
    (x2, y2), (x3, y3) = SKEW[2], SKEW[3]
    t = np.array([x3 - x2, y3 - y2]) / math.hypot(x3 - x2, y3 - y2)
    assert np.allclose(ux[1:-1], 0.1 * t[0]) and np.allclose(uy[1:-1], 0.1 * t[1])
    assert ux[0] == ux[-1] == uy[0] == uy[-1] == 0.0


def test_contravariant_speed_maxima_sit_at_the_corners():
    """The library takes dt and the Courant number of a quadrilateral from its
    four corner nodes: along every grid line of the bilinear map c_xi and
    c_eta are ratios of linear functions to the positive, linear J, so
    max|c_xi|, max|c_eta| and max(|c_xi|/dxi + |c_eta|/deta) over the grid
    are attained at corners. Checked over every node of seeded quadrilaterals."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        d = rng.uniform(-0.25, 0.25, size=(4, 2))
        corners = tuple((x0 + d[k, 0], y0 + d[k, 1])
                        for k, (x0, y0) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))))
        g = O.quad_grid(31, 23, corners)
        axi, aeta = np.abs(g.cxi), np.abs(g.ceta)
        cfl = axi / g.dxi + aeta / g.deta
        for a in (axi, aeta, cfl):
            full = a.max()
            at_corners = max(a[:, j, i].max() for j in (0, -1) for i in (0, -1))
            assert at_corners >= full * (1 - 1e-14)

// Eddy centres of a steady cavity flow (Tables 1-3, Sec. 5.1): host code.
//
// The stream function psi (psi = 0 on the bottom wall, integrated along
// xi = const lines) has its minimum at the centre of the primary, clockwise
// eddy and local maxima at the centres of the counter-rotating eddies in the
// bottom corners. A centre is the extremum node refined by the stationary
// point of the least-squares quadratic over its 3 x 3 neighbourhood, then
// mapped to the physical plane by the trapezoid map of Eq. (3.8.1).
#include <cmath>
#include <cstring>

#include "ifdlbm.h"
#include "internal.h"

namespace {

double cot_of(double theta_deg) {
  if (theta_deg == 90.0) return 0.0;
  const double t = theta_deg * (M_PI / 180.0);
  return std::cos(t) / std::sin(t);
}

// Least-squares quadratic a + b s + c t + d s^2 + e s t + f t^2 over the
// nodes s, t in {-1, 0, 1}. With S = s^2 - 2/3 and T = t^2 - 2/3 the basis
// {1, s, t, S, s t, T} is orthogonal on the 3 x 3 stencil, so each
// coefficient is one projection: sum(s^2) = sum(t^2) = 6, sum(S^2) =
// sum(T^2) = 2, sum((s t)^2) = 4.
struct Quad {
  double a, b, c, d, e, f;
};

Quad fit3x3(const double *psi, int nx, int i, int j) {
  double m = 0, sb = 0, sc = 0, sd = 0, se = 0, sf = 0;
  for (int t = -1; t <= 1; ++t)
    for (int s = -1; s <= 1; ++s) {
      const double p = psi[(j + t) * nx + (i + s)];
      m += p;
      sb += s * p;
      sc += t * p;
      sd += (s * s - 2.0 / 3.0) * p;
      se += s * t * p;
      sf += (t * t - 2.0 / 3.0) * p;
    }
  Quad q;
  q.b = sb / 6.0;
  q.c = sc / 6.0;
  q.d = sd / 2.0;
  q.e = se / 4.0;
  q.f = sf / 2.0;
  q.a = m / 9.0 - (2.0 / 3.0) * (q.d + q.f);
  return q;
}

// Centre of an extremum at node (i, j); `minimum` selects the kind.
ifdlbm_eddy centre(const double *psi, int nx, int ny, ifdlbm_geometry g, int i, int j,
                   bool minimum) {
  ifdlbm_eddy e;
  std::memset(&e, 0, sizeof e);
  e.found = 1;
  e.i = i;
  e.j = j;
  const Quad q = fit3x3(psi, nx, i, j);
  // stationary point: [2d e; e 2f] [s; t] = -[b; c]
  const double A = 2 * q.d, B = q.e, C = 2 * q.f;
  const double det = A * C - B * B;
  double s = 0, t = 0;
  // a minimum needs a positive definite Hessian, a maximum a negative one
  const bool kind_ok = det > 0 && (minimum ? A > 0 : A < 0);
  if (kind_ok) {
    const double ss = (-q.b * C + q.c * B) / det;
    const double tt = (-q.c * A + q.b * B) / det;
    if (std::fabs(ss) <= 1.0 && std::fabs(tt) <= 1.0) {
      s = ss;
      t = tt;
      e.refined = 1;
    }
  }
  e.psi = q.a + q.b * s + q.c * t + q.d * s * s + q.e * s * t + q.f * t * t;
  if (!e.refined) e.psi = psi[j * nx + i];
  e.xi = (i + s) / double(nx - 1);
  e.eta = (j + t) / double(ny - 1);
  const double ct = cot_of(g.theta_deg);
  e.x = g.L * e.xi + g.H * ct * (1.0 - e.eta + 2.0 * e.xi * e.eta);   // Eq. (3.8.1)
  e.y = g.H * e.eta;
  return e;
}

bool strict_max(const double *psi, int nx, int i, int j) {
  const double p = psi[j * nx + i];
  for (int t = -1; t <= 1; ++t)
    for (int s = -1; s <= 1; ++s)
      if ((s || t) && !(p > psi[(j + t) * nx + (i + s)])) return false;
  return true;
}

}  // namespace

extern "C" int ifdlbm_find_eddies(int nx, int ny, ifdlbm_geometry g, const double *psi,
                                  ifdlbm_eddy out[3]) {
  if (nx < 3 || ny < 3 || !psi || !out)
    return ifd::set_global_error(IFDLBM_ERR_INVALID_ARG, "find_eddies: bad arguments");
  if (!(g.L > 0) || !(g.H > 0) || !(g.theta_deg > 0) || !(g.theta_deg <= 90))
    return ifd::set_global_error(IFDLBM_ERR_INVALID_ARG, "find_eddies: bad geometry");
  std::memset(out, 0, 3 * sizeof(ifdlbm_eddy));
  int pi = -1, pj = -1;
  int best[2][2] = {{-1, -1}, {-1, -1}};
  for (int j = 1; j <= ny - 2; ++j)
    for (int i = 1; i <= nx - 2; ++i) {
      const double p = psi[j * nx + i];
      if (!std::isfinite(p))
        return ifd::set_global_error(IFDLBM_ERR_INVALID_ARG, "find_eddies: non-finite psi");
      if (pi < 0 || p < psi[pj * nx + pi]) {
        pi = i;
        pj = j;
      }
      // corner eddies: eta <= 1/2, split at xi = 1/2
      if (2 * j <= ny - 1 && p > 0 && strict_max(psi, nx, i, j)) {
        const int side = (2 * i < nx - 1) ? 0 : 1;
        int *b = best[side];
        if (b[0] < 0 || p > psi[b[1] * nx + b[0]]) {
          b[0] = i;
          b[1] = j;
        }
      }
    }
  if (pi >= 0) out[0] = centre(psi, nx, ny, g, pi, pj, true);
  for (int side = 0; side < 2; ++side)
    if (best[side][0] >= 0) out[1 + side] = centre(psi, nx, ny, g, best[side][0], best[side][1], false);
  return IFDLBM_OK;
}

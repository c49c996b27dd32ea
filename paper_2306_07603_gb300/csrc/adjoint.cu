// Discrete adjoint (reverse mode) of one staged FP64 IFDLBM step.
//
// Forward step n (staged kernels; per node, deviation variables g):
//   K1  (u, v, P) = M(g), geq = E(u, v, P), Pi = sum c c (g - geq),
//       q = k^2 (Pxx^2 + 2 Pxy^2 + Pyy^2)/2, k = -2/((2 lam_p + dt) c_s^2),
//       lam = K/c_s^2 max(q, gmin^2)^((n-1)/2)                (Eqs. 1.4, 2.12-2.14)
//       FP = ap g + bp geq, FB = ab g + bb geq                (Eqs. 2.15-2.16)
//   K2  FBAR = FB - dt/2 A(FB), FH = ah FBAR + bh E(M(FBAR)) (Eqs. 3.7, 2.17)
//       wall b: FH(b) = X(FH(nb))                             (extrapolation)
//   K3  GN = FP - dt A(FH); wall b: GN(b) = X(GN(nb))         (Eq. 3.6, Step 6)
// with A_q = c_xi D_xi + c_eta D_eta the mixed scheme (Eqs. 2.5-2.7, 3.4) and
// X(F) = E(u_w, P(F)) + F - E(u(F), P(F)). Since dE/dP does not depend on u,
// X^T(G) = G - c (e_x ubar + e_y vbar) with (ubar, vbar) = (dE/du)^T G at u(F).
//
// The reverse sweep runs A3 walls -> A3 stencil gather -> A2 walls -> A2
// pointwise -> A2 stencil gather -> A1 pointwise, then reduces the parameter
// partials. Parameters: n (through K = U^(2-n) H^n / Re and the exponent),
// Re (through K) and theta in degrees (through c_xi of Eq. 3.4 via cot theta,
// and the Jacobian of the kinetic-energy objective of Eq. 5.1).
#include <cstdint>

#include "d2q9.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace ifd {

namespace {

struct Ref {
  int cav, i, j;
  bool valid;
};

__device__ __forceinline__ Ref tile_ref(const int *tile_cav, const CavDev *cavs) {
  Ref r;
  const int t = blockIdx.x;
  r.cav = tile_cav[t];
  const CavDev &cv = cavs[r.cav];
  const int lt = t - cv.tile0;
  r.i = (lt % cv.tiles_x) * TILE_X + threadIdx.x;
  r.j = (lt / cv.tiles_x) * TILE_Y + threadIdx.y;
  r.valid = r.i < cv.nx && r.j < cv.ny;
  return r;
}

__device__ __forceinline__ bool interior(const CavDev &cv, int i, int j) {
  return i >= 1 && i <= cv.nx - 2 && j >= 1 && j <= cv.ny - 2;
}

// (dE/d(u, v, P))^T eb at (ux, uy).
__device__ __forceinline__ void equilibrium_T(const double eb[9], double ux, double uy,
                                              const CavDev &cv, double &ub, double &vb,
                                              double &Pb) {
  const double c = cv.c, ics2 = cv.inv_cs2;
  ub = vb = Pb = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double cu = c * (ex(i) * ux + ey(i) * uy);
    const double w = wgt(i) * eb[i];
    const double tt = ics2 + cu * ics2 * ics2;
    ub += w * (c * ex(i) * tt - ux * ics2);
    vb += w * (c * ey(i) * tt - uy * ics2);
    Pb += wbar(i) * eb[i] * ics2;
  }
}

// gb += (dM/dg)^T (ub, vb, Pb) at (ux, uy), M the moments of Eqs. (2.10)-(2.11).
__device__ __forceinline__ void moments_T(double ub, double vb, double Pb, double ux, double uy,
                                          const CavDev &cv, double gb[9]) {
  const double c = cv.c;
  const double alpha = cv.cs2 / wbar(0), beta = wgt(0) / (2.0 * cv.cs2);
  const double A = ub + 2.0 * alpha * beta * ux * Pb, B = vb + 2.0 * alpha * beta * uy * Pb;
#pragma unroll
  for (int i = 0; i < 9; ++i) gb[i] += c * (ex(i) * A + ey(i) * B) - (i >= 1 ? alpha * Pb : 0.0);
}

// G <- X^T(G) at F (the wall rule's transpose; u(F) only).
__device__ __forceinline__ void nee_T(double G[9], const double F[9], const CavDev &cv) {
  double ux, uy, P;
  moments(F, cv.c, cv.cs2, ux, uy, P);
  double ub, vb, Pb;
  equilibrium_T(G, ux, uy, cv, ub, vb, Pb);
#pragma unroll
  for (int i = 0; i < 9; ++i) G[i] -= cv.c * (ex(i) * ub + ey(i) * vb);
}

// The distinct coefficients of the mixed difference of Eq. (2.5) (times 2 d)
// for blend eta, formed once per thread: eta, o = 1 - eta, 2 o, 3 o,
// eta + 2 o and eta + 4 o.
struct Blend {
  double e, o, o2, o3, e2, e4;
};
__device__ __forceinline__ Blend make_blend(double eta) {
  const double o = 1.0 - eta;
  return {eta, o, 2.0 * o, 3.0 * o, eta + 2.0 * o, eta + 4.0 * o};
}

// Coefficient of F[x + k] in the mixed difference of Eq. (2.5) at node x
// (times 2 d), for the upwind side `pos` and the near-wall flags lo / hi.
__device__ __forceinline__ double wmix(int k, bool pos, bool lo, bool hi, const Blend &b) {
  if (pos) {
    if (lo) return k == -1 ? -b.e2 : (k == 0 ? b.o2 : (k == 1 ? b.e : 0.0));
    return k == -2 ? b.o : (k == -1 ? -b.e4 : (k == 0 ? b.o3 : (k == 1 ? b.e : 0.0)));
  }
  if (hi) return k == -1 ? -b.e : (k == 0 ? -b.o2 : (k == 1 ? b.e2 : 0.0));
  return k == -1 ? -b.e : (k == 0 ? -b.o3 : (k == 1 ? b.e4 : (k == 2 ? -b.o : 0.0)));
}

__device__ __forceinline__ double cxi_at(const CavDev &cv, const Geo &g, int q, int i, int j) {
  const double A = cv.c * g.xix[cv.goff + j];
  return ex(q) * A - ey(q) * A * g.xeH[cv.goff + i];
}

// Per-node terms of c_{q xi} and of its theta derivative, formed once for all
// planes: with A = c xi_x and x_eta / H of the node, c_{q xi} = e_x A - e_y A
// x_eta / H (as cxi_at), and, through x_xi = L + 2 H cot eta and x_eta = H cot
// (2 xi - 1), d c_{q xi} / d theta_deg = e_y t1 - e_x t2 with
// t1 = (-A (2 xi - 1) + A x_eta/H K) dcot, t2 = A K dcot, K = 2 H eta xi_x.
struct NodeXi {
  double A, xe, t1, t2;
  __device__ __forceinline__ double cxi(int q) const { return ex(q) * A - ey(q) * A * xe; }
  __device__ __forceinline__ double dcxi(int q) const { return ey(q) * t1 - ex(q) * t2; }
};
__device__ __forceinline__ NodeXi node_xi(const CavDev &cv, const Geo &g, int i, int j) {
  const double xix = g.xix[cv.goff + j];
  const double A = cv.c * xix, xe = g.xeH[cv.goff + i];
  const double K = 2.0 * cv.H * (j * cv.deta) * xix;
  return {A, xe, (-A * (2.0 * (i * cv.dxi) - 1.0) + A * xe * K) * cv.dcot, A * K * cv.dcot};
}

// D_xi F_q at interior node (i, j) of plane F (as in the forward kernels), on
// the upwind side of c_{q xi} = cx.
__device__ __forceinline__ double dxi_with(const CavDev &cv, const double *F, double cx, int i,
                                           int j) {
  const int64_t node = int64_t(j) * cv.pitch + i;
  const int im2 = i >= 2 ? -2 : -1, ip2 = i <= cv.nx - 3 ? 2 : 1;
  return dmix2(F[node + im2], F[node - 1], F[node], F[node + 1], F[node + ip2], cx >= 0.0, i == 1,
               i == cv.nx - 2, cv.eta_b) * cv.inv2dxi;
}
__device__ __forceinline__ double dxi_at(const CavDev &cv, const Geo &g, const double *F, int q,
                                         int i, int j) {
  return dxi_with(cv, F, cxi_at(cv, g, q, i, j), i, j);
}

// Gather of the transposed advection: sum over interior x on the xi and eta
// lines through y of Gb_q(x) dA_q(x)/dF_q(y). c_{q xi}(x) is formed as in
// cxi_at (the row's metric c xi_x loaded once), so that its sign, which picks
// the upwind side, is the forward step's; the constant factors 1 / (2 dxi)
// and c_{q eta} / (2 deta) are applied to each line's sum.
__device__ __forceinline__ double advect_T(const CavDev &cv, const Geo &g, const double *Gb, int q,
                                           int i, int j, const Blend &bl) {
  double acc = 0.0;
  if (j >= 1 && j <= cv.ny - 2) {
    const double A = cv.c * g.xix[cv.goff + j];
    const double *row = Gb + int64_t(j) * cv.pitch;
    double sx = 0.0;
#pragma unroll
    for (int k = -2; k <= 2; ++k) {
      const int xi = i - k;  // F(y) = F(x + k)
      if (xi < 1 || xi > cv.nx - 2) continue;
      const double cx = ex(q) * A - ey(q) * A * g.xeH[cv.goff + xi];
      const double w = wmix(k, cx >= 0.0, xi == 1, xi == cv.nx - 2, bl);
      if (w != 0.0) sx += row[xi] * cx * w;
    }
    acc = sx * cv.inv2dxi;
  }
  const double ceta = double(ey(q)) * cv.c / cv.H;
  if (i >= 1 && i <= cv.nx - 2 && ceta != 0.0) {
    double se = 0.0;
#pragma unroll
    for (int k = -2; k <= 2; ++k) {
      const int yj = j - k;
      if (yj < 1 || yj > cv.ny - 2) continue;
      const double w = wmix(k, ceta >= 0.0, yj == 1, yj == cv.ny - 2, bl);
      if (w != 0.0) se += Gb[int64_t(yj) * cv.pitch + i] * w;
    }
    acc += se * (ceta * cv.inv2deta);
  }
  return acc;
}

// Adds sum over the wall nodes whose extrapolation source is interior node
// (i, j) of their adjoints, transposed through the wall rule at F(i, j).
__device__ __forceinline__ void wall_gather_T(const CavDev &cv, const double *Gplanes,
                                              const double *Fplanes, int i, int j, double out[9]) {
  double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  bool any = false;
  const int bi[3] = {i, i == 1 ? 0 : -1, i == cv.nx - 2 ? cv.nx - 1 : -1};
  const int bj[3] = {j, j == 1 ? 0 : -1, j == cv.ny - 2 ? cv.ny - 1 : -1};
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (a == 0 && b == 0) continue;
      const int wi = bi[a], wj = bj[b];
      if (wi < 0 || wj < 0) continue;
      const int64_t nd = int64_t(wj) * cv.pitch + wi;
#pragma unroll
      for (int q = 0; q < 9; ++q) G[q] += Gplanes[q * cv.plane + nd];
      any = true;
    }
  if (!any) return;
  const int64_t node = int64_t(j) * cv.pitch + i;
  double F[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = Fplanes[q * cv.plane + node];
  nee_T(G, F, cv);
#pragma unroll
  for (int q = 0; q < 9; ++q) out[q] += G[q];
}

__device__ __forceinline__ void tile_sum3(double a, double b, double c, double *ppart, int slot) {
  __shared__ double sh[TILE_X * TILE_Y / 32][3];
  const int lane = threadIdx.x + threadIdx.y * blockDim.x;
  const int w = lane >> 5, l = lane & 31;
  double v[3] = {a, b, c};
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (lane < 3) {
    double acc = 0.0;
    for (int k = 0; k < TILE_X * TILE_Y / 32; ++k) acc += sh[k][lane];
    ppart[int64_t(blockIdx.x) * 12 + slot * 3 + lane] = acc;
  }
}

}  // namespace

// Seed of the kinetic-energy objective (Eq. 5.1) at state g: adjoint of g,
// zero adjoint of lambda, and the direct theta partial (slot 3).
__global__ void k_adj_seed_energy(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  const CavDev &cv = a.cav[r.cav];
  double dth = 0.0;
  if (r.valid) {
    const int64_t node = int64_t(r.j) * cv.pitch + r.i;
    const double *g = a.g + 9 * cv.off;
    double gg[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) gg[q] = g[q * cv.plane + node];
    double ux, uy, P;
    moments(gg, cv.c, cv.cs2, ux, uy, P);
    const double wx = ((r.i == 0 || r.i == cv.nx - 1) ? 0.5 : 1.0) * cv.dxi;
    const double wy = ((r.j == 0 || r.j == cv.ny - 1) ? 0.5 : 1.0) * cv.deta;
    const double J = a.geo.xxi[cv.goff + r.j] * cv.H;
    double *ag = a.adj_g + 9 * cv.off;
#pragma unroll
    for (int q = 0; q < 9; ++q)
      ag[q * cv.plane + node] = wx * wy * J * cv.c * (ex(q) * ux + ey(q) * uy);
    a.adj_lam[cv.off + node] = 0.0;
    const double dJ = 2.0 * cv.H * cv.H * (r.j * cv.deta) * cv.dcot;
    dth = 0.5 * wx * wy * dJ * (ux * ux + uy * uy);
  }
  tile_sum3(0.0, 0.0, dth, a.ppart, 3);
}

// Seed of J = sum over cavities of psi(i*, j*), the stream function at one
// node per cavity (the primary eddy's node for J = psi_min). psi(i, j) =
// sum_{m <= j} w_m deta (u H - v x_eta(xi_i)) with trapezoid weights w_m
// (1/2 at m = 0 and m = j), so dJ/dg_q = w_m deta c (H e_qx - x_eta e_qy) on
// column i*, rows m <= j*, and zero elsewhere; theta enters directly through
// x_eta = H cot(theta) (2 xi - 1).
__global__ void k_adj_seed_psi(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  const CavDev &cv = a.cav[r.cav];
  double dth = 0.0;
  if (r.valid) {
    const int64_t node = int64_t(r.j) * cv.pitch + r.i;
    const int is = a.psi_nodes[2 * r.cav], js = a.psi_nodes[2 * r.cav + 1];
    double *ag = a.adj_g + 9 * cv.off;
    double w = 0.0;
    if (r.i == is && r.j <= js && js > 0) w = ((r.j == 0 || r.j == js) ? 0.5 : 1.0) * cv.deta;
    const double xe = a.geo.xeta[cv.goff + r.i];
#pragma unroll
    for (int q = 0; q < 9; ++q) ag[q * cv.plane + node] = w * cv.c * (cv.H * ex(q) - xe * ey(q));
    a.adj_lam[cv.off + node] = 0.0;
    if (w != 0.0) {
      const double *g = a.g + 9 * cv.off;
      double gg[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) gg[q] = g[q * cv.plane + node];
      double ux, uy, P;
      moments(gg, cv.c, cv.cs2, ux, uy, P);
      dth = -w * uy * cv.H * (2.0 * r.i * cv.dxi - 1.0) * cv.dcot;
    }
  }
  tile_sum3(0.0, 0.0, dth, a.ppart, 3);
}

// A3 walls: adjoint of g_{n+1} at interior nodes next to walls += X^T(walls).
__global__ void k_adj3_walls(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  if (!r.valid) return;
  const CavDev &cv = a.cav[r.cav];
  if (!interior(cv, r.i, r.j)) return;
  if (!(r.i == 1 || r.j == 1 || r.i == cv.nx - 2 || r.j == cv.ny - 2)) return;
  double *ag = a.adj_g + 9 * cv.off;
  double add[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  wall_gather_T(cv, ag, a.gn + 9 * cv.off, r.i, r.j, add);
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
#pragma unroll
  for (int q = 0; q < 9; ++q) a.fbarb[q * cv.plane + node + 9 * cv.off] = add[q];
}

// Applies the wall additions of k_adj3_walls (kept apart so that no thread
// reads a wall adjoint another thread has changed).
__global__ void k_adj_add(AdjArgs a, int which) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  if (!r.valid) return;
  const CavDev &cv = a.cav[r.cav];
  if (!interior(cv, r.i, r.j)) return;
  if (!(r.i == 1 || r.j == 1 || r.i == cv.nx - 2 || r.j == cv.ny - 2)) return;
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
  double *dst = (which == 0 ? a.adj_g : a.fhb) + 9 * cv.off;
  const double *add = a.fbarb + 9 * cv.off;
#pragma unroll
  for (int q = 0; q < 9; ++q) dst[q * cv.plane + node] += add[q * cv.plane + node];
}

// A3 stencil: FHbar(y) = -dt A^T(Gbar') for every node; theta partial (slot 0).
__global__ void k_adj3_stencil(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  const CavDev &cv = a.cav[r.cav];
  double dth = 0.0;
  if (r.valid) {
    const int64_t node = int64_t(r.j) * cv.pitch + r.i;
    const double *ag = a.adj_g + 9 * cv.off;
    const double *fh = a.fh + 9 * cv.off;
    double *fhb = a.fhb + 9 * cv.off;
    fhb[node] = 0.0;
    const Blend bl = make_blend(cv.eta_b);
#pragma unroll
    for (int q = 1; q < 9; ++q)
      fhb[q * cv.plane + node] = -cv.dt * advect_T(cv, a.geo, ag + q * cv.plane, q, r.i, r.j, bl);
    if (interior(cv, r.i, r.j)) {
      const NodeXi nm = node_xi(cv, a.geo, r.i, r.j);
#pragma unroll
      for (int q = 1; q < 9; ++q) {
        const double gb = ag[q * cv.plane + node];
        dth += -cv.dt * gb * nm.dcxi(q) * dxi_with(cv, fh + q * cv.plane, nm.cxi(q), r.i, r.j);
      }
    }
  }
  tile_sum3(0.0, 0.0, dth, a.ppart, 0);
}

// A2 walls: FHbar at interior nodes next to walls += X^T(FHbar at walls).
__global__ void k_adj2_walls(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  if (!r.valid) return;
  const CavDev &cv = a.cav[r.cav];
  if (!interior(cv, r.i, r.j)) return;
  if (!(r.i == 1 || r.j == 1 || r.i == cv.nx - 2 || r.j == cv.ny - 2)) return;
  double add[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  wall_gather_T(cv, a.fhb + 9 * cv.off, a.fh + 9 * cv.off, r.i, r.j, add);
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
#pragma unroll
  for (int q = 0; q < 9; ++q) a.fbarb[q * cv.plane + node + 9 * cv.off] = add[q];
}

// A2 pointwise at interior x: FBARbar = ah FHbar + M^T E^T (bh FHbar); lambda-bar of K2.
__global__ void k_adj2_point(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  if (!r.valid) return;
  const CavDev &cv = a.cav[r.cav];
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
  double *fbarb = a.fbarb + 9 * cv.off;
  if (!interior(cv, r.i, r.j)) {
#pragma unroll
    for (int q = 0; q < 9; ++q) fbarb[q * cv.plane + node] = 0.0;
    a.lamb2[cv.off + node] = 0.0;
    return;
  }
  const double *fh = a.fh + 9 * cv.off;
  const double *fhb = a.fhb + 9 * cv.off;
  const double lam = a.lam[cv.off + node];
  // f-bar(t + dt/2) of the node from the stored f(t + dt/2): Eq. (2.17),
  // f = f-bar + bh (f^eq - f-bar), keeps u and P, so f^eq is that of f and
  // f-bar = (f - bh f^eq) / ah, pointwise (no second evaluation of the
  // half step's stencil)
  double fhv[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) fhv[q] = fh[q * cv.plane + node];
  double ux, uy, P;
  moments(fhv, cv.c, cv.cs2, ux, uy, P);
  double geq[9];
  equilibrium(P, ux, uy, cv.c, cv.inv_cs2, geq);
  const double i4 = 1.0 / (4.0 * lam + cv.dt);
  const double ah = 4.0 * lam * i4, bh = cv.dt * i4;
  const double iah = (4.0 * lam + cv.dt) / (4.0 * lam);  // 1 / ah
  double fbar[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) fbar[q] = (fhv[q] - bh * geq[q]) * iah;
  double hb[9], eb[9], out[9];
  double lb = 0.0;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    hb[q] = fhb[q * cv.plane + node];
    eb[q] = bh * hb[q];
    out[q] = ah * hb[q];
    lb += hb[q] * (fbar[q] - geq[q]);
  }
  double ub, vb, Pb;
  equilibrium_T(eb, ux, uy, cv, ub, vb, Pb);
  moments_T(ub, vb, Pb, ux, uy, cv, out);
#pragma unroll
  for (int q = 0; q < 9; ++q) fbarb[q * cv.plane + node] = out[q];
  a.lamb2[cv.off + node] = 4.0 * cv.dt * i4 * i4 * lb;  // d ah / d lam = -d bh / d lam
}

// A2 stencil: FBbar(y) = FBARbar(y) - dt/2 A^T(FBARbar); theta partial (slot 1).
__global__ void k_adj2_stencil(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  const CavDev &cv = a.cav[r.cav];
  double dth = 0.0;
  if (r.valid) {
    const int64_t node = int64_t(r.j) * cv.pitch + r.i;
    const double *fbarb = a.fbarb + 9 * cv.off;
    const double *fb = a.fb + 9 * cv.off;
    double *fbb = a.fbb + 9 * cv.off;
    const double hdt = 0.5 * cv.dt;
    fbb[node] = fbarb[node];
    const Blend bl = make_blend(cv.eta_b);
#pragma unroll
    for (int q = 1; q < 9; ++q)
      fbb[q * cv.plane + node] = fbarb[q * cv.plane + node] -
                                 hdt * advect_T(cv, a.geo, fbarb + q * cv.plane, q, r.i, r.j, bl);
    if (interior(cv, r.i, r.j)) {
      const NodeXi nm = node_xi(cv, a.geo, r.i, r.j);
#pragma unroll
      for (int q = 1; q < 9; ++q)
        dth += -hdt * fbarb[q * cv.plane + node] * nm.dcxi(q) *
               dxi_with(cv, fb + q * cv.plane, nm.cxi(q), r.i, r.j);
    }
  }
  tile_sum3(0.0, 0.0, dth, a.ppart, 1);
}

// A1 pointwise: adjoint of (g_n, lambda_n); n and Re partials (slot 2).
__global__ void k_adj1(AdjArgs a) {
  const Ref r = tile_ref(a.tile_cav, a.cav);
  const CavDev &cv = a.cav[r.cav];
  double dn = 0.0, dRe = 0.0;
  if (r.valid) {
    const int64_t node = int64_t(r.j) * cv.pitch + r.i;
    const double *g = a.g + 9 * cv.off;
    double gg[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) gg[q] = g[q * cv.plane + node];
    const double lam_p = a.lam_p[cv.off + node];
    const double lam = a.lam[cv.off + node];
    double ux, uy, P;
    moments(gg, cv.c, cv.cs2, ux, uy, P);
    double geq[9], d[9];
    equilibrium(P, ux, uy, cv.c, cv.inv_cs2, geq);
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = gg[q] - geq[q];
    double pxx, pxy, pyy;
    second_moments(d, cv.c, pxx, pxy, pyy);
    const double D = 2.0 * lam_p + cv.dt;
    const double k = -2.0 / (D * cv.cs2);
    const double pp = pxx * pxx + 2.0 * pxy * pxy + pyy * pyy;
    const double q = 0.5 * k * k * pp;
    const bool free = q > cv.gmin2;
    const double qc = free ? q : cv.gmin2;

    const bool in = interior(cv, r.i, r.j);
    double *ag = a.adj_g + 9 * cv.off;
    const double *fbb = a.fbb + 9 * cv.off;
    double pb[9], bb_[9];
#pragma unroll
    for (int qq = 0; qq < 9; ++qq) {
      pb[qq] = in ? ag[qq * cv.plane + node] : 0.0;   // FPbar (FP is read at interior nodes only)
      bb_[qq] = fbb[qq * cv.plane + node];
    }
    const double i2 = 1.0 / (2.0 * lam + cv.dt);
    const double ap = (2.0 * lam - cv.dt) * i2, bp = 2.0 * cv.dt * i2;
    const double ab = (4.0 * lam - cv.dt) * 0.5 * i2, bb = 3.0 * cv.dt * 0.5 * i2;
    double sP = 0.0, sB = 0.0;
#pragma unroll
    for (int qq = 0; qq < 9; ++qq) {
      sP += pb[qq] * d[qq];
      sB += bb_[qq] * d[qq];
    }
    double lb = a.adj_lam[cv.off + node] + a.lamb2[cv.off + node] + 4.0 * cv.dt * i2 * i2 * sP +
                3.0 * cv.dt * i2 * i2 * sB;
    // lam = K/c_s^2 qc^m, m = (n-1)/2, K = U^(2-n) H^n / Re
    dn = lb * lam * (cv.lnHU + 0.5 * log(qc));
    dRe = -lb * lam / cv.Re;
    const double qb = free ? lb * cv.half_nm1 * lam / q : 0.0;
    const double k2 = k * k;
    const double pxxb = qb * k2 * pxx, pxyb = qb * k2 * 2.0 * pxy, pyyb = qb * k2 * pyy;
    const double kb = qb * k * pp;
    const double lam_pb = kb * 4.0 / (D * D * cv.cs2);
    const double c2 = cv.c * cv.c;
    double gb[9], geqb[9];
#pragma unroll
    for (int qq = 0; qq < 9; ++qq) {
      const double db = c2 * (ex(qq) * ex(qq) * pxxb + ex(qq) * ey(qq) * pxyb + ey(qq) * ey(qq) * pyyb);
      gb[qq] = ap * pb[qq] + ab * bb_[qq] + db;
      geqb[qq] = bp * pb[qq] + bb * bb_[qq] - db;
    }
    double ub, vb, Pb;
    equilibrium_T(geqb, ux, uy, cv, ub, vb, Pb);
    moments_T(ub, vb, Pb, ux, uy, cv, gb);
#pragma unroll
    for (int qq = 0; qq < 9; ++qq) ag[qq * cv.plane + node] = gb[qq];
    a.adj_lam[cv.off + node] = lam_pb;
  }
  tile_sum3(dn, dRe, 0.0, a.ppart, 2);
}

// Per cavity: dparams[cav][0..2] += sums over its tiles of the four slots.
__global__ void k_adj_reduce(const CavDev *cavs, const double *ppart, double *dparams) {
  const CavDev &cv = cavs[blockIdx.x];
  __shared__ double sh[128][3];
  double acc[3] = {0, 0, 0};
  for (int t = threadIdx.x; t < cv.nparts; t += blockDim.x)
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[k] += ppart[int64_t(cv.tile0 + t) * 12 + s * 3 + k];
#pragma unroll
  for (int k = 0; k < 3; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 3; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + w][k];
    __syncthreads();
  }
  if (threadIdx.x < 3) dparams[3 * blockIdx.x + threadIdx.x] += sh[0][threadIdx.x];
}

static const dim3 kT(TILE_X, TILE_Y);

void launch_adjoint_seed(const AdjArgs &a, int ntiles, int ncav, double *dparams, cudaStream_t s) {
  cudaMemsetAsync(a.ppart, 0, size_t(ntiles) * 12 * sizeof(double), s);
  k_adj_seed_energy<<<ntiles, kT, 0, s>>>(a);
  k_adj_reduce<<<ncav, 128, 0, s>>>(a.cav, a.ppart, dparams);
}

void launch_adjoint_seed_psi(const AdjArgs &a, int ntiles, int ncav, double *dparams,
                             cudaStream_t s) {
  cudaMemsetAsync(a.ppart, 0, size_t(ntiles) * 12 * sizeof(double), s);
  k_adj_seed_psi<<<ntiles, kT, 0, s>>>(a);
  k_adj_reduce<<<ncav, 128, 0, s>>>(a.cav, a.ppart, dparams);
}

void launch_adjoint_step(const AdjArgs &a, int ntiles, int ncav, double *dparams, cudaStream_t s) {
  cudaMemsetAsync(a.ppart, 0, size_t(ntiles) * 12 * sizeof(double), s);
  k_adj3_walls<<<ntiles, kT, 0, s>>>(a);
  k_adj_add<<<ntiles, kT, 0, s>>>(a, 0);
  k_adj3_stencil<<<ntiles, kT, 0, s>>>(a);
  k_adj2_walls<<<ntiles, kT, 0, s>>>(a);
  k_adj_add<<<ntiles, kT, 0, s>>>(a, 1);
  k_adj2_point<<<ntiles, kT, 0, s>>>(a);
  k_adj2_stencil<<<ntiles, kT, 0, s>>>(a);
  k_adj1<<<ntiles, kT, 0, s>>>(a);
  k_adj_reduce<<<ncav, 128, 0, s>>>(a.cav, a.ppart, dparams);
}

}  // namespace ifd

// Staged IFDLBM step: three launches per time step, no recomputation.
//
//   k_collide  every node: Step (2) (moments, f^eq, lagged power-law lam),
//              Step (3) f-hat^+ (Eq. 2.15) and f-bar^+ (Eq. 2.16)
//   k_half     every node: Step (4) half step f-bar(t+dt/2) (Eq. 3.7), its
//              moments and f(t+dt/2) (Eq. 2.17); wall nodes by
//              non-equilibrium extrapolation from their inner neighbour
//   k_full     every node: Step (5) f-hat(t+dt) (Eq. 3.6); wall nodes by
//              non-equilibrium extrapolation (Step 6); residual partials of
//              Eq. (2.19) and Eq. (5.1)
//
// On GB300 the FP64 pipe runs at a small fraction of the FP32 rate, so the
// FP64 step is bound by FP64 instructions, not bytes: this organisation
// keeps every node's arithmetic to exactly one evaluation and pays with
// intermediate planes (f-bar^+, f-hat^+, f(t+dt/2)) that stay in L2 for
// the grid sizes of a cavity sweep.
//
// A wall node (i, j) takes its neighbour (clamp(i, 1, nx-2), clamp(j, 1,
// ny-2)): the adjacent node along the grid normal on a side, the diagonal
// node at a corner. The lid nodes 0 < i < nx-1 of row ny-1 move at (U, 0);
// every other wall node, the two top corners included, is at rest.
#include <cstdint>

#include "d2q9.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace ifd {

struct NodeRef {
  int cav, i, j;
  bool valid;
};

__device__ __forceinline__ NodeRef tile_node(const int *tile_cav, const CavDev *cavs) {
  NodeRef r;
  const int t = blockIdx.x;
  r.cav = tile_cav[t];
  const CavDev &cv = cavs[r.cav];
  const int lt = t - cv.tile0;
  r.i = (lt % cv.tiles_x) * TILE_X + threadIdx.x;
  r.j = (lt / cv.tiles_x) * TILE_Y + threadIdx.y;
  r.valid = r.i < cv.nx && r.j < cv.ny;
  return r;
}

template <class T>
__device__ __forceinline__ void load9(const T *base, int64_t plane, int64_t node, T v[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) v[q] = base[q * plane + node];
}

template <class T>
__device__ __forceinline__ void store9(T *base, int64_t plane, int64_t node, const T v[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) base[q * plane + node] = v[q];
}

// ---------------------------------------------------------------------------
// Step (2)-(3): collision-side transforms, pointwise
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_collide(StepArgs a) {
  const NodeRef r = tile_node(a.tile_cav, a.cav);
  if (!r.valid) return;
  const CavDev &cv = a.cav[r.cav];
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
  const int64_t b9 = 9 * cv.off;
  T g[9];
  load9((const T *)a.g_in + b9, cv.plane, node, g);
  const double lam_prev = double(((const T *)a.lam_in)[cv.off + node]);

  const T c = T(cv.c), cs2 = T(cv.cs2), ics2 = T(cv.inv_cs2);
  T ux, uy, P;
  moments(g, c, cs2, ux, uy, P);                 // Eqs. (2.10)-(2.11)
  T geq[9];
  equilibrium(P, ux, uy, c, ics2, geq);          // Eq. (2.8)
  T d[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) d[q] = g[q] - geq[q];
  T pxx, pxy, pyy;
  second_moments(d, c, pxx, pxy, pyy);
  const double lam = relaxation_time(pxx, pxy, pyy, lam_prev, cv, a.powtab,
                                     a.powt + int64_t(r.cav) * POWT_SIZE);
  const T L = T(lam), dt = T(cv.dt);
  ((T *)a.lam_out)[cv.off + node] = L;           // lam(t), also next lam_prev

  const T i2 = T(1) / (T(2) * L + dt);
  const T bp = T(2) * dt * i2;     // Eq. (2.15): (2 lam - dt)/(2 lam + dt) = 1 - bp
  const T bb = T(1.5) * dt * i2;   // Eq. (2.16): 3 dt/(4 lam + 2 dt), (4 lam - dt)/(4 lam + 2 dt) = 1 - bb
  T *fp = (T *)a.fp + b9;
  T *fb = (T *)a.fb + b9;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    fp[q * cv.plane + node] = toward(g[q], geq[q], bp);
    fb[q * cv.plane + node] = toward(g[q], geq[q], bb);
  }
  double *m0 = a.m0 + 3 * cv.off;
  m0[node] = double(ux);
  m0[cv.plane + node] = double(uy);
  m0[2 * cv.plane + node] = double(P);
}

// Advection term (c_{q xi} D_xi + c_{q eta} D_eta) F_q at interior node
// (i, j) of plane F (Eqs. 3.4-3.7 with the mixed scheme of Eq. 2.5).
template <class T>
__device__ __forceinline__ T advect(const T *F, int64_t node, int pitch, int i, int j, int nx,
                                    int ny, T cxi, T ceta, const CavDev &cv) {
  // clamped neighbour offsets: the clamped values are never used
  const int im2 = i >= 2 ? -2 : -1, ip2 = i <= nx - 3 ? 2 : 1;
  const int jm2 = j >= 2 ? -2 : -1, jp2 = j <= ny - 3 ? 2 : 1;
  const T f0 = F[node];
  const T eta_b = T(cv.eta_b);
  const T dxi = dmix2(F[node + im2], F[node - 1], f0, F[node + 1], F[node + ip2], cxi >= T(0),
                      i == 1, i == nx - 2, eta_b) * T(cv.inv2dxi);
  const int64_t p = pitch;
  const T deta = dmix2(F[node + jm2 * p], F[node - p], f0, F[node + p], F[node + jp2 * p],
                       ceta >= T(0), j == 1, j == ny - 2, eta_b) * T(cv.inv2deta);
  return cxi * dxi + ceta * deta;
}

__device__ __forceinline__ void wall_neighbour(const CavDev &cv, int i, int j, int &ii, int &jj,
                                               bool &wall, double &uwx, double &uwy) {
  wall = (i == 0) | (j == 0) | (i == cv.nx - 1) | (j == cv.ny - 1);
  ii = min(max(i, 1), cv.nx - 2);
  jj = min(max(j, 1), cv.ny - 2);
  const bool lid = j == cv.ny - 1 && i > 0 && i < cv.nx - 1;
  uwx = lid ? cv.lid_ux : 0.0;
  uwy = lid ? cv.lid_uy : 0.0;
}

// Contravariant velocities of Eq. (3.4) at a node. GEN = false: the
// separable trapezoid metrics (A = c xi_x(eta), B = A x_eta(xi)/H,
// c_eta = c e_y / H); GEN = true: the per-node metric planes of a general
// quadrilateral (a handle holds one kind only, so the kind is a template
// parameter and the trapezoid kernels carry no trace of the general one).
template <bool GEN>
struct NodeMetrics {
  double a, b, c, d;  // A, B, c/H, - (trapezoid); c xi_x, c xi_y, c eta_x, c eta_y (general)
};
template <bool GEN>
__device__ __forceinline__ NodeMetrics<GEN> node_metrics(const CavDev &cv, const Geo &geo, int ii,
                                                         int jj, int64_t node) {
  NodeMetrics<GEN> m;
  if constexpr (GEN) {
    const double *gm = geo.gmet + 7 * cv.off;
    m.a = cv.c * gm[node];
    m.b = cv.c * gm[cv.plane + node];
    m.c = cv.c * gm[2 * cv.plane + node];
    m.d = cv.c * gm[3 * cv.plane + node];
  } else {
    m.a = cv.c * geo.xix[cv.goff + jj];
    m.b = m.a * geo.xeH[cv.goff + ii];
    m.c = cv.c / cv.H;
    m.d = 0.0;
  }
  return m;
}
template <bool GEN>
__device__ __forceinline__ void contravariant(const NodeMetrics<GEN> &m, int q, double &cxi,
                                              double &ceta) {
  if constexpr (GEN) {
    cxi = ex(q) * m.a + ey(q) * m.b;
    ceta = ex(q) * m.c + ey(q) * m.d;
  } else {
    cxi = cxi_of(q, m.a, m.b);
    ceta = ey(q) * m.c;
  }
}

// ---------------------------------------------------------------------------
// Step (4): half step and f(t + dt/2)
// ---------------------------------------------------------------------------
// f(t + dt/2) at interior node (ii, jj): the half step of Eq. (3.7) from
// f-bar^+, then Eq. (2.17) with the node's lambda(t).
template <class T, bool GEN>
__device__ __forceinline__ void half_at(const StepArgs &a, const CavDev &cv, int ii, int jj,
                                        T fh[9]) {
  const T *fb = (const T *)a.fb + 9 * cv.off;
  const int64_t node = int64_t(jj) * cv.pitch + ii;
  const T lam = ((const T *)a.lam_out)[cv.off + node];
  const NodeMetrics<GEN> met = node_metrics<GEN>(cv, a.geo, ii, jj, node);
  const T hdt = T(0.5 * cv.dt);
  T fbar[9];
  fbar[0] = fb[node];
#pragma unroll
  for (int q = 1; q < 9; ++q) {
    const T *F = fb + q * cv.plane;
    double cx, ce;
    contravariant(met, q, cx, ce);
    fbar[q] = F[node] - hdt * advect(F, node, cv.pitch, ii, jj, cv.nx, cv.ny, T(cx), T(ce), cv);
  }
  const T c = T(cv.c), cs2 = T(cv.cs2), ics2 = T(cv.inv_cs2);
  T ux, uy, P;
  moments(fbar, c, cs2, ux, uy, P);              // Eqs. (2.10)-(2.11) on f-bar
  T geq[9];
  equilibrium(P, ux, uy, c, ics2, geq);
  const T L = T(lam), dt = T(cv.dt);
  const T bh = dt / (T(4) * L + dt);             // Eq. (2.17): 4 lam/(4 lam + dt) = 1 - bh
#pragma unroll
  for (int q = 0; q < 9; ++q) fh[q] = toward(fbar[q], geq[q], bh);
}

// Pressure of a deviation set (Eq. 2.11).
template <class T>
__device__ __forceinline__ T pressure_of(const T g[9], const CavDev &cv) {
  T ux, uy, P;
  moments(g, T(cv.c), T(cv.cs2), ux, uy, P);
  return P;
}

// Wall value from the inner neighbour's F (in F on entry). Zeroth-order wall
// pressure: P_b = P_nb. First order (cv.wallp): P_b = 2 P_nb - P_nnb with
// F2 the same quantity at the next node beyond the neighbour.
template <class T>
__device__ __forceinline__ void wall_rule(T F[9], const T F2[9], bool first, double uwx,
                                          double uwy, const CavDev &cv) {
  if (!first) {
    nee(F, T(uwx), T(uwy), cv);
    return;
  }
  const T Pb = T(2) * pressure_of(F, cv) - pressure_of(F2, cv);
  nee_p(F, T(uwx), T(uwy), Pb, T(cv.c), T(cv.cs2), T(cv.inv_cs2));
}

template <class T, bool GEN>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_half(StepArgs a) {
  const NodeRef r = tile_node(a.tile_cav, a.cav);
  if (!r.valid) return;
  const CavDev &cv = a.cav[r.cav];
  int ii, jj;
  bool wall;
  double uwx, uwy;
  wall_neighbour(cv, r.i, r.j, ii, jj, wall, uwx, uwy);
  T fh[9];
  half_at<T, GEN>(a, cv, ii, jj, fh);
  if (wall) {
    T f2[9];
    if (cv.wallp) half_at<T, GEN>(a, cv, 2 * ii - r.i, 2 * jj - r.j, f2);
    wall_rule(fh, f2, cv.wallp != 0, uwx, GEN ? uwy : 0.0, cv);
  }
  store9((T *)a.fh + 9 * cv.off, cv.plane, int64_t(r.j) * cv.pitch + r.i, fh);
}

// ---------------------------------------------------------------------------
// Steps (5)-(6): full step, wall nodes, residual partials
// ---------------------------------------------------------------------------
// f-hat(t + dt) at interior node (ii, jj): the full step of Eq. (3.6).
template <class T, bool GEN>
__device__ __forceinline__ void full_at(const StepArgs &a, const CavDev &cv, int ii, int jj,
                                        T gn[9]) {
  const int64_t b9 = 9 * cv.off;
  const T *fh = (const T *)a.fh + b9;
  const T *fp = (const T *)a.fp + b9;
  const int64_t node = int64_t(jj) * cv.pitch + ii;
  const NodeMetrics<GEN> met = node_metrics<GEN>(cv, a.geo, ii, jj, node);
  const T dt = T(cv.dt);
  gn[0] = fp[node];
#pragma unroll
  for (int q = 1; q < 9; ++q) {
    const T *F = fh + q * cv.plane;
    double cx, ce;
    contravariant(met, q, cx, ce);
    gn[q] = fp[q * cv.plane + node] -
            dt * advect(F, node, cv.pitch, ii, jj, cv.nx, cv.ny, T(cx), T(ce), cv);  // Eq. (3.6)
  }
}

template <class T, bool GEN>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_full(StepArgs a) {
  const NodeRef r = tile_node(a.tile_cav, a.cav);
  const CavDev &cv = a.cav[r.cav];
  Partial p = {0, 0, 0, 0, 0, 0, 0};
  if (r.valid) {
    int ii, jj;
    bool wall;
    double uwx, uwy;
    wall_neighbour(cv, r.i, r.j, ii, jj, wall, uwx, uwy);
    const int64_t b9 = 9 * cv.off;
    T gn[9];
    full_at<T, GEN>(a, cv, ii, jj, gn);
    if (wall) {
      T g2[9];
      if (cv.wallp) full_at<T, GEN>(a, cv, 2 * ii - r.i, 2 * jj - r.j, g2);
      wall_rule(gn, g2, cv.wallp != 0, uwx, GEN ? uwy : 0.0, cv);
    }
    const int64_t me = int64_t(r.j) * cv.pitch + r.i;
    store9((T *)a.g_out + b9, cv.plane, me, gn);

    T ux, uy, P;
    moments(gn, T(cv.c), T(cv.cs2), ux, uy, P);
    const double u1 = double(ux), v1 = double(uy), P1 = double(P);
    if (!(isfinite(u1) && isfinite(v1))) atomicOr(a.status, 1u);
    if (a.want_residual) {
      const double *m0 = a.m0 + 3 * cv.off;
      const double du = u1 - m0[me], dv = v1 - m0[cv.plane + me], dP = P1 - m0[2 * cv.plane + me];
      p.du2 = du * du + dv * dv;
      p.u2 = u1 * u1 + v1 * v1;
      p.dP2 = dP * dP;
      const double Pfull = P1 + a.pref[r.cav];   // P of the deviations plus their reference
      p.P2 = Pfull * Pfull;
      p.du2max = p.du2;
      p.u2max = p.u2;
      const double wx = ((r.i == 0 || r.i == cv.nx - 1) ? 0.5 : 1.0) * cv.dxi;
      const double wy = ((r.j == 0 || r.j == cv.ny - 1) ? 0.5 : 1.0) * cv.deta;
      double J;
      if constexpr (GEN)
        J = a.geo.gmet[7 * cv.off + 6 * cv.plane + me];
      else
        J = a.geo.xxi[cv.goff + r.j] * cv.H;
      p.ek = 0.5 * wx * wy * J * p.u2;  // Eq. (5.1)
    }
  }
  if (a.want_residual) block_partial<TILE_X * TILE_Y / 32>(p, a.part, blockIdx.x);
}

// One block per cavity: fixed-order reduction of that cavity's partials.
__global__ void k_residual_reduce(const CavDev *cavs, const double *part, double *resid) {
  const CavDev &cv = cavs[blockIdx.x];
  reduce_partials(part + int64_t(cv.part0) * NPART, cv.nparts, resid + 4 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// Initial state (Step 1), macros / stream function, state import and export
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_init(const CavDev *cavs, const int *tile_cav,
                                                          T *g, T *lam) {
  const NodeRef r = tile_node(tile_cav, cavs);
  if (!r.valid) return;
  const CavDev &cv = cavs[r.cav];
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
  const bool lid = r.j == cv.ny - 1 && r.i > 0 && r.i < cv.nx - 1;
  T geq[9];
  equilibrium(T(0), lid ? T(cv.lid_ux) : T(0), lid ? T(cv.lid_uy) : T(0), T(cv.c),
              T(cv.inv_cs2), geq);
  store9(g + 9 * cv.off, cv.plane, node, geq);
  lam[cv.off + node] = T(cv.lam0);
}

// Macros at every node and the stream function. A block is 32 xi = const
// lines x MSEG row segments. Pass 1: rho, u, v and the integrand
// I = u y_eta - v x_eta at every node (I parked in psi). Pass 2: each thread
// sums the trapezoid intervals (I_j + I_{j-1}) deta / 2 of its segment. The
// segment sums are scanned in a fixed order in shared memory, and pass 3
// writes psi_j = psi_{j-1} + (I_j + I_{j-1}) deta / 2 from the segment's
// offset (psi = 0 on the bottom wall).
constexpr int MSEG = 32;

template <class T>
__global__ void __launch_bounds__(32 * MSEG)
    k_macros(const CavDev *cavs, Geo geo, int cavity, const double *pref, const T *g,
             double *rho, double *u, double *v, double *psi) {
  const CavDev &cv = cavs[cavity];
  const double p0 = pref[cavity];
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int seg = (cv.ny + MSEG - 1) / MSEG;
  const int j0 = threadIdx.y * seg, j1 = min(cv.ny, j0 + seg);
  const bool col = i < cv.nx;
  const T *gb = g + 9 * cv.off;
  const double *gm = cv.general ? geo.gmet + 7 * cv.off : nullptr;
  __shared__ double part[MSEG][32];
  for (int j = j0; col && j < j1; ++j) {
    T gg[9];
    load9(gb, cv.plane, int64_t(j) * cv.pitch + i, gg);
    T ux, uy, P;
    moments(gg, T(cv.c), T(cv.cs2), ux, uy, P);
    const int64_t o = int64_t(j) * cv.nx + i;
    if (rho) rho[o] = cv.rho0 + (p0 + double(P)) * cv.inv_cs2;
    if (u) u[o] = double(ux);
    if (v) v[o] = double(uy);
    const int64_t nd = int64_t(j) * cv.pitch + i;
    if (psi)
      psi[o] = cv.general ? double(ux) * gm[5 * cv.plane + nd] - double(uy) * gm[4 * cv.plane + nd]
                          : double(ux) * cv.H - double(uy) * geo.xeta[cv.goff + i];
  }
  if (!psi) return;  // uniform over the launch
  __syncthreads();   // every integrand of the block's lines is written
  double sum = 0.0, Iprev = 0.0;
  if (col && j0 < j1) {
    Iprev = j0 > 0 ? psi[int64_t(j0 - 1) * cv.nx + i] : 0.0;
    double Ip = Iprev;
    for (int j = j0; j < j1; ++j) {
      const double I = psi[int64_t(j) * cv.nx + i];
      if (j > 0) sum += 0.5 * (I + Ip) * cv.deta;
      Ip = I;
    }
  }
  part[threadIdx.y][threadIdx.x] = sum;
  __syncthreads();   // segment sums published; every integrand has been read
  double acc = 0.0;
  for (int k = 0; k < int(threadIdx.y); ++k) acc += part[k][threadIdx.x];
  for (int j = j0; col && j < j1; ++j) {
    const int64_t o = int64_t(j) * cv.nx + i;
    const double I = psi[o];
    if (j > 0) acc += 0.5 * (I + Iprev) * cv.deta;
    Iprev = I;
    psi[o] = acc;
  }
}

// Probes: u, v, P (Eqs. 2.10-2.11, P including the reference pressure of the
// stored deviations) at n nodes given as (cavity, i, j); a probe outside its
// cavity (or naming no cavity) gets NaN.
template <class T>
__global__ void k_probe(const CavDev *cavs, int ncav, const double *pref, const T *g, int n,
                        const int *probes, double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int c = probes[3 * k], i = probes[3 * k + 1], j = probes[3 * k + 2];
  if (c < 0 || c >= ncav || i < 0 || j < 0 || i >= cavs[c].nx || j >= cavs[c].ny) {
    out[3 * k] = out[3 * k + 1] = out[3 * k + 2] = nan("");
    return;
  }
  const CavDev &cv = cavs[c];
  T gg[9];
  load9(g + 9 * cv.off, cv.plane, int64_t(j) * cv.pitch + i, gg);
  T ux, uy, P;
  moments(gg, T(cv.c), T(cv.cs2), ux, uy, P);
  out[3 * k] = double(ux);
  out[3 * k + 1] = double(uy);
  out[3 * k + 2] = pref[c] + double(P);
}

template <class T>
__global__ void k_export(const CavDev *cavs, int cavity, const double *pref, const T *g,
                         const T *lam, double *fhat, double *lamo) {
  const CavDev &cv = cavs[cavity];
  const double pt = pref[cavity] * cv.inv_cs2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= cv.nx) return;
  const int64_t node = int64_t(j) * cv.pitch + i, o = int64_t(j) * cv.nx + i;
  const int64_t n2 = int64_t(cv.nx) * cv.ny;
  if (fhat)
#pragma unroll
    for (int q = 0; q < 9; ++q)
      fhat[q * n2 + o] = double(g[9 * cv.off + q * cv.plane + node]) + wgt(q) * cv.rho0 +
                         wbar(q) * pt;
  if (lamo) lamo[o] = double(lam[cv.off + node]);
}

template <class T>
__global__ void k_import(const CavDev *cavs, int cavity, const double *pref, T *g, T *lam,
                         const double *fhat, const double *lami) {
  const CavDev &cv = cavs[cavity];
  const double pt = pref[cavity] * cv.inv_cs2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= cv.nx) return;
  const int64_t node = int64_t(j) * cv.pitch + i, o = int64_t(j) * cv.nx + i;
  const int64_t n2 = int64_t(cv.nx) * cv.ny;
#pragma unroll
  for (int q = 0; q < 9; ++q)
    g[9 * cv.off + q * cv.plane + node] = T(fhat[q * n2 + o] - wgt(q) * cv.rho0 - wbar(q) * pt);
  lam[cv.off + node] = T(lami[o]);
}

// Re-basing of the stored deviations on the mean pressure (FP32 storage):
// a uniform pressure offset is a neutral mode of the scheme that drifts, and
// carrying it in every g_i would make the FP32 rounding of g grow with it.
// k_psum: per tile, sum of P(g) in FP64; k_pshift: per cavity, the mean
// (fixed-order sum over its tiles) into ptile[ntiles + k], pref += mean;
// k_rebase: g_i -= wbar_i mean / c_s^2 at every node (one rounding).
template <class T>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_psum(const CavDev *cavs, const int *tile_cav,
                                                          const T *g, double *ptile) {
  const NodeRef r = tile_node(tile_cav, cavs);
  const CavDev &cv = cavs[r.cav];
  double v = 0.0;
  if (r.valid) {
    T gg[9];
    load9(g + 9 * cv.off, cv.plane, int64_t(r.j) * cv.pitch + r.i, gg);
    T ux, uy, P;
    moments(gg, T(cv.c), T(cv.cs2), ux, uy, P);
    v = double(P);
  }
  __shared__ double sh[TILE_X * TILE_Y];
  const int t = threadIdx.y * TILE_X + threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int w = TILE_X * TILE_Y / 2; w > 0; w >>= 1) {
    if (t < w) sh[t] += sh[t + w];
    __syncthreads();
  }
  if (t == 0) ptile[blockIdx.x] = sh[0];
}

__global__ void k_pshift(const CavDev *cavs, int ntiles, double *ptile, double *pref) {
  const CavDev &cv = cavs[blockIdx.x];
  const int n = cv.tiles_x * cv.tiles_y;
  __shared__ double sh[256];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += ptile[cv.tile0 + k];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mean = sh[0] / (double(cv.nx) * cv.ny);
    ptile[ntiles + blockIdx.x] = mean;
    pref[blockIdx.x] += mean;
  }
}

template <class T>
__global__ void __launch_bounds__(TILE_X *TILE_Y) k_rebase(const CavDev *cavs, const int *tile_cav,
                                                            T *g, const double *ptile, int ntiles) {
  const NodeRef r = tile_node(tile_cav, cavs);
  if (!r.valid) return;
  const CavDev &cv = cavs[r.cav];
  const double pt = ptile[ntiles + r.cav] * cv.inv_cs2;
  T *gb = g + 9 * cv.off;
  const int64_t node = int64_t(r.j) * cv.pitch + r.i;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    T &x = gb[q * cv.plane + node];
    x = T(double(x) - wbar(q) * pt);
  }
}

__global__ void k_pow_selftest(int n, const double *x, double m, const double *tab, double *fast,
                               double *ref) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  fast[k] = pow_fast(x[k], m, tab);
  ref[k] = pow(x[k], m);
}

void launch_pow_selftest(int n, const double *x, double m, const double *tab, double *fast,
                         double *ref, cudaStream_t s) {
  k_pow_selftest<<<(n + 255) / 256, 256, 0, s>>>(n, x, m, tab, fast, ref);
}

// pow_tab on the FP32 roundings of x (tab: a cavity table of exponent m and
// factor C); out[k] = pow_tab(float(x[k])) and out[n + k] = C * CUDA's
// pow(double(float(x[k])), m).
__global__ void k_pow_tab_selftest(int n, const double *x, double m, double C, const double *tab,
                                   double b2, float b3, float b4, float b5, double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float xf = float(x[k]);
  out[k] = pow_tab(xf, tab, m, b2, b3, b4, b5);
  out[n + k] = C * pow(double(xf), m);
}

void launch_pow_tab_selftest(int n, const double *x, double m, double C, const double *tab,
                             double b2, float b3, float b4, float b5, double *out, cudaStream_t s) {
  k_pow_tab_selftest<<<(n + 255) / 256, 256, 0, s>>>(n, x, m, C, tab, b2, b3, b4, b5, out);
}

__global__ void k_pow_f32_selftest(int n, const double *x, double m, double *out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[k] = double(pow_f32(float(x[k]), float(m)));
}

// Per-node metric planes of the general quadrilaterals, one thread per node
// (blockIdx.y = cavity).
__global__ void k_quad_metrics(const CavDev *cavs, const double *corners, double *gmet) {
  const CavDev &cv = cavs[blockIdx.y];
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= int64_t(cv.nx) * cv.ny) return;
  const int j = int(n / cv.nx), i = int(n - int64_t(j) * cv.nx);
  double m[7];
  quad_node_metrics(corners + 8 * blockIdx.y, double(i) / (cv.nx - 1), double(j) / (cv.ny - 1), m);
  double *gm = gmet + 7 * cv.off;
  const int64_t node = int64_t(j) * cv.pitch + i;
#pragma unroll
  for (int t = 0; t < 7; ++t) gm[t * cv.plane + node] = m[t];
}

// FP32 roundings of c xi_x, c xi_y, c eta_x, c eta_y and J (formed in FP64 by
// k_quad_metrics), one thread per node (blockIdx.y = cavity).
__global__ void k_quad_metrics_f32(const CavDev *cavs, const double *gmet, float *qmet_f) {
  const CavDev &cv = cavs[blockIdx.y];
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= int64_t(cv.nx) * cv.ny) return;
  const int j = int(n / cv.nx), i = int(n - int64_t(j) * cv.nx);
  const int64_t node = int64_t(j) * cv.pitch + i;
  const double *gm = gmet + 7 * cv.off;
  float *qm = qmet_f + 5 * cv.off;
#pragma unroll
  for (int t = 0; t < 4; ++t) qm[t * cv.plane + node] = float(cv.c * gm[t * cv.plane + node]);
  qm[4 * cv.plane + node] = float(gm[6 * cv.plane + node]);
}

void launch_quad_metrics_f32(const CavDev *cav, int ncav, int64_t max_n2, const double *gmet,
                             float *qmet_f, cudaStream_t s) {
  const dim3 grid(unsigned((max_n2 + 255) / 256), unsigned(ncav));
  k_quad_metrics_f32<<<grid, 256, 0, s>>>(cav, gmet, qmet_f);
}

void launch_quad_metrics(const CavDev *cav, int ncav, int64_t max_n2, const double *corners,
                         double *gmet, cudaStream_t s) {
  const dim3 grid(unsigned((max_n2 + 255) / 256), unsigned(ncav));
  k_quad_metrics<<<grid, 256, 0, s>>>(cav, corners, gmet);
}

void launch_pow_f32_selftest(int n, const double *x, double m, double *out, cudaStream_t s) {
  k_pow_f32_selftest<<<(n + 255) / 256, 256, 0, s>>>(n, x, m, out);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static const dim3 kTile(TILE_X, TILE_Y);

template <class T> void launch_collide(const StepArgs &a, int ntiles, cudaStream_t s) {
  k_collide<T><<<ntiles, kTile, 0, s>>>(a);
}
template <class T> void launch_half(const StepArgs &a, int ntiles, cudaStream_t s) {
  if (a.geo.gmet)
    k_half<T, true><<<ntiles, kTile, 0, s>>>(a);
  else
    k_half<T, false><<<ntiles, kTile, 0, s>>>(a);
}
template <class T> void launch_full(const StepArgs &a, int ntiles, cudaStream_t s) {
  if (a.geo.gmet)
    k_full<T, true><<<ntiles, kTile, 0, s>>>(a);
  else
    k_full<T, false><<<ntiles, kTile, 0, s>>>(a);
}
void launch_residual_reduce(const CavDev *cav, const double *part, double *resid, int ncav,
                            cudaStream_t s) {
  k_residual_reduce<<<ncav, 256, 0, s>>>(cav, part, resid);
}
template <class T> void launch_init(const CavDev *cav, const int *tile_cav, void *g, void *lam,
                                    int ntiles, cudaStream_t s) {
  k_init<T><<<ntiles, kTile, 0, s>>>(cav, tile_cav, (T *)g, (T *)lam);
}
template <class T> void launch_macros(const CavDev *cav, Geo geo, int cavity, const double *pref,
                                      const void *g, double *rho, double *u, double *v,
                                      double *psi, int nx, int ny, cudaStream_t s) {
  (void)ny;
  k_macros<T><<<(nx + 31) / 32, dim3(32, MSEG), 0, s>>>(cav, geo, cavity, pref, (const T *)g,
                                                        rho, u, v, psi);
}
template <class T> void launch_export(const CavDev *cav, int cavity, const double *pref,
                                      const void *g, const void *lam, double *fhat,
                                      double *lamo, int nx, int ny, cudaStream_t s) {
  k_export<T><<<dim3((nx + 127) / 128, ny), 128, 0, s>>>(cav, cavity, pref, (const T *)g,
                                                          (const T *)lam, fhat, lamo);
}
template <class T> void launch_import(const CavDev *cav, int cavity, const double *pref, void *g,
                                      void *lam, const double *fhat, const double *lami,
                                      int nx, int ny, cudaStream_t s) {
  k_import<T><<<dim3((nx + 127) / 128, ny), 128, 0, s>>>(cav, cavity, pref, (T *)g, (T *)lam,
                                                          fhat, lami);
}
template <class T> void launch_probe(const CavDev *cav, int ncav, const double *pref, const void *g,
                                     int n, const int *probes, double *out, cudaStream_t s) {
  k_probe<T><<<(n + 127) / 128, 128, 0, s>>>(cav, ncav, pref, (const T *)g, n, probes, out);
}
template <class T> void launch_rebase(const CavDev *cav, const int *tile_cav, void *g,
                                      double *pref, double *ptile, int ntiles, int ncav,
                                      cudaStream_t s) {
  k_psum<T><<<ntiles, kTile, 0, s>>>(cav, tile_cav, (const T *)g, ptile);
  k_pshift<<<ncav, 256, 0, s>>>(cav, ntiles, ptile, pref);
  k_rebase<T><<<ntiles, kTile, 0, s>>>(cav, tile_cav, (T *)g, ptile, ntiles);
}

#define IFD_INSTANTIATE(T)                                                                     \
  template void launch_collide<T>(const StepArgs &, int, cudaStream_t);                       \
  template void launch_half<T>(const StepArgs &, int, cudaStream_t);                          \
  template void launch_full<T>(const StepArgs &, int, cudaStream_t);                          \
  template void launch_init<T>(const CavDev *, const int *, void *, void *, int,              \
                               cudaStream_t);                                                  \
  template void launch_macros<T>(const CavDev *, Geo, int, const double *, const void *,      \
                                 double *, double *, double *, double *, int, int,            \
                                 cudaStream_t);                                               \
  template void launch_export<T>(const CavDev *, int, const double *, const void *,           \
                                 const void *, double *, double *, int, int, cudaStream_t);   \
  template void launch_import<T>(const CavDev *, int, const double *, void *, void *,         \
                                 const double *, const double *, int, int, cudaStream_t);     \
  template void launch_probe<T>(const CavDev *, int, const double *, const void *, int,       \
                                const int *, double *, cudaStream_t);                         \
  template void launch_rebase<T>(const CavDev *, const int *, void *, double *, double *, int, \
                                 int, cudaStream_t);
IFD_INSTANTIATE(double)
IFD_INSTANTIATE(float)

}  // namespace ifd

// Fused IFDLBM step: Steps (2)-(6) and the residual partials in one launch.
//
// A CTA of NT threads owns a strip [i0, i1) of at most W = NT - 8 columns of
// one cavity (one thread per column, plus 4 halo columns on each side that it
// recomputes) and a segment [j0, j1) of rows. It marches up the rows;
// iteration k runs
//
//   stage A  row k     moments, f^eq, lagged power-law lambda (FP64 power),
//                      f-hat^+ (Eq. 2.15), f-bar^+ (Eq. 2.16)
//   stage 1  row k-2   half step f-bar(t+dt/2) (Eq. 3.7), its moments,
//                      f(t+dt/2) (Eq. 2.17); wall values by extrapolation
//   stage 2  row k-4   full step f-hat(t+dt) (Eq. 3.6); wall values by
//                      extrapolation (Step 6); residual partials
//
// so that each node's state is read from and written to HBM once per step.
// The state of the rows ahead is prefetched with cp.async into a shared
// staging ring; f-bar^+, f(t+dt/2) and f-hat^+ of the last five rows live in
// shared rings (slot = row mod 5), from which both the xi neighbours (other
// threads) and the eta neighbours (same thread) are read. Wall nodes follow
// the rule of the staged kernels: a side-wall node takes its inner neighbour
// on the same row, a bottom/lid node the node (clamp(i, 1, nx-2), 1 or ny-2);
// row 0 of f(t+dt/2) is made with row 1, row ny-1 one iteration after row
// ny-2 (so that it never takes the ring slot of a row still in use).
//
// FP64 work per node is kept to the power of Eq. (1.4) and the residual
// accumulation: GB300 issues FP64 at 1/64 of the FP32 rate.
#include <cstdint>

#include "d2q9.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace ifd {

namespace {

constexpr int STAGE_ROWS = 3;  // depth of the cp.async prefetch ring (2 rows ahead)

// Shared state per column thread: ~700 B in FP32, so that five 64-thread
// CTAs fit on an SM.
template <class T, int NT>
struct FusedSmem {
  T st_g[STAGE_ROWS][9][NT];      // prefetched state g(t) of rows ahead
  T fb[5][9][NT];                 // f-bar^+
  T fh[5][9][NT];                 // f(t + dt/2)
  T fp[5][9][NT];                 // f-hat^+ (its moments are u, P at t: Eqs. 2.10-2.11)
  T lam[5][NT];                   // lambda(t)
  T gn[9][NT];                    // f-hat(t + dt) of the current stage-2 row
};

__device__ __forceinline__ int slot5(int r) { return (r + 10) % 5; }

// c xi_x of row j and the Jacobian x_xi H: FP64 metrics for FP64 arithmetic,
// their rounded float copies for FP32 arithmetic.
template <class T>
__device__ __forceinline__ T row_cxix(const Geo &g, const CavDev &cv, int j) {
  if constexpr (sizeof(T) == 8)
    return cv.c * g.xix[cv.goff + j];
  else
    return g.cxix_f[cv.goff + j];
}
template <class T>
__device__ __forceinline__ T row_jac(const Geo &g, const CavDev &cv, int j) {
  if constexpr (sizeof(T) == 8)
    return g.xxi[cv.goff + j] * cv.H;
  else
    return g.jac_f[cv.goff + j];
}

__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if (bytes == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Mixed difference of Eqs. (2.5)-(2.7) times 2 d with the upwind side known
// at compile time (eta direction: the side is the sign of e_iy, since
// c_{i eta} = c e_iy / H); `edge` selects the first-order near-wall form.
template <bool POS, class T>
__device__ __forceinline__ T dmix2_side(T fm2, T fm1, T f0, T fp1, T fp2, bool edge, T eta_b) {
  T up;
  if (POS)
    up = edge ? T(2) * (f0 - fm1) : (T(3) * f0 - T(4) * fm1 + fm2);
  else
    up = edge ? T(2) * (fp1 - f0) : -(T(3) * f0 - T(4) * fp1 + fp2);
  return eta_b * (fp1 - fm1) + (T(1) - eta_b) * up;
}

// The same with the side chosen at run time (xi direction): the upwind
// operands are selected, then one stencil is evaluated.
template <class T>
__device__ __forceinline__ T dmix2_sel(T fm2, T fm1, T f0, T fp1, T fp2, bool pos, bool edge_pos,
                                       bool edge_neg, T eta_b) {
  const T fa = pos ? fm1 : fp1, fb = pos ? fm2 : fp2;
  const bool edge = pos ? edge_pos : edge_neg;
  const T u = edge ? T(2) * (f0 - fa) : (T(3) * f0 - T(4) * fa + fb);
  return eta_b * (fp1 - fm1) + (T(1) - eta_b) * (pos ? u : -u);
}

// c_{q xi} D_xi F + c_{q eta} D_eta F at an interior node: `row` is the xi
// row of plane q (this thread at index t), `col` the five eta neighbours.
template <int Q, class T>
__device__ __forceinline__ T advect_q(const T *row, int t, const T col[5], T A, T B, T ceta_unit,
                                      bool clo, bool chi, bool lo, bool hi, T eta_b, T i2dxi,
                                      T i2deta) {
  const T cxi = T(ex(Q)) * A - T(ey(Q)) * B;
  const T f0 = col[2];
  T adv = cxi * dmix2_sel(row[t - 2], row[t - 1], f0, row[t + 1], row[t + 2], cxi >= T(0), clo,
                          chi, eta_b) * i2dxi;
  if constexpr (ey(Q) != 0) {
    const T ceta = T(ey(Q)) * ceta_unit;
    const T dy = (ey(Q) > 0) ? dmix2_side<true>(col[0], col[1], f0, col[3], col[4], lo, eta_b)
                             : dmix2_side<false>(col[0], col[1], f0, col[3], col[4], hi, eta_b);
    adv += ceta * dy * i2deta;
  }
  return adv;
}

template <class T, int Q, int NT>
struct AdvectAll {
  // fills out[q] = F_q - scale * advection_q for q = Q..8
  __device__ __forceinline__ static void run(const T *rows, const T *const cols[5], int t, T A, T B,
                                             T ceta_unit, bool clo, bool chi, bool lo, bool hi,
                                             T eta_b, T i2dxi, T i2deta, T scale, const T *base,
                                             T out[9]) {
    const T col[5] = {cols[0][Q * NT], cols[1][Q * NT], cols[2][Q * NT], cols[3][Q * NT],
                      cols[4][Q * NT]};
    out[Q] = base[Q * NT] - scale * advect_q<Q>(rows + Q * NT, t, col, A, B, ceta_unit, clo, chi,
                                                lo, hi, eta_b, i2dxi, i2deta);
    if constexpr (Q < 8)
      AdvectAll<T, Q + 1, NT>::run(rows, cols, t, A, B, ceta_unit, clo, chi, lo, hi, eta_b, i2dxi,
                                   i2deta, scale, base, out);
  }
};

// Residual terms of one node, summed over up to 8 rows in T before they are
// added to the FP64 partials (a leaf sum; every sum beyond it is FP64).
template <class T>
struct Leaf {
  T du2 = 0, u2 = 0, dP2 = 0, P2 = 0, ek = 0;
  T du2max = 0, u2max = 0;  // maxima are exact in any precision
  int n = 0;
};

template <class T>
__device__ __forceinline__ void leaf_flush(Leaf<T> &l, Partial &p) {
  p.du2 += double(l.du2);
  p.u2 += double(l.u2);
  p.dP2 += double(l.dP2);
  p.P2 += double(l.P2);
  p.ek += double(l.ek);
  l.du2 = l.u2 = l.dP2 = l.P2 = l.ek = T(0);
  l.n = 0;
}

template <class T>
__device__ __forceinline__ void leaf_add(Leaf<T> &l, Partial &p, T u1, T v1, T P1, T u0, T v0,
                                         T P0, T wJ, unsigned *status) {
  if (!(isfinite(u1) && isfinite(v1))) atomicOr(status, 1u);
  const T du = u1 - u0, dv = v1 - v0, dP = P1 - P0;
  const T du2 = du * du + dv * dv, u2 = u1 * u1 + v1 * v1;
  l.du2 += du2;
  l.u2 += u2;
  l.dP2 += dP * dP;
  l.P2 += P1 * P1;
  l.ek += T(0.5) * wJ * u2;
  l.du2max = max(l.du2max, du2);
  l.u2max = max(l.u2max, u2);
  if (++l.n == 8) leaf_flush(l, p);
}

}  // namespace

template <class T, int NT>
__device__ __forceinline__ void fused_task(const FusedArgs &a, FusedSmem<T, NT> &S, int ti) {
  const Task task = a.tasks[ti];
  const CavDev &cv = a.cav[task.cav];
  const int i0 = task.i0, i1 = task.i1, j0 = task.j0, j1 = task.j1;
  const int nx = cv.nx, ny = cv.ny;
  const int t = threadIdx.x;
  const int c = i0 - 4 + t;                          // this thread's column
  const int cc = min(max(c, 0), nx - 1);             // clamped column for loads
  const bool colv = c >= 0 && c < nx;
  const bool own = colv && c >= i0 && c < i1;        // output column (i1 - i0 <= NT - 8)
  const bool inner_c = c >= 1 && c <= nx - 2;
  const bool wall_c = c == 0 || c == nx - 1;
  const int tn = t + (min(max(c, 1), nx - 2) - c);   // thread of the inner neighbour column
  const bool clo = c == 1, chi = c == nx - 2;

  const int64_t b9 = 9 * cv.off;
  const T *gin = (const T *)a.g_in + b9;
  T *gout = (T *)a.g_out + b9;
  const double *lam_in = a.lam_in + cv.off;
  double *lam_out = a.lam_out + cv.off;

  const T c_ = T(cv.c), cs2 = T(cv.cs2), ics2 = T(cv.inv_cs2);
  const T dt = T(cv.dt), hdt = T(0.5 * cv.dt);
  const T eta_b = T(cv.eta_b);
  const T i2dxi = T(cv.inv2dxi), i2deta = T(cv.inv2deta);
  const T ceta_unit = T(cv.c / cv.H);
  const T xeH = T(a.geo.xeH[cv.goff + cc]);          // x_eta / H of this column
  const T wx = T(((c == 0 || c == nx - 1) ? 0.5 : 1.0) * cv.dxi);

  Partial p = {0, 0, 0, 0, 0, 0, 0};
  Leaf<T> leaf;
  T u0s = T(0), v0s = T(0), P0s = T(0);              // u, v, P(t) of row 0

  const int kb = j0 - 4, ke = j1 + 3;
  const int rlo = max(kb, 0), rhi = min(ke, ny - 1);  // rows stage A needs
  auto prefetch = [&](int r) {
    if (r >= rlo && r <= rhi) {
      const int s = r % STAGE_ROWS;
      const int64_t node = int64_t(r) * cv.pitch + cc;
#pragma unroll
      for (int q = 0; q < 9; ++q) cp_async(&S.st_g[s][q][t], gin + q * cv.plane + node, sizeof(T));
    }
    cp_commit();
  };
  // lambda_prev of the row Step (2) works on next, loaded one row ahead
  auto lam_load = [&](int r) {
    return (r >= rlo && r <= rhi) ? lam_in[int64_t(r) * cv.pitch + cc] : 0.0;
  };
  // per-cavity constants of the relaxation time, converted once
  const double gmin2 = cv.gmin2, half_nm1 = cv.half_nm1, Kics2 = cv.Kics2;
  const T wy_in = T(cv.deta), wy_edge = T(0.5 * cv.deta);
  // Step (2) for row r from the staging ring: moments, f^eq and lambda(t).
  // lambda of row k + 1 is formed during the full step of row k, so that the
  // FP64 power overlaps FP32 work instead of delaying the row it belongs to.
  T nux = 0, nuy = 0, nP = 0, ngeq[9];
  double nlam = 0.0;
  struct Collided {
    T ux, uy, P, geq[9];
    double lam;
  };
  auto collide = [&](int r, double lam_prev) {
    Collided o;
    const int s = (r + STAGE_ROWS) % STAGE_ROWS;
    T g[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) g[q] = S.st_g[s][q][t];
    moments(g, c_, cs2, o.ux, o.uy, o.P);                 // Eqs. (2.10)-(2.11)
    equilibrium(o.P, o.ux, o.uy, c_, ics2, o.geq);        // Eq. (2.8)
    T d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = g[q] - o.geq[q];
    T pxx, pxy, pyy;
    second_moments(d, c_, pxx, pxy, pyy);
    // Eqs. (2.12)-(2.14), (1.4): strain rate in T, power in FP64 (as relaxation_time)
    const T k = T(-2) / ((T(2) * T(lam_prev) + dt) * cs2);
    const T Sxx = k * pxx, Sxy = k * pxy, Syy = k * pyy;
    double q = double(T(0.5) * (Sxx * Sxx + T(2) * Sxy * Sxy + Syy * Syy));
    q = q > gmin2 ? q : gmin2;
    o.lam = Kics2 * pow_fast(q, half_nm1, a.powtab);
    return o;
  };
  auto take = [&](const Collided &o) {
    nux = o.ux;
    nuy = o.uy;
    nP = o.P;
#pragma unroll
    for (int q = 0; q < 9; ++q) ngeq[q] = o.geq[q];
    nlam = o.lam;
  };
#pragma unroll
  for (int r = 0; r < STAGE_ROWS - 1; ++r) prefetch(kb + r);
  cp_wait<STAGE_ROWS - 2>();
  if (kb >= 0 && kb < ny) take(collide(kb, lam_load(kb)));
  double lp_next = lam_load(kb + 1);  // lambda_prev of row k + 1

  for (int k = kb; k <= ke; ++k) {
    prefetch(k + STAGE_ROWS - 1);
    cp_wait<STAGE_ROWS - 2>();                     // rows k and k + 1 have landed (own column)

    // ---------------- stage A: row k (lambda formed in the previous iteration) ----------------
    if (k >= 0 && k < ny) {
      const int s = k % STAGE_ROWS, sA = slot5(k);
      if (own && k >= j0 && k < j1) lam_out[int64_t(k) * cv.pitch + c] = nlam;
      const T L = T(nlam);
      const T i2 = T(1) / (T(2) * L + dt);
      const T ap = (T(2) * L - dt) * i2, bp = T(2) * dt * i2;  // Eq. (2.15)
      const T i4 = T(0.5) * i2;
      const T ab = (T(4) * L - dt) * i4, bb = T(3) * dt * i4;  // Eq. (2.16)
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const T gq = S.st_g[s][q][t];
        S.fb[sA][q][t] = ab * gq + bb * ngeq[q];
        S.fp[sA][q][t] = ap * gq + bp * ngeq[q];
      }
      S.lam[sA][t] = L;
      if (k == 0) {
        u0s = nux;
        v0s = nuy;
        P0s = nP;
      }
    }
    // No barrier: stage A writes only this thread's column of row k; other
    // threads read a ring row across columns only two iterations later.

    // ---------------- stage 1: row m = k - 2 ----------------
    const int m = k - 2;
    const bool do1 = m >= 1 && m <= ny - 2;
    if (do1 && inner_c && t >= 2 && t < NT - 2) {
      const int sm = slot5(m), sm1 = slot5(m - 1), sm2 = slot5(m - 2), sp1 = slot5(m + 1),
                sp2 = slot5(m + 2);
      const T A = row_cxix<T>(a.geo, cv, m);           // c xi_x
      const T B = A * xeH;                             // c xi_x x_eta / H
      const bool lo = m == 1, hi = m == ny - 2;
      T fbar[9];
      fbar[0] = S.fb[sm][0][t];
      {
        const T *cols[5] = {&S.fb[sm2][0][t], &S.fb[sm1][0][t], &S.fb[sm][0][t], &S.fb[sp1][0][t],
                            &S.fb[sp2][0][t]};
        AdvectAll<T, 1, NT>::run(&S.fb[sm][0][0], cols, t, A, B, ceta_unit, clo, chi, lo, hi, eta_b,
                                 i2dxi, i2deta, hdt, &S.fb[sm][0][t], fbar);   // Eq. (3.7)
      }
      T ux, uy, P;
      moments(fbar, c_, cs2, ux, uy, P);
      T geq[9];
      equilibrium(P, ux, uy, c_, ics2, geq);
      const T L = S.lam[sm][t];
      const T i4 = T(1) / (T(4) * L + dt);
      const T ah = T(4) * L * i4, bh = dt * i4;                       // Eq. (2.17)
#pragma unroll
      for (int q = 0; q < 9; ++q) S.fh[sm][q][t] = ah * fbar[q] + bh * geq[q];
    }
    __syncthreads();
    if (m >= 1 && m < ny && t >= 2 && t < NT - 2 && colv) {
      if (do1 && wall_c) {                            // side walls of row m
        T F[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) F[q] = S.fh[slot5(m)][q][tn];
        nee(F, T(0), T(0), cv);
#pragma unroll
        for (int q = 0; q < 9; ++q) S.fh[slot5(m)][q][t] = F[q];
      }
      if (m == 1 || m == ny - 1) {                    // bottom row 0 / lid row ny-1
        const bool lid = m == ny - 1;
        const int src = lid ? slot5(ny - 2) : slot5(1), dst = lid ? slot5(ny - 1) : slot5(0);
        T F[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) F[q] = S.fh[src][q][tn];
        nee(F, (lid && inner_c) ? T(cv.U) : T(0), T(0), cv);
#pragma unroll
        for (int q = 0; q < 9; ++q) S.fh[dst][q][t] = F[q];
      }
    }
    // No barrier: stage 2 reads other columns only of row k - 4, finished two
    // iterations ago, and the eta neighbours from its own column.

    // ---------------- stage 2: row o = k - 4 ----------------
    const int o = k - 4;
    const bool do2 = o >= 1 && o <= ny - 2 && o >= j0 && o < j1;
    if (do2 && inner_c && t >= 4 && t < NT - 4) {
      const int so = slot5(o), so1 = slot5(o - 1), so2 = slot5(o - 2), sp1 = slot5(o + 1),
                sp2 = slot5(o + 2);
      const T A = row_cxix<T>(a.geo, cv, o);
      const T B = A * xeH;
      const bool lo = o == 1, hi = o == ny - 2;
      T gnv[9];
      gnv[0] = S.fp[so][0][t];
      {
        const T *cols[5] = {&S.fh[so2][0][t], &S.fh[so1][0][t], &S.fh[so][0][t], &S.fh[sp1][0][t],
                            &S.fh[sp2][0][t]};
        AdvectAll<T, 1, NT>::run(&S.fh[so][0][0], cols, t, A, B, ceta_unit, clo, chi, lo, hi, eta_b,
                                 i2dxi, i2deta, dt, &S.fp[so][0][t], gnv);     // Eq. (3.6)
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) S.gn[q][t] = gnv[q];
    }
    if (k + 1 <= rhi && k + 1 >= 0) take(collide(k + 1, lp_next));  // lambda of the next row
    lp_next = lam_load(k + 2);
    __syncthreads();
    if (do2 && own) {
      const int so = slot5(o);
      T gnv[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) gnv[q] = S.gn[q][tn];
      if (wall_c) nee(gnv, T(0), T(0), cv);
      const int64_t node = int64_t(o) * cv.pitch + c;
#pragma unroll
      for (int q = 0; q < 9; ++q) gout[q * cv.plane + node] = gnv[q];
      if (a.want_residual) {
        T ux, uy, P, u0, v0, P0;
        moments(gnv, c_, cs2, ux, uy, P);
        T fpo[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) fpo[q] = S.fp[so][q][t];
        moments(fpo, c_, cs2, u0, v0, P0);  // u, P at t (moments of f-hat^+ equal those of f-hat)
        const T wJ = wx * wy_in * row_jac<T>(a.geo, cv, o);
        leaf_add(leaf, p, ux, uy, P, u0, v0, P0, wJ, a.status);
      }
      // wall rows produced with their neighbour rows
      const bool bottom = o == 1 && j0 == 0;
      const bool top = o == ny - 2 && j1 == ny;
      if (bottom || top) {
        T F[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) F[q] = S.gn[q][tn];
        nee(F, (top && inner_c) ? T(cv.U) : T(0), T(0), cv);
        const int r = bottom ? 0 : ny - 1;
        const int64_t nd = int64_t(r) * cv.pitch + c;
#pragma unroll
        for (int q = 0; q < 9; ++q) gout[q * cv.plane + nd] = F[q];
        if (a.want_residual) {
          T wx2, wy2, wP2;
          moments(F, c_, cs2, wx2, wy2, wP2);
          T ou = u0s, ov = v0s, oP = P0s;
          if (!bottom) {
            T fpr[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) fpr[q] = S.fp[slot5(r)][q][t];
            moments(fpr, c_, cs2, ou, ov, oP);
          }
          const T wJ = wx * wy_edge * row_jac<T>(a.geo, cv, r);
          leaf_add(leaf, p, wx2, wy2, wP2, ou, ov, oP, wJ, a.status);
        }
      }
    }
  }
  cp_wait<0>();
  if (a.want_residual) {
    leaf_flush(leaf, p);
    p.du2max = double(leaf.du2max);
    p.u2max = double(leaf.u2max);
    block_partial<NT / 32>(p, a.part, ti);
  }
  __syncthreads();  // the next task reuses the shared rings
}

// Schedules: 0 one CTA per task; 1 persistent CTAs taking positions
// blockIdx.x, blockIdx.x + gridDim.x, ... of the largest-first order;
// 2 persistent CTAs taking positions from an atomic counter (no waiting on
// other CTAs: a CTA that finds the list exhausted returns).
template <class T, int NT>
__global__ void __launch_bounds__(NT) k_fused(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FusedSmem<T, NT> &S = *reinterpret_cast<FusedSmem<T, NT> *>(smem_raw);
  __shared__ int next;
  if (a.schedule == 0) {
    fused_task<T, NT>(a, S, blockIdx.x);
    return;
  }
  for (int it = 0;; ++it) {
    int pos;
    if (a.schedule == 1) {
      pos = blockIdx.x + it * gridDim.x;
    } else {
      if (threadIdx.x == 0) next = atomicAdd(a.counter, 1);
      __syncthreads();
      pos = next;
      __syncthreads();
    }
    if (pos >= a.ntasks) return;
    fused_task<T, NT>(a, S, a.order[pos]);
  }
}

template <class T, int NT>
static void configure_nt() {
  static bool configured = false;  // the attribute is per function
  if (!configured) {
    cudaFuncSetAttribute(k_fused<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(sizeof(FusedSmem<T, NT>)));
    configured = true;
  }
}

template <class T, int NT>
static void launch_fused_nt(const FusedArgs &a, int grid, cudaStream_t s) {
  configure_nt<T, NT>();
  k_fused<T, NT><<<grid, NT, int(sizeof(FusedSmem<T, NT>)), s>>>(a);
}

template <class T, int NT>
static int blocks_per_sm_nt() {
  configure_nt<T, NT>();
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused<T, NT>, NT,
                                                int(sizeof(FusedSmem<T, NT>)));
  return n;
}

template <class T> int fused_blocks_per_sm(int nt) {
  switch (nt) {
    case 64: return blocks_per_sm_nt<T, 64>();
    case 128: return blocks_per_sm_nt<T, 128>();
    case 256:
      if constexpr (sizeof(T) == 4) return blocks_per_sm_nt<T, 256>();
      return 0;
  }
  return 0;
}

template <class T> int fused_smem_bytes(int nt) {
  switch (nt) {
    case 64: return int(sizeof(FusedSmem<T, 64>));
    case 128: return int(sizeof(FusedSmem<T, 128>));
    case 256: return sizeof(T) == 4 ? int(sizeof(FusedSmem<T, 256>)) : -1;
  }
  return -1;
}

template <class T> bool launch_fused(const FusedArgs &a, int nt, int ntasks, cudaStream_t s) {
  switch (nt) {
    case 64: launch_fused_nt<T, 64>(a, ntasks, s); return true;
    case 128: launch_fused_nt<T, 128>(a, ntasks, s); return true;
    case 256:
      if constexpr (sizeof(T) == 4) {
        launch_fused_nt<T, 256>(a, ntasks, s);
        return true;
      }
      return false;
  }
  return false;
}

template bool launch_fused<float>(const FusedArgs &, int, int, cudaStream_t);
template bool launch_fused<double>(const FusedArgs &, int, int, cudaStream_t);
template int fused_smem_bytes<float>(int);
template int fused_smem_bytes<double>(int);
template int fused_blocks_per_sm<float>(int);
template int fused_blocks_per_sm<double>(int);

}  // namespace ifd

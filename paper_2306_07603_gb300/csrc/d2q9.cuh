// Device-side lattice arithmetic of the IFDLBM step (D2Q9).
//
// All distributions are handled as deviations from the rest equilibrium,
// g_i = F_i - w_i rho0 (F = f, f-hat, f-bar, ...). Every transform of the
// scheme is affine with coefficients summing to one and every difference
// of a constant vanishes, so the scheme acts on g exactly as on F; only
// the moments (Eqs. 2.10-2.11) and the equilibrium (Eq. 2.8) drop their
// rho0 terms.
#pragma once
#include <cuda_runtime.h>

#include "fastpow.cuh"
#include "internal.h"

namespace ifd {

// D2Q9 velocity directions, Eq. (2.9): e_0 = 0, e_1..4 axes, e_5..8 diagonals.
__host__ __device__ constexpr int ex(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// Weights w_i and pressure weights wbar_i of Eq. (2.9).
__host__ __device__ constexpr double wgt(int i) {
  return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr double wbar(int i) {
  return i == 0 ? -5.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// FP32 arithmetic keeps the moment identities of Eqs. (2.8), (2.10)-(2.11)
// free of systematic error: the weights are carried as the integers 36 w_i
// and 36 wbar_i, and the non-representable factors 1/36 and 1/5 as pairs of
// floats (hi + lo, ~48 bits), so that the only FP32 errors left are the
// roundings of the operations. A fixed relative error in a weight (1/9 and
// 1/36 are not floats) would make the collision drive u and P towards
// (1 + delta) u and (1 + delta) P every step, a bias that the slowest modes
// of a cavity integrate over thousands of steps.
struct F2 {
  float hi, lo;
};
__host__ __device__ constexpr F2 f2_of(double x) { return {float(x), float(x - double(float(x)))}; }
constexpr F2 INV36 = f2_of(1.0 / 36.0);
constexpr F2 INV5 = f2_of(1.0 / 5.0);
__device__ __forceinline__ float mul_f2(float x, F2 k) { return fmaf(x, k.hi, x * k.lo); }
__host__ __device__ constexpr int w36(int i) { return i == 0 ? 16 : (i <= 4 ? 4 : 1); }
__host__ __device__ constexpr int wbar36(int i) { return i == 0 ? -20 : (i <= 4 ? 4 : 1); }

// Velocity and pressure of a deviation set, Eqs. (2.10)-(2.11):
//   u = c sum_i e_i g_i,
//   P = c_s^2 / wbar_0 (-sum_{i>0} g_i + w_0 |u|^2 / (2 c_s^2))
//     = (3 c^2 sum_{i>0} g_i - 2 |u|^2) / 5            (c_s^2 = c^2/3).
template <class T>
__device__ __forceinline__ void moments(const T g[9], T c, T cs2, T &ux, T &uy, T &P) {
  ux = c * ((g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]));
  uy = c * ((g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]));
  T s = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
  T uu = ux * ux + uy * uy;
  if constexpr (sizeof(T) == 4)
    P = mul_f2(T(3) * (c * c) * s - T(2) * uu, INV5);
  else
    P = (cs2 / T(wbar(0))) * (-s + T(wgt(0)) * uu / (T(2) * cs2));
}

// Designed equilibrium, Eq. (2.8) (quadratic term over 2 c_s^4), minus w_i rho0.
template <class T>
__device__ __forceinline__ void equilibrium(T P, T ux, T uy, T c, T inv_cs2, T geq[9]) {
  const T uu = ux * ux + uy * uy;
  const T pterm = P * inv_cs2;
  const T half_inv_cs2 = T(0.5) * inv_cs2;
  const T half_inv_cs4 = half_inv_cs2 * inv_cs2;
  const T base = -uu * half_inv_cs2;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T cu = c * (T(ex(i)) * ux + T(ey(i)) * uy);
    const T quad = cu * inv_cs2 + cu * cu * half_inv_cs4 + base;
    if constexpr (sizeof(T) == 4)
      geq[i] = mul_f2(T(wbar36(i)) * pterm + T(w36(i)) * quad, INV36);
    else
      geq[i] = T(wbar(i)) * pterm + T(wgt(i)) * quad;
  }
}

// The transforms of Eqs. (2.15)-(2.17) have coefficients summing to one,
// a F + b f^eq with a = 1 - b; they are evaluated as F + b (f^eq - F), so
// that u and P, which F and f^eq share, are kept to the rounding of the
// small difference rather than of F.
template <class T>
__device__ __forceinline__ T toward(T F, T feq, T b) {
  return F + b * (feq - F);
}

// Implicit form of Eq. (2.14): lam = C max(a / (2 lam + dt), gamma_min)^(n-1)
// with C = K / c_s^2 and a = 2 sqrt((Pxx^2 + 2 Pxy^2 + Pyy^2) / 2) / c_s^2,
// Pxx.. the second moments of f-hat - f^eq (Eq. 2.18 at the same lam turns
// them into gamma-dot(lam) = a / (2 lam + dt)). F(lam) = lam - C max(...)^(n-1)
// increases strictly, so the root is unique: it is the clamp value
// lam_c = C gamma_min^(n-1) when gamma-dot(lam_c) <= gamma_min, and otherwise
// lies in [0, lam_c] (n < 1) or [lam_c, C (a/dt)^(n-1)] (n > 1) with
// gamma-dot > gamma_min. Newton from lam_start, kept inside the bracket by
// bisection, one FP64 power per iteration; it stops once the Newton step is
// below 4e-15 of lam (F = lam - P is itself a difference of nearly equal
// numbers, so steps much smaller than that are rounding). Kept out of line so
// that the lagged path is compiled as without it.
static __device__ __noinline__ double lambda_implicit(double a, double lam_start, const CavDev &cv,
                                                      const double *powtab) {
  const double C = cv.Kics2, dt = cv.dt, m = cv.nm1, lamc = cv.lam0;
  if (m == 0.0) return C;
  if (a <= cv.gmin * (2.0 * lamc + dt)) return lamc;
  double lo, hi;
  if (m < 0.0) {
    lo = 0.0;
    hi = lamc;
  } else {
    lo = lamc;
    hi = C * pow_fast((a / dt) * (a / dt), cv.half_nm1, powtab);
  }
  double lam = (lam_start > lo && lam_start < hi) ? lam_start : 0.5 * (lo + hi);
  for (int it = 0; it < 20; ++it) {
    const double x = 2.0 * lam + dt;
    const double g = a / x;
    const double P = C * pow_fast(g * g, cv.half_nm1, powtab);
    const double F = lam - P;
    if (F == 0.0) break;                                   // the root itself
    if (F > 0.0) hi = lam; else lo = lam;
    double next = lam - F / (1.0 + 2.0 * m * P / x);
    if (!(next >= lo && next <= hi)) next = 0.5 * (lo + hi);
    const bool done = fabs(next - lam) <= 4e-15 * next;
    lam = next;
    if (done) break;
  }
  return lam;
}

// The same solve in FP32 for the FP32-deviation form, with the FP32 power
// (pow_f32, relative error ~1e-6 for these arguments): F is then known to
// about 1e-6 of lam, so the iteration stops once the Newton step is below
// 4e-6 of lam, after at most 10 iterations. As with the power, this error
// reaches the populations only through the relaxation weights, far below the
// FP32 rounding of the stored deviations.
static __device__ __noinline__ float lambda_implicit_f32(float a, float lam_start,
                                                         const CavDev &cv) {
  const float C = float(cv.Kics2), dt = float(cv.dt), m = float(cv.nm1), hm = float(cv.half_nm1);
  const float lamc = float(cv.lam0);
  if (cv.nm1 == 0.0) return C;
  if (a <= float(cv.gmin) * (2.0f * lamc + dt)) return lamc;
  float lo, hi;
  if (m < 0.0f) {
    lo = 0.0f;
    hi = lamc;
  } else {
    lo = lamc;
    hi = C * pow_f32((a / dt) * (a / dt), hm);
  }
  float lam = (lam_start > lo && lam_start < hi) ? lam_start : 0.5f * (lo + hi);
  for (int it = 0; it < 10; ++it) {
    const float x = 2.0f * lam + dt;
    const float g = a / x;
    const float P = C * pow_f32(g * g, hm);
    const float F = lam - P;
    if (F == 0.0f) break;
    if (F > 0.0f) hi = lam; else lo = lam;
    float next = lam - F / (1.0f + 2.0f * m * P / x);
    if (!(next >= lo && next <= hi)) next = 0.5f * (lo + hi);
    const bool done = fabsf(next - lam) <= 4e-6f * next;
    lam = next;
    if (done) break;
  }
  return lam;
}

// Relaxation time of Step (2): strain rate from f^ne (Eqs. 2.12-2.13, with
// f = f(f-hat, lam_prev) of Eq. 2.18), q = |gamma-dot|^2 = 2 D:D, the
// clamped power law mu = K max(|gamma-dot|, gamma_min)^(n-1) evaluated as
// K max(q, gamma_min^2)^((n-1)/2) (Eq. 1.4), and lam = mu / c_s^2 (Eq. 2.14).
// Pxx, Pxy, Pyy are sum_i c_ia c_ib (g_i - geq_i). The strain rate is formed
// in T (the storage precision); the power law of Eq. (1.4) and the implicit
// form's solve are FP64, as the FP32-deviation form specifies: pow_fast for
// an FP64 strain rate, pow_tab (FP64 result, error within 6e-16) for the FP32
// one, clamped at cv.gmin2_f. With cv.pow32 (FP32 storage only, an opt-in)
// they are FP32 instead (pow_f32, lambda_implicit_f32; the clamp at the
// largest float not above gamma_min^2). powt: the cavity's pow_tab table.
template <class T>
__device__ __forceinline__ double relaxation_time(T Pxx, T Pxy, T Pyy, double lam_prev,
                                                  const CavDev &cv, const double *powtab,
                                                  const double *powt) {
  if (cv.implicit) {
    const T G2 = T(0.5) * (Pxx * Pxx + T(2) * Pxy * Pxy + Pyy * Pyy);
    if constexpr (sizeof(T) == 4)
      if (cv.pow32)
        return double(lambda_implicit_f32(2.0f * sqrtf(G2) * float(cv.inv_cs2), float(lam_prev), cv));
    return lambda_implicit(2.0 * sqrt(double(G2)) * cv.inv_cs2, lam_prev, cv, powtab);
  }
  // f^ne = 2 lam_prev/(2 lam_prev + dt) (f-hat - f^eq);  S = -sum c c f^ne / (lam_prev c_s^2)
  const T k = T(-2) / ((T(2) * T(lam_prev) + T(cv.dt)) * T(cv.cs2));
  const T Sxx = k * Pxx, Sxy = k * Pxy, Syy = k * Pyy;
  if constexpr (sizeof(T) == 4) {
    if (cv.pow32) {
      const float q = fmaxf(0.5f * (Sxx * Sxx + 2.0f * Sxy * Sxy + Syy * Syy),
                            __double2float_rd(cv.gmin2));
      return double(float(cv.Kics2) * pow_f32(q, float(cv.half_nm1)));
    }
    const float q = fmaxf(0.5f * (Sxx * Sxx + 2.0f * Sxy * Sxy + Syy * Syy), cv.gmin2_f);
    return pow_tab(q, powt, cv.half_nm1, cv.pb2, cv.pb3, cv.pb4, cv.pb5);
  }
  double q = double(T(0.5) * (Sxx * Sxx + T(2) * Sxy * Sxy + Syy * Syy));
  q = q > cv.gmin2 ? q : cv.gmin2;
  return cv.Kics2 * pow_fast(q, cv.half_nm1, powtab);
}

// Second moments of the non-equilibrium deviation d_i = g_i - geq_i.
template <class T>
__device__ __forceinline__ void second_moments(const T d[9], T c, T &Pxx, T &Pxy, T &Pyy) {
  const T c2 = c * c;
  const T diag = (d[5] + d[6]) + (d[7] + d[8]);
  Pxx = c2 * ((d[1] + d[3]) + diag);
  Pyy = c2 * ((d[2] + d[4]) + diag);
  Pxy = c2 * ((d[5] - d[6]) + (d[7] - d[8]));
}

// Mixed difference of Eqs. (2.5)-(2.7) times 2 d:
//   eta_b (F[k+1] - F[k-1]) + (1 - eta_b) U,
// U the 2nd-order upwind difference times 2 d on the side given by the
// sign of the contravariant velocity (c >= 0 uses k-2..k, c < 0 uses
// k..k+2), reduced to first order where that stencil would leave the grid
// (k = 1 for c >= 0, k = N-2 for c < 0).
template <class T>
__device__ __forceinline__ T dmix2(T fm2, T fm1, T f0, T fp1, T fp2, bool pos, bool lo, bool hi,
                                   T eta_b) {
  const T central = fp1 - fm1;
  T up;
  if (pos)
    up = lo ? T(2) * (f0 - fm1) : (T(3) * f0 - T(4) * fm1 + fm2);
  else
    up = hi ? T(2) * (fp1 - f0) : -(T(3) * f0 - T(4) * fp1 + fp2);
  return eta_b * central + (T(1) - eta_b) * up;
}

// Contravariant velocities of Eq. (3.4) for the trapezoid map, where
// eta_x = 0, eta_y = 1/H, xi_x = 1/x_xi, xi_y = -x_eta/(H x_xi):
//   c_{i xi} = c xi_x (e_ix - e_iy x_eta/H),  c_{i eta} = c e_iy / H.
__device__ __forceinline__ double cxi_of(int q, double A, double B) {
  // A = c xi_x, B = c xi_x x_eta / H
  return double(ex(q)) * A - double(ey(q)) * B;
}

// Wall-node rule (Sec. 4) with a given wall pressure Pb:
// F_b = f^eq(Pb, u_w) + F_nb - f^eq(P_nb, u_nb), F holding F_nb on entry.
template <class T>
__device__ __forceinline__ void nee_p(T F[9], T uwx, T uwy, T Pb, T c, T cs2, T ics2) {
  T ux, uy, P;
  moments(F, c, cs2, ux, uy, P);
  T fw[9], fn[9];
  equilibrium(Pb, uwx, uwy, c, ics2, fw);
  equilibrium(P, ux, uy, c, ics2, fn);
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = fw[q] + (F[q] - fn[q]);
}

// Wall-node rule (Sec. 4) with the pressure extrapolated at zeroth order:
// F_b = f^eq(P_nb, u_w) + F_nb - f^eq(P_nb, u_nb).
template <class T>
__device__ __forceinline__ void nee(T F[9], T uwx, T uwy, T c, T cs2, T ics2) {
  T ux, uy, P;
  moments(F, c, cs2, ux, uy, P);
  T fw[9], fn[9];
  equilibrium(P, uwx, uwy, c, ics2, fw);
  equilibrium(P, ux, uy, c, ics2, fn);
#pragma unroll
  for (int q = 0; q < 9; ++q) F[q] = fw[q] + (F[q] - fn[q]);
}
template <class T>
__device__ __forceinline__ void nee(T F[9], T uwx, T uwy, const CavDev &cv) {
  nee(F, uwx, uwy, T(cv.c), T(cv.cs2), T(cv.inv_cs2));
}

}  // namespace ifd

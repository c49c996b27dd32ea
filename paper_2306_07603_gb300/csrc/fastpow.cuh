// x^m in FP64 for the power-law viscosity, Eq. (1.4), with few FP64 instructions.
//
// GB300 issues FP64 at 1/64 of the FP32 rate, so a general-purpose pow is
// the most expensive part of the relaxation time. This evaluates
// 2^(m log2 x) by the table-driven reduction of P. T. P. Tang ("Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15, 1989; "... of the logarithm function", ACM TOMS
// 16, 1990), with 256-entry tables built on the host in extended precision:
//
//   log2 x = e + log2(1/r_j) + log2(1 + t),  t = f r_j - 1,  |t| < 2^-9
//   2^y    = 2^k * 2^(j/256) * 2^r,          |r| <= 2^-9
//
// The leading one or two terms of each series are FP64; the tails, whose
// magnitudes are below 4e-9, are formed in FP32 (their rounding then stays
// below 5e-16 absolute). About 20 FP64 instructions. log2 x and y are kept
// as single doubles, so their rounding (each at most |y| 2^-53 relative)
// gives a relative error of about ln2 |y| 2^-52 on top of ~3e-16 from the
// series: within 5e-16 + 2.2e-16 |m log2 x| for normal x > 0 and |y| < 1000
// (checked against CUDA's pow by the self-test entry point).
#pragma once
#include <cuda_runtime.h>

namespace ifd {

// Table layout (3 x 256 doubles): r_j = 1/(1 + (j + 1/2)/256), L_j = -log2(r_j),
// T_j = 2^(j/256).
constexpr int POW_TABLE_SIZE = 3 * 256;

__device__ __forceinline__ double pow_fast(double x, double m, const double *__restrict__ tab) {
  constexpr double K1 = 1.4426950408889634074;       // 1/ln 2
  constexpr double LN2 = 0.69314718055994530942;
  constexpr double MAGIC = 6755399441055744.0;       // 1.5 * 2^52
  // log2 x: x = 2^e f, f in [1, 2); j = top 8 bits of the fraction
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int e = ((hi >> 20) & 0x7FF) - 1023;
  const int j = (hi >> 12) & 0xFF;
  const double f = __hiloint2double((hi & 0x000FFFFF) | 0x3FF00000, lo);
  const double t = fma(f, __ldg(tab + j), -1.0);
  const double t2 = t * t;
  double s = fma(t2, -0.5 * K1, t * K1);             // t/ln2 - t^2/(2 ln2)
  const float tf = float(t);
  const float c32 = float(K1 / 3.0) + tf * (float(-K1 / 4.0) + tf * float(K1 / 5.0));
  s = fma(t2 * t, double(c32), s);                   // + t^3 (1/3 - t/4 + t^2/5)/ln2
  const double lg = (double(e) + __ldg(tab + 256 + j)) + s;
  // 2^y, y = m log2 x: N = round(256 y), r = y - N/256
  const double y = m * lg;
  const double v = fma(y, 256.0, MAGIC);
  const int N = __double2loint(v);
  const double r = fma(v - MAGIC, -1.0 / 256.0, y);
  const double a = r * LN2;
  const float af = float(a);
  const float tail = af * (1.0f / 6.0f + af * (1.0f / 24.0f));
  const double sr = fma(a * a, 0.5 + double(tail), a);  // 2^r - 1
  const double T = __ldg(tab + 512 + (N & 255));
  const double res = fma(T, sr, T);
  return __hiloint2double(__double2hiint(res) + ((N >> 8) << 20), __double2loint(res));
}

// x^m in FP32 for the FP32-deviation form: 2^(m log2 x) with CUDA's log2f
// and exp2f (1 and 2 ulp by the CUDA math documentation). For normal x > 0
// its relative error is about ln2 2^-24 (2 |m log2 x| + |m log2 x|) from the
// roundings of log2 x and of y = m log2 x, plus 2 ulp: within
// 3e-7 + 1.3e-7 |m log2 x|. The strain rate it is applied to is itself
// formed in FP32, and lambda enters the step only through the relaxation
// weights of Eqs. (2.15)-(2.17), which multiply f - f^eq, so this error
// reaches the populations far below their FP32 rounding. The GB300 FP64 pipe
// runs at 1/64 of the FP32 rate; this takes the power off it.
__device__ __forceinline__ float pow_f32(float x, float m) { return exp2f(m * log2f(x)); }

}  // namespace ifd

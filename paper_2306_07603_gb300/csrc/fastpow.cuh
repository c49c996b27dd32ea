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

// C x^m in FP64 for an FP32 argument x (the strain rate of the FP32-deviation
// form is formed in FP32): a table-driven binomial evaluation with 7 FP64
// instructions. With x = 2^(e-127) f, f in [1, 2) its fraction, j the leading 8
// bits of the fraction and c_j = 1 + (j + 1/2)/256 the centre of that interval,
//
//   C x^m = [C 2^(m (e - 127))] [c_j^m] (1 + t)^m,   t = f / c_j - 1, |t| <= 2^-9,
//
// the first two factors come from per-cavity FP64 tables built on the host in
// extended precision, and (1 + t)^m = 1 + b1 t + b2 t^2 + ... + b5 t^5 is the
// binomial series (b_k = m (m-1) ... (m-k+1) / k!; the next term is below
// 2^-54 |b6| for |t| <= 2^-9). t is formed in FP64 from the exact fraction as
// f (1/c_j) - 1 (absolute error <= 1.2e-16); the terms from t^3 on, whose sum
// is below 1e-9, take their coefficient c3 = b3 + b4 t + b5 t^2 in FP32 (its
// error reaches the sum as t^3 dc3 < 1e-16). Relative error: table roundings
// (2 x 2^-53), the products and the final fma (3 x 2^-53) and the series
// (< 2e-16): within 6e-16 for every normal x > 0, independent of m log2 x
// (checked against CUDA's pow by the self-test entry point). The argument
// must be a normal float (the callers clamp it at or above FLT_MIN).
//
// Per-cavity table (POWT_SIZE doubles): [2j] = c_j^m, [2j + 1] = 1/c_j
// (j = 0..255); [512 + e] = C 2^(m (e - 127)) (e = 0..255).
constexpr int POWT_SIZE = 768;

__device__ __forceinline__ double pow_tab(float x, const double *__restrict__ tab, double b1,
                                          double b2, float b3, float b4, float b5) {
  const unsigned bits = __float_as_uint(x);
  const unsigned e = bits >> 23;                 // biased exponent (x > 0)
  const unsigned j = (bits >> 15) & 255u;        // leading 8 bits of the fraction
  const unsigned frac = bits & 0x7FFFFFu;
  // the fraction 1.frac exactly, as a double (integer moves, no conversion)
  const double f = __hiloint2double(int(0x3FF00000u | (frac >> 3)), int(frac << 29));
  const double2 dr = __ldg(reinterpret_cast<const double2 *>(tab) + j);
  const double t = fma(f, dr.y, -1.0);           // f / c_j - 1
  // t to ~1e-7 for the tail: f - c_j is exact in FP32 (both in [1, 2), 2^-9 apart at most)
  const float cj = __uint_as_float(0x3F804000u | (j << 15));
  const float tf = __fdividef(__uint_as_float(0x3F800000u | frac) - cj, cj);
  const float c3 = fmaf(tf, fmaf(tf, b5, b4), b3);
  const double w = fma(t, fma(t, double(c3), b2), b1);
  const double P = __ldg(tab + 512 + e) * dr.x;  // C 2^(m (e - 127)) c_j^m
  return fma(P, t * w, P);
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

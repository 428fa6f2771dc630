// pivot_device.cuh -- FP64 device math of the PIVOT hot path (sm_103a).
//
// Notation (appendix "five-stage LBR construction"; Section 2, normalised
// Black function):
//   x = -|ln(F/K)| <= 0   log-moneyness of the out-of-the-money equivalent
//                         (stage 1, put-call reduction; Jaeckel's sign, the
//                         paper's k = ln(K/F) = -x for OTM calls)
//   s = sigma sqrt(T)     total volatility (the paper's sigma_tau)
//   h = x/s, t = s/2
//   b(x,s)   = e^{x/2} Phi(h + t) - e^{-x/2} Phi(h - t)   (Eq. app_normalized_black)
//   b_s(x,s) = exp(-(h^2 + t^2)/2) / sqrt(2 pi)          (its s-derivative)
//   b_max    = e^{x/2}                                   (Eq. app_b_bounds)
// With Y(z) = Phi(z)/phi(z) = sqrt(pi/2) erfcx(-z/sqrt 2) and
// e^{x/2} phi(h + t) = e^{-x/2} phi(h - t) = b_s:
//   b         = b_s * rho,    rho   = Y(h + t) - Y(h - t)
//   b_max - b = b_s * gamma,  gamma = Y(-h - t) + Y(h - t)   (sum of positives)
// rho cancels when t << |h| near the money; there it is summed as the
// Taylor series in t of Y(h + t) - Y(h - t), whose coefficients
// c_n = Y^(n)(h)/n! follow from Y' = 1 + zY:
//   c_0 = Y(h), c_1 = 1 + h Y(h), c_{n+1} = (h c_n + c_{n-1})/(n + 1),
//   rho = 2 sum_{k odd} c_k t^k.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pivot {

constexpr double kSqrt2Pi = 2.50662827463100050242;    // sqrt(2 pi)
constexpr double kInvSqrt2Pi = 0.398942280401432677940; // 1/sqrt(2 pi)
constexpr double kSqrtPiOver2 = 1.25331413731550025121; // sqrt(pi/2)
constexpr double kInvSqrt2 = 0.707106781186547524401;
constexpr double kSqrt2 = 1.41421356237309504880;
constexpr double kLnSqrt2Pi = 0.918938533204672741780;
constexpr double kInvSqrt3 = 0.577350269189625764509;
constexpr double kTwoPiOver3Sqrt3 = 1.20919957615614523543; // 2 pi / (3 sqrt 3)

// Taylor zone of rho: t <= kTaylorT and |x| <= kTaylorX; 9 odd terms reach
// double precision for t <= 0.25 at every h <= 0 (c_n(h) <= c_n(0)).
// Outside it the difference Y(h + t) - Y(h - t) is used: its rounding moves
// sigma by about eps Y(h + t) / s <= eps / |x| in relative terms, at most
// 10 eps for |x| >= 0.1, and by <= 1.25 eps / s <= 2.5 eps for t > 0.25.
constexpr double kTaylorT = 0.25;
constexpr double kTaylorX = 0.1;

enum Region : int { kLower = 0, kMidLow = 1, kMidHigh = 2, kUpper = 3 };

// The LBR arithmetic below is written once for both precisions: double for
// the plain path, float for the guess and first Householder step of the
// mixed path.  Math<R> maps each function to its CUDA precision variant.
template <typename R>
struct Math;
// The Mills ratio M(w) = Y(-w) = Phi(-w)/phi(w) = sqrt(pi/2) erfcx(w/sqrt 2),
// w >= 0, in FP64: degree-9 Chebyshev interpolants on 177 intervals of [0, 128)
// (coefficients written by gen_mills_table.py, ~1 ulp) and the asymptotic series
// M(w) ~ (1/w) sum_n (-1)^n (2n-1)!! / w^(2n) from 128 on (nine terms, truncation
// below 1e-27 there).  Every Mills ratio the solver and the adjoint evaluate is
// Y at a non-positive argument, i.e. M of its negation, so the table takes w
// itself: no scaling of the argument or of the result.  The interval is read
// off the bit pattern of w (interval 0 = [0, 1/16), then 16 equal parts per
// binade up to 128), so the table covers every Mills ratio of a normal-range
// price in one branch (the series only serves iterates far outside it) and the
// FP64 pipe sees one fma for the local variable and the Horner chain; the
// table rows are 96 bytes and hit L1.
#include "mills_table.inc"

__device__ __forceinline__ double mills_neg(double w) {
  const uint64_t bits = uint64_t(__double_as_longlong(w)) & 0x7fffffffffffffffull; // w = -0 too
  if (bits < 0x4060000000000000ull) { // |w| < 128
    // biased exponent and top four mantissa bits, less those of 1/16, plus one (0 below 1/16)
    const int k = max(int(bits >> 48) - ((1023 - 4) << 4) + 1, 0);
    const double* c = kMillsCoef[k];
    const double tau = fma(w, __ldg(c + 10), __ldg(c + 11)); // in [-1, 1]; scale 2^j, offset an integer
    double v = __ldg(c + 9);
#pragma unroll
    for (int j = 8; j >= 0; --j) v = fma(v, tau, __ldg(c + j));
    return v;
  }
  const double iw = 1.0 / w;
  const double q = iw * iw;
  double s = 2027025.0;
  s = fma(s, q, -135135.0);
  s = fma(s, q, 10395.0);
  s = fma(s, q, -945.0);
  s = fma(s, q, 105.0);
  s = fma(s, q, -15.0);
  s = fma(s, q, 3.0);
  s = fma(s, q, -1.0);
  s = fma(s, q, 1.0);
  return s * iw;
}

// Table-driven FP64 logarithm and exponential (P. T. P. Tang's method, ACM TOMS
// 16(4) 1990 and 15(2) 1989; tables by gen_elementary_tables.py).  Both are
// within 1 ulp and run almost wholly as fma on the FP64 pipe: the table
// index and the exponent come from bit patterns and the rounding of a value
// plus 1.5 2^52, not from floor or conversion instructions.
//   log: v = 2^e m, c = 1 + j/1024 nearest m (j in [0, 1024]), f = (m - c)/c,
//        ln v = (e ln2_hi + ln c_hi) + (e ln2_lo + ln c_lo + ln(1 + f)),
//        ln(1 + f) to degree 5 (|f| <= 1/2048, truncation below f^6/6 ~ 2^-66);
//        the hi sum is exact, and near v = 1 (j = 0, or j = 1024 with e = -1)
//        both sums reduce to ln(1 + f).  (A 129-entry table needed degree 7:
//        the 1,025 entries, 24 KB, cost two FMAs less per logarithm.)
//   exp: v = n ln2/128 + r, |r| <= ln2/256: e^v = 2^(n >> 7) 2^((n & 127)/128) e^r,
//        e^r - 1 to degree 5.
// Inputs outside their plain range (log: not positive normal finite; exp:
// |v| >= 708) take the library functions.
#include "elementary_tables.inc"

__device__ __forceinline__ double log_fp64(double v) {
  const uint64_t b = uint64_t(__double_as_longlong(v));
  if (b - 0x0010000000000000ull >= 0x7fe0000000000000ull) return ::log(v);
  const int e = int(b >> 52) - 1023;
  const double m = __longlong_as_double(int64_t((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  const double tr = fma(m - 1.0, 1024.0, 6755399441055744.0);
  const int j = int(uint64_t(__double_as_longlong(tr)) & 0x7ffull);
  const double jd = tr - 6755399441055744.0;
  const double f = (m - fma(jd, 0.0009765625, 1.0)) * __ldg(&kLogInvC[j]);
  double q = 0.2;
  q = fma(q, f, -0.25);
  q = fma(q, f, 1.0 / 3.0);
  q = fma(q, f, -0.5);
  q = fma(q, f, 1.0);
  const double ed = __longlong_as_double(0x4338000000000000LL + e) - 6755399441055744.0; // double(e)
  const double hi = fma(ed, kLn2Hi, __ldg(&kLogCHi[j]));
  const double lo = fma(ed, kLn2Lo, __ldg(&kLogCLo[j])) + q * f;
  return hi + lo;
}

__device__ __forceinline__ double exp_fp64(double v) {
  if ((uint64_t(__double_as_longlong(v)) & 0x7fffffffffffffffull) >= 0x4086200000000000ull) return ::exp(v); // |v| >= 708
  const double tr = fma(v, k128ByLn2, 6755399441055744.0);
  const int n = int(__double_as_longlong(tr)); // the low 32 bits: round(128 v / ln 2)
  const double fn = tr - 6755399441055744.0;
  double r = fma(-fn, kLn2By128Hi, v);
  r = fma(-fn, kLn2By128Lo, r);
  double p = 1.0 / 120.0;
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p *= r;
  const int k = n & 127;
  const double th = __ldg(&kExp2Hi[k]);
  const double res = fma(th, p, __ldg(&kExp2Lo[k])) + th;
  return __longlong_as_double(__double_as_longlong(res) + (int64_t(n >> 7) << 52));
}

// Y(z) = Phi(z)/phi(z) for any z: M(-z) for z <= 0, and for z > 0 the reflection
// Y(z) = 1/phi(z) - Y(-z) = sqrt(2 pi) e^{z^2/2} - M(z), with z^2 split exactly by an fma
__device__ __forceinline__ double mills_fp64(double z) {
  if (__double_as_longlong(z) <= 0) return mills_neg(-z); // z <= 0 (and -0)
  const double p = z * z, e = fma(z, z, -p);              // z^2 = p + e exactly
  const double ex = kSqrt2Pi * exp_fp64(0.5 * p);
  return !(p >= 1418.0) ? fma(ex, 0.5 * e, ex) - mills_neg(z) : INFINITY; // NaN stays NaN
}

template <>
struct Math<double> {
  // erfcx(v / sqrt 2) = sqrt(2/pi) M(v) for v >= 0
  static __device__ __forceinline__ double erfcx_half_(double v) { return 0.797884560802865355880 * mills_neg(v); }
  static __device__ __forceinline__ double exp_(double v) { return exp_fp64(v); }
  static __device__ __forceinline__ double log_(double v) { return log_fp64(v); }
  static __device__ __forceinline__ double sqrt_(double v) { return ::sqrt(v); }
  // the LBR node's s_c = sqrt(2|x|), which only places the guess's interpolation nodes: the float
  // square root (relative error ~6e-8, against the guess's ~1e-2 interpolation error)
  static __device__ __forceinline__ double sqrt_node_(double v) { return double(::sqrtf(float(v))); }
  // the guesses' cube roots, to seed accuracy (~1e-7 relative, against the guess's ~1e-2
  // interpolation error): v = m 2^(3q + r) with m in [1, 2), r in {0, 1, 2} from the exponent
  // bits, the float cube root of m 2^r, and q added to its exponent as an integer; arguments
  // outside the positive normal range take the library's FP64 cbrt
  static __device__ __forceinline__ double cbrt_(double v) {
    const int64_t b = __double_as_longlong(v);
    if (!(b > 0x000fffffffffffffLL && b < 0x7ff0000000000000LL)) return ::cbrt(v);
    const int e = int(b >> 52) - 1023;
    const int q = (e >= 0 ? e : e - 2) / 3; // floor(e / 3)
    const int r = e - 3 * q;
    const float m = __int_as_float(0x3f800000 | int((b >> 29) & 0x7fffff)) * float(1 << r);
    const uint32_t cb = __float_as_uint(::cbrtf(m)); // in [1, 2)
    return __longlong_as_double(int64_t((uint64_t(((cb >> 23) & 0xff) - 127 + 1023 + q) << 52) |
                                        (uint64_t(cb & 0x7fffff) << 29)));
  }
  static __device__ __forceinline__ double ncdf_(double v) { return ::normcdf(v); }
  static __device__ __forceinline__ double fma_(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double fmin_(double a, double b);
  static __device__ __forceinline__ double fmax_(double a, double b);
  static constexpr double kTiny = 1e-290;     // below this a cube root argument is scaled
  static constexpr double kScaleUp = 0x1p300;  // 2^300
  static constexpr double kScaleDown = 0x1p-100; // its cube root, inverted
};
template <>
struct Math<float> {
  static __device__ __forceinline__ float erfcx_(float v) { return ::erfcxf(v); }
  static __device__ __forceinline__ float erfcx_half_(float v) { return ::erfcxf(v * float(kInvSqrt2)); }
  static __device__ __forceinline__ float exp_(float v) { return ::expf(v); }
  static __device__ __forceinline__ float log_(float v) { return ::logf(v); }
  static __device__ __forceinline__ float sqrt_(float v) { return ::sqrtf(v); }
  static __device__ __forceinline__ float sqrt_node_(float v) { return ::sqrtf(v); }
  static __device__ __forceinline__ float cbrt_(float v) { return ::cbrtf(v); }
  static __device__ __forceinline__ float ncdf_(float v) { return ::normcdff(v); }
  static __device__ __forceinline__ float fma_(float a, float b, float c) { return ::fmaf(a, b, c); }
  static __device__ __forceinline__ float fmin_(float a, float b) { return ::fminf(a, b); }
  static __device__ __forceinline__ float fmax_(float a, float b) { return ::fmaxf(a, b); }
  static constexpr float kTiny = 1e-35f;
  static constexpr float kScaleUp = 0x1p60f;
  static constexpr float kScaleDown = 0x1p-20f;
};

// Quotients off the rounding-critical path.  An IEEE double division is a reciprocal estimate,
// refinement, a correction of the quotient and a special-case test, ~8 FP64 instructions; where
// the quotient only feeds a guess, a Householder correction or a derivative ratio, the
// reciprocal of a normal d from the hardware estimate (rcp.approx.ftz.f64) refined by two
// Newton-Raphson steps y <- y + y (1 - d y) (each doubles the correct bits; P. Markstein, IBM J.
// Res. Dev. 34(1), 1990) serves: 4 FMAs, within 1 ulp of 1/d (it matched the IEEE reciprocal on
// every one of 2^30 sampled normal d).  a / d is then a * (1/d), within 2 ulps.
__device__ __forceinline__ double rcp_normal(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}
// a / d to 2 ulps; d outside [2^-1022, 2^1021) in magnitude (zero, subnormal, huge, inf, NaN) takes the
// IEEE division, whose special cases the estimate would flush
__device__ __forceinline__ double div_fast(double a, double d) {
  const uint64_t m = uint64_t(__double_as_longlong(d)) & 0x7fffffffffffffffull;
  if (m - 0x0010000000000000ull < 0x7fb0000000000000ull) return a * rcp_normal(d);
  return a / d;
}
// the same in either precision: float keeps its own division
__device__ __forceinline__ double quot(double a, double d) { return div_fast(a, d); }
__device__ __forceinline__ float quot(float a, float d) { return a / d; }

// Y(z) = Phi(z)/phi(z).  Kept out of line: it is called from many sites and
// one shared copy keeps the kernels' instruction footprint small.
static __device__ __noinline__ double mills_any(double z) { return mills_fp64(z); }
static __device__ __noinline__ float mills_any(float z) { return float(kSqrtPiOver2) * ::erfcxf(-z * float(kInvSqrt2)); }
template <typename R>
__device__ __forceinline__ R mills_y(R z) {
  return mills_any(z);
}

// Y(z) for z <= 0: the table at -z, no reflection branch
static __device__ __noinline__ double mills_small(double z) { return mills_neg(-z); }
// ... in either precision (the float path keeps mills_y)
template <typename R>
__device__ __forceinline__ R mills_nonpos(R z);
template <>
__device__ __forceinline__ double mills_nonpos<double>(double z) { return mills_small(z); }
template <>
__device__ __forceinline__ float mills_nonpos<float>(float z) { return mills_y<float>(z); }

// ln b_s(x, s) = -(h^2 + t^2)/2 - ln sqrt(2 pi)
template <typename R>
__device__ __forceinline__ R log_bs(R h, R t) {
  return Math<R>::fma_(R(-0.5), Math<R>::fma_(h, h, t * t), R(-kLnSqrt2Pi));
}

template <typename R>
__device__ __forceinline__ R rho_taylor(R h, R t) {
  R c_prev = mills_nonpos<R>(h);            // c_0 (h <= 0)
  R c_cur = Math<R>::fma_(h, c_prev, R(1)); // c_1
  const R t2 = t * t;
  R acc = c_cur, tp = R(1);
  // c_{n+1} = (h c_n + c_{n-1}) / (n + 1), two steps per odd term
#pragma unroll
  for (int m = 1; m < 9; ++m) {
    const int n = 2 * m - 1;
    R c_next = Math<R>::fma_(h, c_cur, c_prev) * R(1.0 / double(n + 1));
    c_prev = c_cur;
    c_cur = c_next;
    c_next = Math<R>::fma_(h, c_cur, c_prev) * R(1.0 / double(n + 2));
    c_prev = c_cur;
    c_cur = c_next;
    tp *= t2;
    acc = Math<R>::fma_(c_cur, tp, acc);
  }
  return R(2) * t * acc;
}

// rho = b / b_s for x <= 0, s > 0
template <typename R>
__device__ __forceinline__ R rho_of(R x, R h, R t) {
  if (t <= R(kTaylorT) && x >= R(-kTaylorX)) return rho_taylor<R>(h, t);
  return mills_y<R>(h + t) - mills_y<R>(h - t);
}

// gamma = (b_max - b) / b_s
template <typename R>
__device__ __forceinline__ R gamma_of(R h, R t) {
  return mills_y<R>(-h - t) + mills_y<R>(h - t);
}

// Delbourgo-Gregory rational cubic Hermite interpolant on [z0, z1] through
// (z0, y0), (z1, y1) with end slopes d0, d1 and shape parameter r (r = 3 is
// the cubic Hermite; larger r pulls towards the chord).
template <typename R>
__device__ __forceinline__ R rational_cubic(R z, R z0, R z1, R y0, R y1, R d0, R d1, R r) {
  const R D = z1 - z0;
  const R tau = quot(z - z0, D);
  const R om = R(1) - tau;
  const R num = y0 * om * om * om + (r * y0 + D * d0) * tau * om * om + (r * y1 - D * d1) * tau * tau * om +
                y1 * tau * tau * tau;
  const R den = Math<R>::fma_((r - R(3)) * tau, om, R(1));
  return quot(num, den);
}

// Shape parameter with zero second derivative at the right end (z1) and at
// least the monotonicity bound (d0 + d1)/m of the Delbourgo-Gregory form.
// In the interpolant's own parameters S''(1) = 2 (D d0 + (r - 1) D d1 +
// r (y0 - y1)) / D^2 and S''(0) = -2 ((r - 1) D d0 + D d1 + r (y0 - y1)) / D^2.
template <typename R>
__device__ __forceinline__ R shape_zero_curv_right(R D, R y0, R y1, R d0, R d1) {
  const R r = quot(D * (d1 - d0), D * d1 + y0 - y1);
  const R rmono = quot((d0 + d1) * D, y1 - y0);
  return Math<R>::fmax_(r, rmono);
}
// ... zero second derivative at the left end (z0)
template <typename R>
__device__ __forceinline__ R shape_zero_curv_left(R D, R y0, R y1, R d0, R d1) {
  const R r = quot(D * (d0 - d1), D * d0 + y0 - y1);
  const R rmono = quot((d0 + d1) * D, y1 - y0);
  return Math<R>::fmax_(r, rmono);
}
template <typename R>
__device__ __forceinline__ R shape_monotone(R D, R y0, R y1, R d0, R d1) {
  return Math<R>::fmax_(R(3), quot((d0 + d1) * D, y1 - y0));
}

// ---------------------------------------------------------------------------
// Row preparation (Algorithm 1 forward normalisation with r = 0; appendix
// stages 1-2).
// ---------------------------------------------------------------------------
// Sign and class tests on the bit pattern: integer instructions, which leave
// the FP64 pipe (2 lanes per cycle per SM on this part) to the arithmetic.
// positive, finite and non-zero: bits - 1 < bits(+inf) - 1 as unsigned
__device__ __forceinline__ bool pos_finite(double v) {
  return uint64_t(__double_as_longlong(v)) - 1ull < 0x7fefffffffffffffull;
}
__device__ __forceinline__ bool finite64(double v) {
  return (uint64_t(__double_as_longlong(v)) & 0x7fffffffffffffffull) < 0x7ff0000000000000ull;
}
// positive and normal (neither zero, subnormal, infinite nor NaN)
__device__ __forceinline__ bool pos_normal(double v) {
  return uint64_t(__double_as_longlong(v)) - 0x0010000000000000ull < 0x7fe0000000000000ull;
}
// v < 0 for a non-NaN v (-0 is not negative)
__device__ __forceinline__ bool neg64(double v) {
  return uint64_t(__double_as_longlong(v)) > 0x8000000000000000ull;
}
// v == 0 (either sign)
__device__ __forceinline__ bool zero64(double v) { return (uint64_t(__double_as_longlong(v)) << 1) == 0ull; }
// a > b (a <= b) for non-negative finite a, b: their bit patterns order as integers
__device__ __forceinline__ bool gt_pos(double a, double b) { return __double_as_longlong(a) > __double_as_longlong(b); }
__device__ __forceinline__ bool le_pos(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }
// Order tests of arbitrary-sign doubles as integers: key(a) < key(b) iff a < b for non-NaN
// a, b (-0 sorts just below +0).  Overloaded for float (plain compares on the FP32 pipe).
__device__ __forceinline__ int64_t key64(double v) {
  const int64_t b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool nan64(double v) {
  return (uint64_t(__double_as_longlong(v)) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool cmp_lt(double a, double b) { return key64(a) < key64(b); }
__device__ __forceinline__ bool cmp_le(double a, double b) { return key64(a) <= key64(b); }
__device__ __forceinline__ bool cmp_lt(float a, float b) { return a < b; }
__device__ __forceinline__ bool cmp_le(float a, float b) { return a <= b; }
// v > 0 and v <= 0 from the sign and magnitude bits (a NaN with clear sign bit counts as > 0)
__device__ __forceinline__ bool gt0(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool le0(double v) { return __double_as_longlong(v) <= 0; }
__device__ __forceinline__ bool gt0(float v) { return v > 0.0f; }
__device__ __forceinline__ bool le0(float v) { return v <= 0.0f; }
// |d| < c for c >= 0
__device__ __forceinline__ bool abs_lt(double d, double c) {
  return (uint64_t(__double_as_longlong(d)) & 0x7fffffffffffffffull) < uint64_t(__double_as_longlong(c));
}
// fmin / fmax with their NaN rule (a NaN argument yields the other one), without the FP64 pipe
__device__ __forceinline__ double fmin64(double a, double b) {
  return (nan64(a) || (!nan64(b) && cmp_lt(b, a))) ? b : a;
}
__device__ __forceinline__ double fmax64(double a, double b) {
  return (nan64(a) || (!nan64(b) && cmp_lt(a, b))) ? b : a;
}
__device__ __forceinline__ double Math<double>::fmin_(double a, double b) { return fmin64(a, b); }
__device__ __forceinline__ double Math<double>::fmax_(double a, double b) { return fmax64(a, b); }

__device__ __forceinline__ bool bad_inputs(double F, double K, double T, int flag) {
  // also rejects NaN and +-inf
  return !pos_finite(F) || !pos_finite(K) || !pos_finite(T) || (flag != 1 && flag != -1);
}

// 2v for a non-negative finite double v from its bit pattern, on the integer pipes: a
// subnormal doubles its integer (crossing into the normal range correctly), a normal one
// gains one in its exponent, and beyond the range the result is +inf.  A negative v gives
// a negative pattern, which every *_pos test orders below all non-negative values.
__device__ __forceinline__ double twice_pos(double v) {
  const int64_t b = __double_as_longlong(v);
  const int64_t e = b >> 52;
  return __longlong_as_double(e == 0 ? (b << 1) : (e >= 2046 ? 0x7ff0000000000000LL : b + (1LL << 52)));
}

// -|ln(F/K)| from mn = min(F, K), mx = max(F, K), branch-free and accurate
// near the money: r = mn/mx is correctly rounded, so its residual
// c = (mn - r mx)/mn is exact to first order (one fma) and
// ln(mn/mx) = ln r + ln(1 + c) = ln r + c + O(c^2), |c| <= 2^-53.
__device__ __forceinline__ double neg_abs_log_ratio(double mn, double mx, double* ratio = nullptr) {
  const double r = div_fast(mn, mx);
  const double c = div_fast(fma(-r, mx, mn), mn);
  if (ratio) *ratio = r;
  return log_fp64(r) + c;
}

// The wide-range form of moneyness (F K outside the normal range, or min/max below it,
// i.e. |ln(F/K)| above ~708): rsq from the two factors, ln(min/max) from the IEEE quotient
// and its residual while the quotient is normal, else as the difference of two logarithms
// (no cancellation at that size).
static __device__ __noinline__ void moneyness_wide(double mn, double mx, double& x, double& bmax, double& rsq) {
  rsq = rsqrt(mn) * rsqrt(mx);
  bmax = mn * rsq;
  const double r = mn / mx;
  if (r >= 0x1p-1022) x = -fabs(::log(r) + fma(-r, mx, mn) / mn);
  else x = ::log(mn) - ::log(mx);
}

// b_max = min(F, K) / sqrt(F K) from rsq = 1/sqrt(F K): the one definition both
// phases use, so that a row's b_max is the same wherever it is formed
__device__ __forceinline__ double bmax_of(double F, double K, double rsq) { return (gt_pos(F, K) ? K : F) * rsq; }

// x = -|ln(F/K)|, b_max = e^{x/2} = sqrt(min/max) and rsq = 1/sqrt(F K) from one
// reciprocal square root: b_max = min(F, K) rsq, so r = b_max^2 is min/max to a few
// ulps, and its residual c = (min - r max)/min (one fma, then times 1/min = rsq^2 max)
// gives ln(min/max) = ln r + c to first order (|c| ~ 2^-50, its square far below
// rounding): no division and no square root.  The sign is forced: x is never above 0.
__device__ __forceinline__ void moneyness(double F, double K, double& x, double& bmax, double& rsq) {
  const bool fk = gt_pos(F, K); // F, K positive: integer order of the bit patterns
  const double mn = fk ? K : F, mx = fk ? F : K;
  const double p = F * K;
  rsq = rsqrt(p);
  bmax = mn * rsq;
  const double r = bmax * bmax;
  const uint64_t pb = uint64_t(__double_as_longlong(p)), rb = uint64_t(__double_as_longlong(r));
  if (pb - 0x0010000000000000ull < 0x7fe0000000000000ull && rb >= 0x0010000000000000ull) {
    const double c = fma(-r, mx, mn) * (rsq * rsq * mx);
    x = -fabs(log_fp64(r) + c);
  } else {
    moneyness_wide(mn, mx, x, bmax, rsq);
  }
}

// Stage 1 for one quote: validity, the time value tv = P - intrinsic (exact
// up to one rounding) and cv = U - P (U = F for calls, K for puts).  Rows that
// need no solve get their status and sigma here (Section 3.1: invalid rows
// are NaN; PIVOT_ROW_* codes).
struct Quote {
  double tv, cv;
  int status;   // 0: solve
  double sigma; // result when status != 0
};

__device__ __forceinline__ Quote classify_quote(double F, double K, double T, double P, int flag) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  Quote q;
  q.tv = q.cv = 0.0;
  q.status = 0;
  q.sigma = 0.0;
  if (bad_inputs(F, K, T, flag) || !finite64(P)) {
    q.status = 3;
    q.sigma = qnan;
    return q;
  }
  // U = a (F for calls, K for puts), intrinsic a - b in the money (a > b).  The time value
  // P - a + b is rounded once: by Sterbenz's lemma b - a is exact when a <= 2b, and P - a is
  // exact when a/2 <= P <= 2a, so P + (b - a) or (P - a) + b covers every price in or near the
  // no-arbitrage interval [a - b, a].  Below it, with a > 2b and P < a/2, P < a/2 < a - b: the
  // time value is negative whatever its rounding, and only its sign is used.  The same three
  // FP64 additions serve every lane (no branch), and U - P = -(P - a) exactly.
  const bool call = flag > 0;
  const double a = call ? F : K, b = call ? K : F;
  const bool itm = gt_pos(a, b);
  const double d = P - a;
  const bool near = le_pos(a, twice_pos(b));
  const double tv = (near ? P : d) + (near ? b - a : b);
  q.tv = !itm ? P : (!near && gt_pos(a, twice_pos(P))) ? -1.0 : tv;
  q.cv = -d;
  if (neg64(q.tv)) { q.status = 1; q.sigma = qnan; }
  else if (neg64(q.cv)) { q.status = 2; q.sigma = qnan; }
  else if (zero64(q.tv)) { q.status = 4; q.sigma = 0.0; }
  else if (zero64(q.cv)) { q.status = 5; q.sigma = INFINITY; }
  return q;
}

// ln beta for a solved row; beta near or below the subnormal range takes it
// from ln tv so that it keeps its relative accuracy
__device__ __forceinline__ double log_beta(double beta, double F, double K, double T, double P, int flag) {
  if (gt_pos(beta, 1e-290)) return log_fp64(beta);
  const Quote q = classify_quote(F, K, T, P, flag);
  return log_fp64(q.tv) + log_fp64(rsqrt(F * K));
}

// ---------------------------------------------------------------------------
// The LBR node as functions of u = |x| alone (appendix stage 4): with
// w = sqrt(u), e = erfcx(w), s_l = s_c - sqrt(pi/2)(1 - e) and
// s_u = s_c + sqrt(pi/2)(1 + e), the node values scale with b_max:
//   b_l = b_max u FL(w), b_s(s_l) = b_max GL(w), b_max - b_u = b_max FU(w),
//   b_s(s_u) = b_max GU(w), s_l = u SL(w)
// (node_table.inc, degree-6 Chebyshev pieces in float on 97 intervals of
// [0, 64) indexed by the bit pattern of w, generated with mpmath by
// gen_node_table.py, ~1e-7 relative).  The node only places the guess's
// interpolation nodes and the region tests, so float precision is far below
// the guess's own interpolation error; SL keeps s_l's relative accuracy where
// s_c - sqrt(pi/2)(1 - e) would cancel (u -> 0).  u >= 4096 (|F/K| beyond
// e^4096) takes the evaluated node, and so does the float node of the mixed
// form, whose evaluation runs on the FP32 pipe and costs less than the table's
// loads and conversions.
// ---------------------------------------------------------------------------
#include "node_table.inc"

constexpr int kNodeDeg = 6;
constexpr float kNodeMaxU = 4096.0f;

// a non-negative double below 2^128 as a float by its bits (mantissa truncated; values
// below the float normal range give 0): integer instructions only
__device__ __forceinline__ float pos_to_float(double v) {
  const uint64_t b = uint64_t(__double_as_longlong(v));
  const int ef = int(b >> 52) - 1023 + 127;
  if (ef <= 0) return 0.0f;
  return __uint_as_float((uint32_t(ef) << 23) | uint32_t((b >> 29) & 0x7fffff));
}
// a positive normal float (or 0) as a double by its bits: integer instructions only
__device__ __forceinline__ double pos_to_double(float f) {
  const uint32_t b = __float_as_uint(f);
  if (b == 0u) return 0.0;
  return __longlong_as_double(int64_t((uint64_t((b >> 23) - 127 + 1023) << 52) | (uint64_t(b & 0x7fffff) << 29)));
}
template <typename R>
__device__ __forceinline__ R from_float(float f);
template <>
__device__ __forceinline__ double from_float<double>(float f) { return pos_to_double(f); }
template <>
__device__ __forceinline__ float from_float<float>(float f) { return f; }
template <typename R>
__device__ __forceinline__ float to_float(R v);
template <>
__device__ __forceinline__ float to_float<double>(double v) { return pos_to_float(v); }
template <>
__device__ __forceinline__ float to_float<float>(float v) { return v; }

struct NodeTab {
  float w, e, sl_u, fl_u, gl, fu, gu;
};

__device__ __forceinline__ float node_poly(const float* c, float tau) {
  float v = __ldg(c + kNodeDeg);
#pragma unroll
  for (int j = kNodeDeg - 1; j >= 0; --j) v = fmaf(v, tau, __ldg(c + j));
  return v;
}

// the node functions at u (float, 0 <= u < kNodeMaxU)
__device__ __forceinline__ NodeTab node_tab(float u) {
  NodeTab t;
  t.w = sqrtf(u);
  const uint32_t bits = __float_as_uint(t.w);
  // biased exponent and top three mantissa bits, less those of 1/64, plus one (0 below 1/64)
  const int k = max(int(bits >> 20) - ((127 - 6) << 3) + 1, 0);
  const float* c = kNodeCoef[k];
  const float tau = fmaf(t.w, __ldg(c), __ldg(c + 1));
  c += 2;
  t.e = node_poly(c, tau);
  t.sl_u = node_poly(c + (kNodeDeg + 1), tau);
  t.fl_u = node_poly(c + 2 * (kNodeDeg + 1), tau);
  t.gl = node_poly(c + 3 * (kNodeDeg + 1), tau);
  t.fu = node_poly(c + 4 * (kNodeDeg + 1), tau);
  t.gu = node_poly(c + 5 * (kNodeDeg + 1), tau);
  return t;
}

// s_l = u SL(w) alone (the guesses)
__device__ __forceinline__ float node_sl_u(float u, float& w) {
  w = sqrtf(u);
  const uint32_t bits = __float_as_uint(w);
  const int k = max(int(bits >> 20) - ((127 - 6) << 3) + 1, 0);
  const float* c = kNodeCoef[k];
  const float tau = fmaf(w, __ldg(c), __ldg(c + 1));
  return node_poly(c + 2 + (kNodeDeg + 1), tau);
}

// ---------------------------------------------------------------------------
// LBR boundary, region and rational initial guess (appendix stage 4).
// The boundary is the inflection point s_c = sqrt(2|x|) of b(x, .) and the
// two points s_l, s_u where its tangent there reaches 0 and b_max.  In closed
// form, with e = erfcx(sqrt|x|):
//   b_c = b_max (1 - e)/2,  b_s(s_c) = b_max/sqrt(2 pi),
//   s_l = s_c - sqrt(pi/2)(1 - e),  s_u = s_c + sqrt(pi/2)(1 + e).
// Only one of b_l = b(s_l), b_u = b(s_u) is needed per row (the side of b_c
// that beta is on); both cost two erfcx and one exp and are evaluated by the
// same branch-free code: b_l = b_s (Y(h + t) - Y(h - t)) and
// b_max - b_u = b_s (Y(-h - t) + Y(h - t)).  The node only seeds the guess,
// so the difference form is accurate enough for it everywhere.
// ---------------------------------------------------------------------------
template <typename R>
struct Node {
  R x;    // -|ln(F/K)|
  R bmax; // e^{x/2}
  R e;    // erfcx(sqrt|x|)
  R bn;   // b_l (lower side) or b_max - b_u (upper side)
  R bsn;  // b_s at that node
  R bb;   // beta, or beta_c = b_max - beta in the upper region
};

template <typename R>
__device__ __forceinline__ int classify(R x, R bmax, R beta, R betac, Node<R>& nd) {
  using M = Math<R>;
  const R ax = -x;
  const float uf = to_float<R>(ax);
  if (sizeof(R) == 8 && uf < kNodeMaxU) {
    // the tabulated node: b_c, and b_l, b_s(s_l) or b_max - b_u, b_s(s_u), all times b_max
    const NodeTab tb = node_tab(uf);
    const R e = from_float<R>(tb.e);
    const R bc = R(0.5) * bmax * (R(1) - e);
    const bool low = cmp_le(beta, bc);
    nd.x = x;
    nd.bmax = bmax;
    nd.e = e;
    nd.bn = bmax * (low ? ax * from_float<R>(tb.fl_u) : from_float<R>(tb.fu));
    nd.bsn = bmax * from_float<R>(low ? tb.gl : tb.gu);
    int region;
    if (low) region = cmp_lt(beta, nd.bn) ? kLower : kMidLow;
    else region = cmp_le(beta, bmax - nd.bn) ? kMidHigh : kUpper;
    nd.bb = (region == kUpper) ? betac : beta;
    return region;
  }
  const R sc = M::sqrt_node_(R(2) * ax);
  const R e = M::erfcx_half_(sc); // erfcx(sqrt|x|), sc >= 0
  const R bc = R(0.5) * bmax * (R(1) - e);
  const bool low = cmp_le(beta, bc);
  const R sl = sc - R(kSqrtPiOver2) * (R(1) - e);
  const R su = sc + R(kSqrtPiOver2) * (R(1) + e);
  const bool has_l = gt0(sl);
  const R sn = low ? (has_l ? sl : R(1)) : su;
  const R h = quot(x, sn), t = R(0.5) * sn;
  // both arguments are <= 0: h + t < 0 below s_c, -h - t < 0 above it, h - t < 0 always
  const R y1 = mills_nonpos<R>(low ? h + t : -h - t);
  const R y2 = mills_nonpos<R>(h - t);
  const R bs = M::exp_(log_bs<R>(h, t));
  const R val = bs * (low ? y1 - y2 : y1 + y2);
  nd.x = x;
  nd.bmax = bmax;
  nd.e = e;
  nd.bn = (low && !has_l) ? R(0) : val;
  nd.bsn = bs;
  int region;
  if (low) region = cmp_lt(beta, nd.bn) ? kLower : kMidLow;
  else region = cmp_le(beta, bmax - val) ? kMidHigh : kUpper;
  nd.bb = (region == kUpper) ? betac : beta;
  return region;
}

// -Phi^{-1}(G) for the guesses, G in (0, 1/2].  In double, for G from 1e-37
// on (the float range) and where `fast` (rows with beta >= kDeepBeta, whose
// lower-region G stays above ~1e-35): the float inverse normal CDF, within a
// few float ulps (relative error ~1e-6 in the guess), five orders of magnitude
// below the guess's own interpolation error (~1e-2), which the FP64
// Householder steps remove.  Other arguments take the library's FP64 function.
constexpr double kDeepBeta = 1e-100;
template <typename R>
__device__ __forceinline__ R neg_ncdfinv(R G, bool fast);
template <>
__device__ __forceinline__ float neg_ncdfinv<float>(float G, bool) { return -::normcdfinvf(G); }
template <>
__device__ __forceinline__ double neg_ncdfinv<double>(double G, bool fast) {
  if (fast && cmp_le(1e-37, G)) return -double(::normcdfinvf(float(G)));
  return -::normcdfinv(G);
}

// Rational initial guess s^(0) of the row's region from its node.
// lnbeta is ln beta (lower region only).
// kFastInv: -Phi^{-1} by neg_ncdfinv's float start and Newton step where it applies (else the
// library function throughout)
// s_c and (for the sides below the inflection) s_l of a row's node: from the node table
// while |x| < 4096, where s_l = |x| SL keeps its relative accuracy as |x| -> 0
template <typename R>
__device__ __forceinline__ R node_sc(R ax, float uf) {
  return (sizeof(R) == 8 && uf < kNodeMaxU) ? R(kSqrt2) * from_float<R>(sqrtf(uf)) : Math<R>::sqrt_node_(R(2) * ax);
}
template <typename R>
__device__ __forceinline__ R node_sl(R ax, float uf, R sc, R e) {
  if (sizeof(R) == 8 && uf < kNodeMaxU) {
    float w;
    return ax * from_float<R>(node_sl_u(uf, w));
  }
  return sc - R(kSqrtPiOver2) * (R(1) - e);
}

// exp(-a^2/2) and Phi(-a) = exp(-a^2/2) erfcx(a/sqrt 2) / 2 for a >= 0, as the lower and upper
// guesses use them: they place a rational interpolation's end value and slope, so the FP64 form
// takes them at float precision (~1e-7 relative, against the guess's ~1e-2 interpolation error)
// while exp(-a^2/2) is a normal float (a < 9), and in FP64 beyond.
template <typename R>
__device__ __forceinline__ void seed_tail(R a, R& ea, R& Pa) {
  using M = Math<R>;
  if (sizeof(R) == 8 && cmp_lt(double(a), 9.0)) {
    const float af = float(a);
    const float e = ::expf(-0.5f * af * af);
    ea = R(e);
    Pa = R(0.5f * e * Math<float>::erfcx_half_(af));
    return;
  }
  ea = M::exp_(R(-0.5) * a * a);
  Pa = R(0.5) * ea * M::erfcx_half_(a);
}

template <typename R, bool kFastInv = true>
__device__ __forceinline__ R region_guess(int region, const Node<R>& nd, R lnbeta) {
  using M = Math<R>;
  const R x = nd.x, ax = -x;
  const float uf = to_float<R>(ax);
  const R sc = node_sc<R>(ax, uf);
  const R e = nd.e;
  switch (region) {
    case kLower: {
      // lower tail: b ~ kappa Phi(-|x|/(sqrt3 s))^3 as s -> 0, kappa = 2 pi |x| / (3 sqrt 3).
      // Interpolate G = Phi(-|x|/(sqrt3 s)) against u = (beta/kappa)^(1/3) on [0, u_l]
      // (G(0) = 0, G'(0) = 1, G(u_l), G'(u_l) exact), then invert G for s.
      const R sl = node_sl<R>(ax, uf, sc, e);
      const R bl = nd.bn, bsl = nd.bsn, beta = nd.bb;
      const R kap = R(kTwoPiOver3Sqrt3) * ax, inv_kap = quot(R(1), kap);
      // u = (beta/kappa)^(1/3); below ~1e-290 the cube root of the argument scaled by 2^300 times
      // 2^-100 (exact scalings, no branch), and through ln beta only where beta/kappa underflowed
      const R v = beta * inv_kap;
      const bool tiny = cmp_lt(v, M::kTiny);
      R u = M::cbrt_(tiny ? v * M::kScaleUp : v) * (tiny ? M::kScaleDown : R(1));
      if (__builtin_expect(!gt0(v), 0)) u = M::exp_((lnbeta - M::log_(kap)) * R(1.0 / 3.0));
      const R ul = M::cbrt_(bl * inv_kap);
      // a_l only places the interpolation's end point: a float quotient in the FP64 form
      const R al = sizeof(R) == 8 ? R(float(ax) * float(kInvSqrt3) / float(sl)) : quot(ax * R(kInvSqrt3), sl);
      // Phi(-al) = phi(al) Y(-al) = exp(-al^2/2) erfcx(al/sqrt 2) / 2: one exponential shared with phi(al)
      R eal, Gl;
      seed_tail<R>(al, eal, Gl);
      const R dGl = quot(R(3) * bl * (R(kInvSqrt2Pi) * eal) * al, sl * ul * bsl);
      const R r = shape_monotone<R>(ul, R(0), Gl, R(1), dGl);
      const R G = M::fmin_(rational_cubic<R>(u, R(0), ul, R(0), Gl, R(1), dGl, r), R(0.5));
      return quot(ax * R(kInvSqrt3), neg_ncdfinv<R>(G, kFastInv && cmp_le(kDeepBeta, double(beta))));
    }
    case kMidLow: {
      // rational cubic in b on [b_l, b_c], zero curvature of s(b) at the inflection b_c
      const R dc = quot(R(kSqrt2Pi), nd.bmax); // ds/db at s_c
      const R sl = node_sl<R>(ax, uf, sc, e);
      const R bc = R(0.5) * nd.bmax * (R(1) - e);
      const R bl = nd.bn;
      const bool blp = gt0(bl);
      const R d0 = blp ? quot(R(1), nd.bsn) : dc;
      const R s0 = blp ? sl : R(0);
      const R D = bc - bl;
      const R r = shape_zero_curv_right<R>(D, s0, sc, d0, dc);
      return rational_cubic<R>(nd.bb, bl, bc, s0, sc, d0, dc, r);
    }
    case kMidHigh: {
      // rational cubic in b on [b_c, b_u], zero curvature of s(b) at b_c
      const R dc = quot(R(kSqrt2Pi), nd.bmax);
      const R su = sc + R(kSqrtPiOver2) * (R(1) + e);
      const R bc = R(0.5) * nd.bmax * (R(1) - e);
      const R bu = nd.bmax - nd.bn;
      const R d1 = quot(R(1), nd.bsn);
      const R D = bu - bc;
      const R r = shape_zero_curv_left<R>(D, sc, su, dc, d1);
      return rational_cubic<R>(nd.bb, bc, bu, sc, su, dc, d1, r);
    }
    default: {
      // upper tail: b_max - b ~ 2 Phi(-s/2) as s -> inf.  Interpolate
      // v = Phi(-s/2) against u = (b_max - beta)/2 on [0, u_u], v'(0) = 1.
      const R su = sc + R(kSqrtPiOver2) * (R(1) + e);
      const R uu = R(0.5) * nd.bn;
      // Phi(-su/2) and phi(su/2) from one exponential, as in the lower region
      R esu, vu;
      seed_tail<R>(R(0.5) * su, esu, vu);
      const R dvu = quot(R(kInvSqrt2Pi) * esu, nd.bsn);
      const R r = shape_monotone<R>(uu, R(0), vu, R(1), dvu);
      const R v = M::fmin_(rational_cubic<R>(R(0.5) * nd.bb, R(0), uu, R(0), vu, R(1), dvu, r), R(0.5));
      return R(2) * neg_ncdfinv<R>(v, kFastInv);
    }
  }
}

// ---------------------------------------------------------------------------
// One Householder(3) step (appendix stage 5) on the region's objective
//   lower:  f = 1/ln b(s) - 1/ln beta
//   middle: f = b(s) - beta
//   upper:  f = ln(b_max - beta) - ln(b_max - b(s))
// with b2 = b''/b' = x^2/s^3 - s/4 and b3 = b'''/b' = b2^2 - 3x^2/s^4 - 1/4:
//   s <- s + nu (1 + h2 nu / 2) / (1 + nu (h2 + h3 nu / 6)),
//   nu = -f/f', h2 = f''/f', h3 = f'''/f'.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R householder_step(R x, R beta, R lnbetac, R inv_lnbeta, int region, R s) {
  using M = Math<R>;
  const R inv_s = R(1) / s;
  const R h = x * inv_s, t = R(0.5) * s;
  const R hh = h * h;
  const R b2 = (hh - t * t) * inv_s;                                  // b''/b'
  const R b3 = M::fma_(b2, b2, R(-3) * hh * inv_s * inv_s) - R(0.25); // b'''/b'
  R nu, h2, h3;
  if (region == kLower) {
    const R rho = rho_of<R>(x, h, t);
    const R L = log_bs<R>(h, t) + M::log_(rho); // ln b
    const R q = R(1) / rho;                     // (ln b)' = b'/b
    const R iL = R(1) / L;
    // nu = -(1/L - 1/Lb) L^2 / q = rho L (Lb - L) / Lb
    nu = rho * L * (R(1) - L * inv_lnbeta);
    h2 = b2 - q * M::fma_(R(2), iL, R(1));
    h3 = b3 - R(3) * b2 * q + R(2) * q * q - R(6) * q * (b2 - q) * iL + R(6) * q * q * iL * iL;
  } else if (region == kUpper) {
    const R gam = gamma_of<R>(h, t);
    const R pg = R(1) / gam; // b'/(b_max - b)
    const R f = lnbetac - log_bs<R>(h, t) - M::log_(gam);
    nu = -f * gam;
    h2 = b2 + pg;
    h3 = b3 + R(3) * pg * b2 + R(2) * pg * pg;
  } else {
    const R rho = rho_of<R>(x, h, t);
    const R bs = M::exp_(log_bs<R>(h, t));
    nu = beta / bs - rho; // (beta - b)/b'
    h2 = b2;
    h3 = b3;
  }
  const R num = nu * M::fma_(R(0.5) * h2, nu, R(1));
  const R den = M::fma_(nu, M::fma_(h3 * R(1.0 / 6.0), nu, h2), R(1));
  return s + num / den;
}

// ---------------------------------------------------------------------------
// The FP64 Householder(3) step of the binned kernels.  Same objectives as
// householder_step<double>, evaluated through the two Mills ratios of
// non-positive argument only (one table evaluation each, no exponential):
//   ya = Y(-|h + t|),  yb = Y(h - t)   (h - t < 0 always)
// and the reflection Y(z) + Y(-z) = 1/phi(z), which at z = h + t reads
//   Y(h + t) + Y(-h - t) = b_max / b_s = E1          (e^{x/2} phi(h+t) = b_s)
// so the larger ratio costs one multiply once 1/b_s is known:
//   rho   = ya - yb            (h + t <= 0),  E1 - ya - yb   (h + t > 0)
//   gamma = ya + yb            (h + t > 0),   E1 - ya + yb   (h + t <= 0)
// (the same cancellation as Y(h+t) - Y(h-t) itself).  The middle objective's
// Newton ratio nu = (beta - b)/b_s = beta / b_s - rho takes 1/b_s = exp(-ln b_s)
// once.  The step records where it evaluated (z_a = -|h + t|, z_b = h - t)
// and the two ratios, so that the adjoint at the final iterate needs no new
// Mills ratio (adjoint_reuse).
// kF32Ratios: the derivative ratios h2, h3 of the step (and those of b) in
// float.  For the last step of the mixed form, whose iterate is within ~1e-6
// relative, they only enter through nu (h2 nu / 2 + ...) ~ nu^2: their float
// rounding moves s by ~1e-7 nu^2, below double rounding.  nu itself, the
// residual, stays double.
// ---------------------------------------------------------------------------
// 1/s for an iterate s > 0.  Roots below 2^-1000 occur only at the money (x = 0, a time
// value near or below the subnormal range), where h = x/s = 0 whatever s is and the other
// products with 1/s carry a power of s that has already underflowed; there 1/s itself would
// overflow (s subnormal) and turn h into 0 * inf.  The reciprocal is taken of max(s, 2^-1000),
// the maximum by an integer compare of the bit patterns (no rounding-critical use: an error of
// 1/s moves the evaluation point, not the step's target).
__device__ __forceinline__ double inv_iterate(double s) {
  return div_fast(1.0, le_pos(s, 0x1p-1000) ? 0x1p-1000 : s);
}

struct Last {
  double s;      // the iterate of the last evaluation
  double za, zb; // arguments of the two Mills ratios there
  double ya, yb; // Y(za), Y(zb)
  double lbs;    // ln b_s there
  double ibs;    // 1/b_s there, or 0 when the step did not form it
  bool pair;     // false: the Taylor zone of rho evaluated neither
};


template <bool kF32Ratios>
__device__ __forceinline__ double step64(double x, double bmax, double beta, double lnbetac, double inv_lnbeta,
                                         int region, double s, Last& last) {
  const double inv_s = inv_iterate(s);
  const double h = x * inv_s, t = 0.5 * s, hpt = h + t;
  const double lbs = log_bs<double>(h, t);
  const bool taylor = region != kUpper && le_pos(t, kTaylorT) && le_pos(-x, kTaylorX);
  last.s = s;
  last.za = -fabs(hpt);
  last.zb = h - t;
  last.pair = !taylor;
  double ya = 0.0, yb = 0.0;
  if (!taylor) {
    ya = mills_small(last.za);
    yb = mills_small(last.zb);
  }
  last.ya = ya;
  last.yb = yb;
  last.lbs = lbs;
  // 1/b_s where the middle objective or the larger ratio of the pair needs it
  const bool hpos = gt0(hpt);
  const bool need_ibs = region == kMidLow || region == kMidHigh || (region == kLower ? hpos : !hpos);
  double ibs = need_ibs ? exp_fp64(-lbs) : 0.0;
  double E1 = bmax * ibs;
  double beta_ibs = beta * ibs;
  last.ibs = need_ibs ? ibs : 0.0; // for adjoint_reuse (0: not formed)
  if (!finite64(ibs)) {
    // b_s below ~1e-308 (|ln(F/K)| beyond ~1400): the products in logarithms
    E1 = kSqrt2Pi * exp_fp64(0.5 * hpt * hpt);
    beta_ibs = exp_fp64(log_fp64(beta) - lbs);
    last.ibs = 0.0;
  }
  double nu, L = 0.0, q = 0.0, iL = 0.0;
  if (region == kUpper) {
    const double gam = hpos ? ya + yb : (E1 - ya) + yb;
    q = div_fast(1.0, gam);
    nu = -(lnbetac - lbs - log_fp64(gam)) * gam;
  } else {
    const double rho = taylor ? rho_taylor<double>(h, t) : (!hpos ? ya - yb : (E1 - ya) - yb);
    if (region == kLower) {
      L = lbs + log_fp64(rho); // ln b
      // 1/rho and 1/L from one division: 1/rho = L / (rho L), 1/L = rho / (rho L)
      const double inv = div_fast(1.0, rho * L);
      q = L * inv;
      iL = rho * inv;
      nu = rho * L * (1.0 - L * inv_lnbeta);
    } else {
      nu = beta_ibs - rho;
    }
  }
  if (kF32Ratios) {
    const float fis = float(inv_s), fh = float(h), ft = float(t), fhh = fh * fh;
    const float b2 = (fhh - ft * ft) * fis;
    const float b3 = fmaf(b2, b2, -3.0f * fhh * fis * fis) - 0.25f;
    float h2 = b2, h3 = b3;
    const float fq = float(q);
    if (region == kLower) {
      const float fiL = float(iL);
      h2 = b2 - fq * fmaf(2.0f, fiL, 1.0f);
      h3 = b3 - 3.0f * b2 * fq + 2.0f * fq * fq - 6.0f * fq * (b2 - fq) * fiL + 6.0f * fq * fq * fiL * fiL;
    } else if (region == kUpper) {
      h2 = b2 + fq;
      h3 = b3 + 3.0f * fq * b2 + 2.0f * fq * fq;
    }
    // (1 + h2 nu/2) / (1 + nu (h2 + h3 nu/6)) - 1 = -nu (h2/2 + h3 nu/6) / (1 + nu (h2 + h3 nu/6))
    const float fnu = float(nu);
    const float a = fmaf(h3 * (1.0f / 6.0f), fnu, h2);
    const float corr = -fnu * fmaf(h3 * (1.0f / 6.0f), fnu, 0.5f * h2) / fmaf(fnu, a, 1.0f);
    return s + fma(nu, double(corr), nu);
  }
  // b''/b' = x^2/s^3 - s/4 = h w - s/4 and b'''/b' = (b''/b')^2 - 3 w^2 - 1/4, w = h/s
  const double w = h * inv_s;
  const double b2 = fma(h, w, -0.25 * s);
  const double b3 = fma(b2, b2, fma(-3.0 * w, w, -0.25));
  double h2 = b2, h3 = b3;
  if (region == kLower) {
    h2 = b2 - q * fma(2.0, iL, 1.0);
    // b3 - 3 b2 q + 2 q^2 - 6 q (b2 - q) iL + 6 q^2 iL^2 = b3 + q (2 q - 3 b2 + 6 iL (q iL + q - b2))
    h3 = fma(q, fma(6.0 * iL, fma(q, iL, q - b2), fma(-3.0, b2, q + q)), b3);
  } else if (region == kUpper) {
    h2 = b2 + q;
    h3 = fma(q, fma(3.0, b2, q + q), b3); // b3 + 3 q b2 + 2 q^2
  }
  const double num = nu * fma(0.5 * h2, nu, 1.0);
  const double den = fma(nu, fma(h3 * (1.0 / 6.0), nu, h2), 1.0);
  return s + div_fast(num, den);
}


// The final FP64 step of the mixed form.  Its iterate comes from the float
// solve (within ~1e-6 relative), so every region takes the Newton ratio of
// f = b - beta, written without logarithms (beta and beta_c exact in double):
//   nu = (beta - b) / b_s = beta / b_s - rho                 (lower, middle)
//      = gamma - beta_c / b_s                                (upper, b_max - b = b_s gamma)
// and the Householder(3) factor of b itself (h2 = b''/b', h3 = b'''/b') in
// float from the float iterate: it enters as nu^2 (h2/2 + h3 nu/6) ~ 1e-12 s,
// so float rounding there is below double rounding of s.  Near the lower tail
// b'' / b' ~ x^2/s^3 is large, but the quartic error constant ~ (x^2/s^2)^3
// times (1e-6)^4 stays far below 1e-16 wherever beta is a normal number.
// Also records 1/b_s at s (ibs) for adjoint_reuse.
__device__ __forceinline__ double step64_final(double x, double bmax, double bb, int region, double s, float sf,
                                               float xf, Last& last) {
  const double inv_s = inv_iterate(s);
  const double h = x * inv_s, t = 0.5 * s, hpt = h + t;
  const double lbs = log_bs<double>(h, t);
  const bool taylor = region != kUpper && le_pos(t, kTaylorT) && le_pos(-x, kTaylorX);
  last.s = s;
  last.za = -fabs(hpt);
  last.zb = h - t;
  last.pair = !taylor;
  double ya = 0.0, yb = 0.0;
  if (!taylor) {
    ya = mills_small(last.za);
    yb = mills_small(last.zb);
  }
  last.ya = ya;
  last.yb = yb;
  double ibs = exp_fp64(-lbs);
  double nu;
  if (finite64(ibs)) {
    const double E1 = bmax * ibs;
    if (region == kUpper) {
      const double gam = gt0(hpt) ? ya + yb : (E1 - ya) + yb;
      nu = gam - bb * ibs;
    } else {
      const double rho = taylor ? rho_taylor<double>(h, t) : (le0(hpt) ? ya - yb : (E1 - ya) - yb);
      nu = bb * ibs - rho;
    }
  } else {
    // b_s below the normal range (subnormal beta, or |ln(F/K)| beyond ~1400): in logarithms
    const double E1 = kSqrt2Pi * exp_fp64(0.5 * hpt * hpt);
    if (region == kUpper) {
      const double gam = (hpt > 0.0) ? ya + yb : (E1 - ya) + yb;
      nu = gam - exp_fp64(log_fp64(bb) - lbs);
    } else {
      const double rho = taylor ? rho_taylor<double>(h, t) : (hpt <= 0.0 ? ya - yb : (E1 - ya) - yb);
      nu = exp_fp64(log_fp64(bb) - lbs) - rho;
    }
    ibs = 0.0; // not usable by the adjoint
  }
  last.lbs = lbs;
  last.ibs = ibs;
  const float fis = 1.0f / sf, fh = xf * fis, ft = 0.5f * sf, fhh = fh * fh;
  const float b2 = (fhh - ft * ft) * fis;
  const float b3 = fmaf(b2, b2, -3.0f * fhh * fis * fis) - 0.25f;
  const float fnu = float(nu);
  const float a = fmaf(b3 * (1.0f / 6.0f), fnu, b2);
  const float corr = -fnu * fmaf(b3 * (1.0f / 6.0f), fnu, 0.5f * b2) / fmaf(fnu, a, 1.0f);
  return s + fma(nu, double(corr), nu);
}

// The FP64 solve of the binned kernels: guess plus `steps` step64 steps; the
// last step's Mills ratios are left in `last` for adjoint_reuse.
template <bool kFastInv = true>
__device__ __forceinline__ double solve64(int region, const Node<double>& nd, double lnbeta, int steps, Last& last) {
  const double lnbetac = (region == kUpper) ? log_fp64(nd.bb) : 0.0;
  const double inv_lnbeta = (region == kLower) ? div_fast(1.0, lnbeta) : 0.0;
  double s = region_guess<double, kFastInv>(region, nd, lnbeta);
  for (int i = 0; i < steps; ++i) s = step64<false>(nd.x, nd.bmax, nd.bb, lnbetac, inv_lnbeta, region, s, last);
  return s;
}

// The mixed solve of the binned kernels: float guess and `steps - 1` float
// steps, then one step64 with float derivative ratios from the float iterate
// (x, bmax, bb and lnbeta in double).
__device__ __forceinline__ double solve_mixed64(int region, const Node<float>& nf, double x, double bmax, double bb,
                                                int steps, Last& last) {
  const float lnbeta_f = (region == kLower) ? logf(nf.bb) : 0.0f; // beta >= 1e-30 on this path
  const float lnbetac_f = (region == kUpper) ? logf(nf.bb) : 0.0f;
  const float inv_lnbeta_f = (region == kLower) ? 1.0f / lnbeta_f : 0.0f;
  float sf = region_guess<float>(region, nf, lnbeta_f);
  for (int i = 1; i < steps; ++i) sf = householder_step<float>(nf.x, nf.bb, lnbetac_f, inv_lnbeta_f, region, sf);
  return step64_final(x, bmax, bb, region, double(sf), sf, nf.x, last);
}

// ln v in float for a positive normal double v of any exponent: v = m 2^e with
// m in [1, 2) read off the bit pattern (its top 23 mantissa bits), so no value
// leaves the float range.
__device__ __forceinline__ float log_of_double_f(double v) {
  const uint64_t b = uint64_t(__double_as_longlong(v));
  const int e = int((b >> 52) & 0x7ff) - 1023;
  const float m = __int_as_float(0x3f800000 | int((b >> 29) & 0x7fffff));
  return fmaf(float(e), 0.693147180559945309f, logf(m));
}

constexpr double kDeepAccept = 1e-5;

// The mixed solve of a deep lower-tail row (beta below the float range,
// |x| >= 0.1).  Far in the lower tail b ~ b_s rho with rho ~ s^3/x^2 (the
// Mills ratios' leading terms), i.e.
//   ln beta ~ -x^2/(2 s^2) - s^2/8 + 3 ln s - 2 ln|x| - ln sqrt(2 pi),
// whose solution for s by one fixed-point pass from s_a = |x|/sqrt(-2 ln beta)
// seeds two float Householder(3) steps on the lower objective (which needs
// only ln beta) and the final FP64 step.  Returns NaN when the FP64 step moves
// the float iterate by more than kDeepAccept (relative): the caller then
// takes the FP64 path.
__device__ __forceinline__ double solve_deep_mixed64(double x, double bmax, double beta, Last& last) {
  const float lnb = log_of_double_f(beta);
  const float ax = float(-x), xf = -ax;
  const float lax = logf(ax);
  const float sa = ax * rsqrtf(-2.0f * lnb);
  const float w = -lnb + 3.0f * logf(sa) - 2.0f * lax - float(kLnSqrt2Pi) - 0.125f * sa * sa;
  float sf = w > 0.0f ? ax * rsqrtf(2.0f * w) : sa;
  const float inv_lnb = 1.0f / lnb;
  sf = householder_step<float>(xf, 0.0f, 0.0f, inv_lnb, kLower, sf);
  sf = householder_step<float>(xf, 0.0f, 0.0f, inv_lnb, kLower, sf);
  if (!(sf > 0.0f && sf < INFINITY)) return __longlong_as_double(0x7ff8000000000000LL);
  const double s = step64_final(x, bmax, beta, kLower, double(sf), sf, xf, last);
  return fabs(s - double(sf)) <= kDeepAccept * s ? s : __longlong_as_double(0x7ff8000000000000LL);
}


// ---------------------------------------------------------------------------
// Adjoint (Eq. implicit_iv / method_vjp) with the low-vega gate (Section 3.3).
// d1 = ln(F/K)/s + s/2, d2 = d1 - s, V = sqrt(FK) sqrt(T) b_s;
// dsigma/dF = -Delta_F/V = -Y(d1)/(F sqrt T) (call), Y(-d1)/(F sqrt T) (put)
// dsigma/dK = -Delta_K/V =  Y(d2)/(K sqrt T) (call), -Y(-d2)/(K sqrt T) (put)
// (F phi(d1) = K phi(d2)); dsigma/dP = 1/V, dsigma/dT = -sigma/(2T).
// ---------------------------------------------------------------------------
struct Grad {
  double dP, dF, dK, dT;
};

__device__ __forceinline__ double signed_log_moneyness(double F, double K) {
  const double l = neg_abs_log_ratio(fmin(F, K), fmax(F, K)); // -|ln(F/K)|
  return F >= K ? -l : l;
}

// Gradient of a row whose sigma is not finite and positive: invalid rows
// (NaN sigma, bad inputs) are NaN in every mode; rows on a bound of the price
// interval (sigma = 0 or +inf) have V = 0 and sit outside every G_tau.
__device__ __forceinline__ Grad degenerate_grad(bool invalid, double g, int mode) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  double v = qnan;
  if (!invalid) {
    if (mode == 1) v = zero64(g) ? 0.0 : qnan;
    if (mode >= 2) v = 0.0;
  }
  Grad out;
  out.dP = out.dF = out.dK = out.dT = v;
  return out;
}

// The gated adjoint of a row with finite sigma > 0, from quantities the
// caller may already hold: s = sigma sqrt(T), xs = ln(F/K) (signed),
// inv_sqT = 1/sqrt(T), rsq = 1/sqrt(F K).  1/F = K rsq^2, 1/K = F rsq^2 and
// V = sqrt(FK) sqrt(T) b_s keep it to one division and one exp besides Y.
__device__ __forceinline__ Grad adjoint_core(double F, double K, int flag, double sigma, double s, double xs,
                                             double inv_sqT, double rsq, double g, double tau, int mode) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  Grad out;
  const double h = xs / s, t = 0.5 * s;
  const double rsq2 = rsq * rsq;
  const double V = exp(log_bs<double>(h, t)) * (F * K * rsq) / inv_sqT;
  const double d1 = h + t, d2 = h - t;
  // call: jF = -Y(d1)/(F sqrt T), jK = Y(d2)/(K sqrt T); put: the same of -d1, -d2 with signs flipped
  const double sg = flag > 0 ? 1.0 : -1.0;
  const double jF = -sg * mills_y<double>(sg * d1) * (K * rsq2) * inv_sqT;
  const double jK = sg * mills_y<double>(sg * d2) * (F * rsq2) * inv_sqT;
  const double jT = -0.5 * sigma * inv_sqT * inv_sqT;
  const bool in_g = fabs(V) > tau;
  if (mode == 0 || (mode <= 2 && in_g)) {
    out.dP = g / V;
    out.dF = g * jF;
    out.dK = g * jK;
    out.dT = g * jT;
    return out;
  }
  if (mode == 1) {
    const double v = (g == 0.0) ? 0.0 : qnan;
    out.dP = out.dF = out.dK = out.dT = v;
    return out;
  }
  if (mode == 2) {
    out.dP = out.dF = out.dK = out.dT = 0.0;
    return out;
  }
  // smooth gate w = V^2/(V^2 + tau^2) on every row; w/V = V/(V^2 + tau^2)
  double w, wP;
  if (V > tau) {
    const double inv_V = 1.0 / V;
    const double r = tau * inv_V;
    w = 1.0 / fma(r, r, 1.0);
    wP = w * inv_V;
  } else {
    const double inv_tau = 1.0 / tau;
    const double r = V * inv_tau;
    const double den = 1.0 / fma(r, r, 1.0);
    w = r * r * den;
    wP = r * inv_tau * den;
  }
  out.dP = g * wP;
  out.dF = g * jF * w;
  out.dK = g * jK * w;
  out.dT = g * jT * w;
  return out;
}

// Y(z0 + d) to second order from Y(z0): Y' = 1 + zY, Y'' = z + (1 + z^2) Y
// = z Y' + Y.  |d| <~ 1e-5 |z0| at the final iterate of every solve, so the
// third-order term (Y''' d^3 / 6, relative ~ d^3 / |z|^3 for z < 0) is below
// 1e-15.
__device__ __forceinline__ double mills_shift(double y0, double z0, double d) {
  const double y1 = fma(z0, y0, 1.0);
  const double y2 = fma(z0, y1, y0);
  return fma(fma(0.5 * y2, d, y1), d, y0);
}

// The gated adjoint of a solved row (as adjoint_core) at its final s, with the
// Mills ratios carried from the last Householder evaluation (`last`) instead
// of evaluated anew.  x = -|ln(F/K)|, bmax = e^{x/2}.  With h = x/s, t = s/2,
// E1 = b_max / b_s and E2 = 1 / (b_max b_s) (1/phi(h + t) and 1/phi(h - t)):
//   Y(h + t), Y(-h - t): one is ya, the other E1 - ya
//   Y(h - t) = yb,  Y(t - h) = E2 - yb
// and the four quote types need (theta = flag):
//   F <= K: d1 = h + t, d2 = h - t;  F > K: d1 = t - h, d2 = -(h + t);
//   dsigma/dF uses Y(theta d1), dsigma/dK uses Y(theta d2).
// 1/V = (1/b_s) rsq / sqrt(T) needs no division.  kUnitG: the upstream gradient is 1 on every
// row (no gbar), so the products by g are left out (x * 1 = x for every double, NaN included).
template <bool kUnitG = false>
__device__ __forceinline__ Grad adjoint_reuse(double F, double K, int flag, double sigma, double s, double x,
                                              double bmax, double inv_sqT, double rsq, double g, double tau, int mode,
                                              const Last& last) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  const double inv_s = inv_iterate(s);
  const double h = x * inv_s, t = 0.5 * s, hpt = h + t;
  const double za = -fabs(hpt), zb = h - t;
  // the shift is used while the final step was small: |s - s_last| < 1e-5 s bounds the argument
  // moves by 1e-5 (|z| + s), so the neglected third-order term stays below ~1e-11 relative
  const bool near = last.pair && abs_lt(s - last.s, 1e-5 * s);
  const double ya = near ? mills_shift(last.ya, last.za, za - last.za) : mills_small(za);
  const double yb = near ? mills_shift(last.yb, last.zb, zb - last.zb) : mills_small(zb);
  const double lbs = log_bs<double>(h, t);
  double ibs;
  if (__double_as_longlong(last.ibs) > 0 && abs_lt(lbs - last.lbs, 1e-3)) {
    // 1/b_s from the last step's: exp(-d) to third order, d = lbs - last.lbs (|d| < 1e-3: d^4/24 < 5e-14)
    const double d = lbs - last.lbs;
    ibs = last.ibs * fma(fma(fma(d, -1.0 / 6.0, 0.5), d, -1.0), d, 1.0);
  } else {
    ibs = exp_fp64(-lbs);
  }
  // 1/b_max = max(F, K) rsq (b_max = min(F, K) rsq, as the caller formed it)
  const double inv_bmax = (gt_pos(F, K) ? F : K) * rsq;
  double E1 = bmax * ibs, E2 = ibs * inv_bmax;
  if (!finite64(ibs)) {
    // b_s underflows (|ln(F/K)| beyond ~1400): the reflections from their own exponents
    E1 = kSqrt2Pi * exp_fp64(0.5 * hpt * hpt);
    E2 = kSqrt2Pi * exp_fp64(0.5 * zb * zb);
  }
  const bool hneg = le0(hpt);
  const double y_hpt = hneg ? ya : E1 - ya;  // Y(h + t)
  const double y_mhpt = hneg ? E1 - ya : ya; // Y(-h - t)
  const bool call = flag > 0, fle = le_pos(F, K);
  const bool itm = call ? !fle : fle;
  const double y_tmh = itm ? E2 - yb : 0.0; // Y(t - h), in-the-money quotes only
  const double u1 = fle ? (call ? y_hpt : y_mhpt) : (call ? y_tmh : yb);  // Y(theta d1)
  const double u2 = fle ? (call ? yb : y_tmh) : (call ? y_mhpt : y_hpt);  // Y(theta d2)
  // with c = rsq / sqrt(T): 1/V = c / b_s, 1/(F sqrt T) = (K rsq) c, 1/(K sqrt T) = (F rsq) c,
  // where K rsq and F rsq are b_max and 1/b_max in some order (the same products); the signs go
  // on the Mills ratios (a select, not a multiplication)
  const double c = rsq * inv_sqT;
  const double jP = ibs * c; // 1/V, V = b_s sqrt(F K) sqrt(T)
  const double jF = (call ? -u1 : u1) * ((fle ? inv_bmax : bmax) * c);
  const double jK = (call ? u2 : -u2) * ((fle ? bmax : inv_bmax) * c);
  const double jT = (-0.5 * sigma) * (inv_sqT * inv_sqT);
  Grad out;
  const bool in_g = cmp_lt(tau * jP, 1.0); // V > tau
  if (mode == 0 || (mode <= 2 && in_g)) {
    out.dP = kUnitG ? jP : g * jP;
    out.dF = kUnitG ? jF : g * jF;
    out.dK = kUnitG ? jK : g * jK;
    out.dT = kUnitG ? jT : g * jT;
    return out;
  }
  if (mode == 1) {
    const double v = (g == 0.0) ? 0.0 : qnan;
    out.dP = out.dF = out.dK = out.dT = v;
    return out;
  }
  if (mode == 2) {
    out.dP = out.dF = out.dK = out.dT = 0.0;
    return out;
  }
  // smooth gate w = V^2/(V^2 + tau^2); w/V = V/(V^2 + tau^2)
  double w, wP;
  if (in_g) {
    const double r = tau * jP;
    w = 1.0 / fma(r, r, 1.0);
    wP = w * jP;
  } else {
    const double inv_tau = 1.0 / tau;
    const double r = 1.0 / (tau * jP); // V / tau
    const double den = 1.0 / fma(r, r, 1.0);
    w = r * r * den;
    wP = r * inv_tau * den;
  }
  out.dP = kUnitG ? wP : g * wP;
  out.dF = (kUnitG ? jF : g * jF) * w;
  out.dK = (kUnitG ? jK : g * jK) * w;
  out.dT = (kUnitG ? jT : g * jT) * w;
  return out;
}

__device__ __forceinline__ Grad gated_adjoint(double F, double K, double T, int flag, double sigma, double g,
                                              double tau, int mode) {
  if (bad_inputs(F, K, T, flag) || !(sigma >= 0.0) || isnan(g)) return degenerate_grad(true, g, mode);
  if (sigma == 0.0 || sigma == INFINITY) return degenerate_grad(false, g, mode);
  const double xs = signed_log_moneyness(F, K);
  const double inv_sqT = rsqrt(T);
  const double s = sigma / inv_sqT;
  return adjoint_core(F, K, flag, sigma, s, xs, inv_sqT, rsqrt(F * K), g, tau, mode);
}

// ---------------------------------------------------------------------------
// Black-Scholes form on xi = (S, K, tau, r, q) (Eq. app_forward_price,
// Algorithm 1): F = S e^{(r-q) tau}, B = e^{r tau} V, then the Black-76 path.
// er = e^{r tau} and ec = e^{(r-q) tau}; NaN for a non-finite r or q, which
// makes F NaN and the row a bad input.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bs_factors(double tau, double r, double q, double& er, double& ec) {
  if (isfinite(r) && isfinite(q)) {
    er = exp_fp64(r * tau);
    ec = exp_fp64((r - q) * tau);
  } else {
    er = ec = __longlong_as_double(0x7ff8000000000000LL);
  }
}

struct BSGrad {
  double dV, dS, dK, dT, dr, dq;
};

// The xi-gradient from the Black-76 one at F = S ec, B = er V: sigma depends on
// (V, S, r, q) only through B and F, so dV = er dB and dS = ec dF; the rate and
// dividend terms follow from homogeneity (F dF + K dK + B dB = 0):
//   dr = tau (B dB + F dF) = -tau K dK,   dq = -tau F dF,
//   dtau = dT + r B dB + (r - q) F dF = dT - q F dF - r K dK.
// A zero rate or yield adds no term (keeps an infinite Mills ratio from making 0 inf).
__device__ __forceinline__ BSGrad bs_grad(const Grad& d, double F, double K, double tau, double r, double q,
                                          double er, double ec) {
  BSGrad o;
  const double fdF = F * d.dF, kdK = K * d.dK;
  o.dV = d.dP * er;
  o.dS = d.dF * ec;
  o.dK = d.dK;
  o.dr = -tau * kdK;
  o.dq = -tau * fdF;
  o.dT = d.dT - (q != 0.0 ? q * fdF : 0.0) - (r != 0.0 ? r * kdK : 0.0);
  return o;
}

// ---------------------------------------------------------------------------
// Black-76 price with r = 0: intrinsic + sqrt(FK) b(x, s), vega.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void black_price_row(double F, double K, double T, double sigma, int flag, double& P,
                                                double& V) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  if (bad_inputs(F, K, T, flag) || !(sigma >= 0.0)) {
    P = qnan;
    V = qnan;
    return;
  }
  const bool call = flag > 0;
  const double intrinsic = call ? fmax(F - K, 0.0) : fmax(K - F, 0.0);
  double x, bmax, rsq;
  moneyness(F, K, x, bmax, rsq);
  const double sqT = sqrt(T);
  const double rfk = sqrt(F * K);
  if (sigma == 0.0) {
    P = intrinsic;
    V = (x == 0.0) ? rfk * sqT * kInvSqrt2Pi : 0.0;
    return;
  }
  if (sigma == INFINITY) {
    P = call ? F : K;
    V = 0.0;
    return;
  }
  const double s = sigma * sqT;
  const double h = x / s, t = 0.5 * s;
  const double bs = exp(log_bs<double>(h, t));
  double b;
  if (s > 2.0 && s * s > -2.0 * x) {
    b = bmax - bs * gamma_of<double>(h, t); // above the inflection and s > 2: b >~ 0.4 b_max
  } else {
    b = bs * rho_of<double>(x, h, t);
  }
  P = intrinsic + rfk * b;
  V = rfk * sqT * bs;
}

// ---------------------------------------------------------------------------
// VJP of the Black-76 price (r = 0) in (sigma, F, K, T).
// Phi(z) = erfc(-z/sqrt 2)/2 has no cancellation on either tail.
// ---------------------------------------------------------------------------
struct PriceGrad {
  double dsigma, dF, dK, dT;
};

__device__ __forceinline__ PriceGrad black_price_vjp_row(double F, double K, double T, double sigma, int flag,
                                                         double g) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  PriceGrad o;
  if (bad_inputs(F, K, T, flag) || !(sigma >= 0.0) || isnan(g)) {
    o.dsigma = o.dF = o.dK = o.dT = qnan;
    return o;
  }
  const double sg = flag > 0 ? 1.0 : -1.0;
  const double xs = signed_log_moneyness(F, K);
  if (sigma == 0.0 || sigma == INFINITY) {
    // one-sided limits: the price is the intrinsic value (sigma = 0) or the upper bound
    const bool itm = sg * xs > 0.0;
    const double half = (xs == 0.0) ? 0.5 : 0.0;
    double dPdF, dPdK;
    if (sigma == 0.0) {
      dPdF = sg * (itm ? 1.0 : half);
      dPdK = -sg * (itm ? 1.0 : half);
    } else {
      dPdF = flag > 0 ? 1.0 : 0.0;
      dPdK = flag > 0 ? 0.0 : 1.0;
    }
    const double V0 = (sigma == 0.0 && xs == 0.0) ? sqrt(F * K) * sqrt(T) * kInvSqrt2Pi : 0.0;
    o.dsigma = g * V0;
    o.dF = g * dPdF;
    o.dK = g * dPdK;
    o.dT = 0.0;
    return o;
  }
  const double sqT = sqrt(T);
  const double s = sigma * sqT;
  const double h = xs / s, t = 0.5 * s;
  const double V = sqrt(F * K) * sqT * exp(log_bs<double>(h, t));
  const double d1 = h + t, d2 = h - t;
  // call: dP/dF = Phi(d1), dP/dK = -Phi(d2); put: dP/dF = -Phi(-d1), dP/dK = Phi(-d2)
  const double dPdF = sg * 0.5 * erfc(-sg * d1 * kInvSqrt2);
  const double dPdK = -sg * 0.5 * erfc(-sg * d2 * kInvSqrt2);
  o.dsigma = g * V;
  o.dF = g * dPdF;
  o.dK = g * dPdK;
  o.dT = g * V * sigma / (2.0 * T);
  return o;
}

}  // namespace pivot

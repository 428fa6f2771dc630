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

// Y(z) = Phi(z)/phi(z).  Kept out of line: it is called from many sites and
// one shared copy keeps the kernels' instruction footprint small.
__device__ __noinline__ double mills_y(double z) { return kSqrtPiOver2 * erfcx(-z * kInvSqrt2); }

// ln b_s(x, s) = -(h^2 + t^2)/2 - ln sqrt(2 pi)
__device__ __forceinline__ double log_bs(double h, double t) {
  return fma(-0.5, fma(h, h, t * t), -kLnSqrt2Pi);
}

__device__ __forceinline__ double rho_taylor(double h, double t) {
  double c_prev = mills_y(h);           // c_0
  double c_cur = fma(h, c_prev, 1.0);   // c_1
  const double t2 = t * t;
  double acc = c_cur, tp = 1.0;
  // c_{n+1} = (h c_n + c_{n-1}) / (n + 1), two steps per odd term
#pragma unroll
  for (int m = 1; m < 9; ++m) {
    const int n = 2 * m - 1;
    double c_next = fma(h, c_cur, c_prev) * (1.0 / double(n + 1));
    c_prev = c_cur;
    c_cur = c_next;
    c_next = fma(h, c_cur, c_prev) * (1.0 / double(n + 2));
    c_prev = c_cur;
    c_cur = c_next;
    tp *= t2;
    acc = fma(c_cur, tp, acc);
  }
  return 2.0 * t * acc;
}

// rho = b / b_s for x <= 0, s > 0
__device__ __forceinline__ double rho_of(double x, double h, double t) {
  if (t <= kTaylorT && x >= -kTaylorX) return rho_taylor(h, t);
  return mills_y(h + t) - mills_y(h - t);
}

// gamma = (b_max - b) / b_s
__device__ __forceinline__ double gamma_of(double h, double t) { return mills_y(-h - t) + mills_y(h - t); }

// Delbourgo-Gregory rational cubic Hermite interpolant on [z0, z1] through
// (z0, y0), (z1, y1) with end slopes d0, d1 and shape parameter r (r = 3 is
// the cubic Hermite; larger r pulls towards the chord).
__device__ __forceinline__ double rational_cubic(double z, double z0, double z1, double y0, double y1,
                                                 double d0, double d1, double r) {
  const double D = z1 - z0;
  const double tau = (z - z0) / D;
  const double om = 1.0 - tau;
  const double num = y0 * om * om * om + (r * y0 + D * d0) * tau * om * om + (r * y1 - D * d1) * tau * tau * om +
                     y1 * tau * tau * tau;
  const double den = fma((r - 3.0) * tau, om, 1.0);
  return num / den;
}

// Shape parameter with zero second derivative at the right end (z1) and at
// least the monotonicity bound (d0 + d1)/m of the Delbourgo-Gregory form.
__device__ __forceinline__ double shape_zero_curv_right(double D, double y0, double y1, double d0, double d1) {
  const double r = D * (d1 - d0) / (D * d1 + y0 - y1);
  const double rmono = (d0 + d1) * D / (y1 - y0);
  return fmax(r, rmono);
}
// ... zero second derivative at the left end (z0)
__device__ __forceinline__ double shape_zero_curv_left(double D, double y0, double y1, double d0, double d1) {
  const double r = D * (d0 - d1) / (D * d0 + y0 - y1);
  const double rmono = (d0 + d1) * D / (y1 - y0);
  return fmax(r, rmono);
}
__device__ __forceinline__ double shape_monotone(double D, double y0, double y1, double d0, double d1) {
  return fmax(3.0, (d0 + d1) * D / (y1 - y0));
}

// ---------------------------------------------------------------------------
// Row preparation (Algorithm 1 forward normalisation with r = 0; appendix
// stages 1-2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool bad_inputs(double F, double K, double T, int flag) {
  // also rejects NaN and +-inf
  return !(F > 0.0 && F < INFINITY) || !(K > 0.0 && K < INFINITY) || !(T > 0.0 && T < INFINITY) ||
         (flag != 1 && flag != -1);
}

// P - F + K (call) or P - K + F (put) with two error-free TwoSums, one rounding
__device__ __forceinline__ double time_value_itm(double P, double a, double b) {
  // P - a + b
  double s1 = P - a, bb = s1 - P;
  double e1 = (P - (s1 - bb)) + (-a - bb);
  double s2 = s1 + b;
  double bb2 = s2 - s1;
  double e2 = (s1 - (s2 - bb2)) + (b - bb2);
  return s2 + (e1 + e2);
}

// -|ln(F/K)| from mn = min(F, K), mx = max(F, K), branch-free and accurate
// near the money: r = mn/mx is correctly rounded, so its residual
// c = (mn - r mx)/mn is exact to first order (one fma) and
// ln(mn/mx) = ln r + ln(1 + c) = ln r + c + O(c^2), |c| <= 2^-53.
__device__ __forceinline__ double neg_abs_log_ratio(double mn, double mx, double* ratio = nullptr) {
  const double r = mn / mx;
  const double c = fma(-r, mx, mn) / mn;
  if (ratio) *ratio = r;
  return log(r) + c;
}

// x = -|ln(F/K)|, b_max = e^{x/2} = sqrt(min/max)
__device__ __forceinline__ void moneyness(double F, double K, double& x, double& bmax) {
  double r;
  x = neg_abs_log_ratio(fmin(F, K), fmax(F, K), &r);
  bmax = sqrt(r);
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
  if (bad_inputs(F, K, T, flag) || !(fabs(P) < INFINITY)) {
    q.status = 3;
    q.sigma = qnan;
    return q;
  }
  const bool call = flag > 0;
  const bool itm = call ? (F > K) : (K > F);
  q.tv = itm ? (call ? time_value_itm(P, F, K) : time_value_itm(P, K, F)) : P;
  q.cv = (call ? F : K) - P;
  if (q.tv < 0.0) { q.status = 1; q.sigma = qnan; }
  else if (q.cv < 0.0) { q.status = 2; q.sigma = qnan; }
  else if (q.tv == 0.0) { q.status = 4; q.sigma = 0.0; }
  else if (q.cv == 0.0) { q.status = 5; q.sigma = INFINITY; }
  return q;
}

// ln beta for a solved row; beta near or below the subnormal range takes it
// from ln tv so that it keeps its relative accuracy
__device__ __forceinline__ double log_beta(double beta, double F, double K, double T, double P, int flag) {
  if (beta > 1e-290) return log(beta);
  const Quote q = classify_quote(F, K, T, P, flag);
  return log(q.tv) + log(rsqrt(F * K));
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
struct Node {
  double x;    // -|ln(F/K)|
  double bmax; // e^{x/2}
  double e;    // erfcx(sqrt|x|)
  double bn;   // b_l (lower side) or b_max - b_u (upper side)
  double bsn;  // b_s at that node
  double bb;   // beta, or beta_c = b_max - beta in the upper region
};

__device__ __forceinline__ int classify(double x, double bmax, double beta, double betac, Node& nd) {
  const double ax = -x;
  const double sc = sqrt(2.0 * ax);
  const double e = erfcx(sc * kInvSqrt2);
  const double bc = 0.5 * bmax * (1.0 - e);
  const bool low = beta <= bc;
  const double sl = sc - kSqrtPiOver2 * (1.0 - e);
  const double su = sc + kSqrtPiOver2 * (1.0 + e);
  const bool has_l = sl > 0.0;
  const double sn = low ? (has_l ? sl : 1.0) : su;
  const double h = x / sn, t = 0.5 * sn;
  const double y1 = mills_y(low ? h + t : -h - t);
  const double y2 = mills_y(h - t);
  const double bs = exp(log_bs(h, t));
  const double val = bs * (low ? y1 - y2 : y1 + y2);
  nd.x = x;
  nd.bmax = bmax;
  nd.e = e;
  nd.bn = (low && !has_l) ? 0.0 : val;
  nd.bsn = bs;
  int region;
  if (low) region = (beta < nd.bn) ? kLower : kMidLow;
  else region = (beta <= bmax - val) ? kMidHigh : kUpper;
  nd.bb = (region == kUpper) ? betac : beta;
  return region;
}

// Rational initial guess s^(0) of the row's region from its node.
// lnbeta is ln beta (lower region only).
__device__ __forceinline__ double region_guess(int region, const Node& nd, double lnbeta) {
  const double x = nd.x, ax = -x;
  const double sc = sqrt(2.0 * ax);
  const double e = nd.e;
  const double dc = kSqrt2Pi / nd.bmax; // ds/db at s_c
  switch (region) {
    case kLower: {
      // lower tail: b ~ kappa Phi(-|x|/(sqrt3 s))^3 as s -> 0, kappa = 2 pi |x| / (3 sqrt 3).
      // Interpolate G = Phi(-|x|/(sqrt3 s)) against u = (beta/kappa)^(1/3) on [0, u_l]
      // (G(0) = 0, G'(0) = 1, G(u_l), G'(u_l) exact), then invert G for s.
      const double sl = sc - kSqrtPiOver2 * (1.0 - e);
      const double bl = nd.bn, bsl = nd.bsn, beta = nd.bb;
      const double kap = kTwoPiOver3Sqrt3 * ax;
      const double u = (beta > 1e-280) ? cbrt(beta / kap) : exp((lnbeta - log(kap)) * (1.0 / 3.0));
      const double ul = cbrt(bl / kap);
      const double al = ax * kInvSqrt3 / sl;
      const double Gl = normcdf(-al);
      const double dGl = 3.0 * bl * (kInvSqrt2Pi * exp(-0.5 * al * al)) * al / (sl * ul * bsl);
      const double r = shape_monotone(ul, 0.0, Gl, 1.0, dGl);
      const double G = fmin(rational_cubic(u, 0.0, ul, 0.0, Gl, 1.0, dGl, r), 0.5);
      return ax * kInvSqrt3 / (-normcdfinv(G));
    }
    case kMidLow: {
      // rational cubic in b on [b_l, b_c], zero curvature of s(b) at the inflection b_c
      const double sl = sc - kSqrtPiOver2 * (1.0 - e);
      const double bc = 0.5 * nd.bmax * (1.0 - e);
      const double bl = nd.bn;
      const double d0 = (bl > 0.0) ? 1.0 / nd.bsn : dc;
      const double s0 = (bl > 0.0) ? sl : 0.0;
      const double D = bc - bl;
      const double r = shape_zero_curv_right(D, s0, sc, d0, dc);
      return rational_cubic(nd.bb, bl, bc, s0, sc, d0, dc, r);
    }
    case kMidHigh: {
      // rational cubic in b on [b_c, b_u], zero curvature of s(b) at b_c
      const double su = sc + kSqrtPiOver2 * (1.0 + e);
      const double bc = 0.5 * nd.bmax * (1.0 - e);
      const double bu = nd.bmax - nd.bn;
      const double d1 = 1.0 / nd.bsn;
      const double D = bu - bc;
      const double r = shape_zero_curv_left(D, sc, su, dc, d1);
      return rational_cubic(nd.bb, bc, bu, sc, su, dc, d1, r);
    }
    default: {
      // upper tail: b_max - b ~ 2 Phi(-s/2) as s -> inf.  Interpolate
      // v = Phi(-s/2) against u = (b_max - beta)/2 on [0, u_u], v'(0) = 1.
      const double su = sc + kSqrtPiOver2 * (1.0 + e);
      const double uu = 0.5 * nd.bn;
      const double vu = normcdf(-0.5 * su);
      const double dvu = (kInvSqrt2Pi * exp(-0.125 * su * su)) / nd.bsn;
      const double r = shape_monotone(uu, 0.0, vu, 1.0, dvu);
      const double v = fmin(rational_cubic(0.5 * nd.bb, 0.0, uu, 0.0, vu, 1.0, dvu, r), 0.5);
      return -2.0 * normcdfinv(v);
    }
  }
}

// ---------------------------------------------------------------------------
// One Householder(3) step (appendix stage 5) on the region's objective
//   lower:  f = 1/ln b(s) - 1/ln beta
//   middle: f = b(s) - beta
//   upper:  f = ln(b_max - beta) - ln(b_max - b(s))
// with b''/b' = x^2/s^3 - s/4 and b'''/b' = (b''/b')^2 - 3x^2/s^4 - 1/4:
//   s <- s + nu (1 + h2 nu / 2) / (1 + nu (h2 + h3 nu / 6)),
//   nu = -f/f', h2 = f''/f', h3 = f'''/f'.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double householder_step(double x, double beta, double lnbetac, double inv_lnbeta,
                                                   int region, double s) {
  const double inv_s = 1.0 / s;
  const double h = x * inv_s, t = 0.5 * s;
  const double hh = h * h;
  const double b2 = (hh - t * t) * inv_s;                    // b''/b'
  const double b3 = fma(b2, b2, -3.0 * hh * inv_s * inv_s) - 0.25; // b'''/b'
  double nu, h2, h3;
  if (region == kLower) {
    const double rho = rho_of(x, h, t);
    const double L = log_bs(h, t) + log(rho); // ln b
    const double q = 1.0 / rho;               // (ln b)' = b'/b
    const double iL = 1.0 / L;
    // nu = -(1/L - 1/Lb) L^2 / q = rho L (Lb - L) / Lb
    nu = rho * L * (1.0 - L * inv_lnbeta);
    h2 = b2 - q * fma(2.0, iL, 1.0);
    h3 = b3 - 3.0 * b2 * q + 2.0 * q * q - 6.0 * q * (b2 - q) * iL + 6.0 * q * q * iL * iL;
  } else if (region == kUpper) {
    const double gam = gamma_of(h, t);
    const double pg = 1.0 / gam; // b'/(b_max - b)
    const double f = lnbetac - log_bs(h, t) - log(gam);
    nu = -f * gam;
    h2 = b2 + pg;
    h3 = b3 + 3.0 * pg * b2 + 2.0 * pg * pg;
  } else {
    const double rho = rho_of(x, h, t);
    const double bs = exp(log_bs(h, t));
    nu = beta / bs - rho; // (beta - b)/b'
    h2 = b2;
    h3 = b3;
  }
  const double num = nu * fma(0.5 * h2, nu, 1.0);
  const double den = fma(nu, fma(h3 * (1.0 / 6.0), nu, h2), 1.0);
  return s + num / den;
}

// Guess plus `steps` Householder(3) steps for a classified row; returns s.
__device__ __forceinline__ double solve_region(int region, const Node& nd, double lnbeta, int steps) {
  const double lnbetac = (region == kUpper) ? log(nd.bb) : 0.0;
  const double inv_lnbeta = (region == kLower) ? 1.0 / lnbeta : 0.0;
  double s = region_guess(region, nd, lnbeta);
  for (int i = 0; i < steps; ++i) s = householder_step(nd.x, nd.bb, lnbetac, inv_lnbeta, region, s);
  return s;
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

__device__ __forceinline__ Grad gated_adjoint(double F, double K, double T, int flag, double sigma, double g,
                                              double tau, int mode) {
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  Grad out;
  if (bad_inputs(F, K, T, flag) || !(sigma >= 0.0) || isnan(g)) {
    out.dP = out.dF = out.dK = out.dT = qnan;
    return out;
  }
  if (sigma == 0.0 || sigma == INFINITY) {
    // on a bound of the price interval: V = 0, outside every G_tau
    double v = qnan;
    if (mode == 1) v = (g == 0.0) ? 0.0 : qnan;
    if (mode >= 2) v = 0.0;
    out.dP = out.dF = out.dK = out.dT = v;
    return out;
  }
  const double xs = signed_log_moneyness(F, K);
  const double sqT = sqrt(T);
  const double s = sigma * sqT;
  const double inv_s = 1.0 / s;
  const double h = xs * inv_s, t = 0.5 * s;
  const double V = sqrt(F * K) * sqT * exp(log_bs(h, t));
  const double d1 = h + t, d2 = h - t;
  // call: jF = -Y(d1)/(F sqrt T), jK = Y(d2)/(K sqrt T); put: the same of -d1, -d2 with signs flipped
  const double sg = flag > 0 ? 1.0 : -1.0;
  const double jF = -sg * mills_y(sg * d1) / (F * sqT);
  const double jK = sg * mills_y(sg * d2) / (K * sqT);
  const double jT = -sigma / (2.0 * T);
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
    const double r = tau / V;
    w = 1.0 / fma(r, r, 1.0);
    wP = w / V;
  } else {
    const double r = V / tau;
    const double den = 1.0 / fma(r, r, 1.0);
    w = r * r * den;
    wP = (r / tau) * den;
  }
  out.dP = g * wP;
  out.dF = g * jF * w;
  out.dK = g * jK * w;
  out.dT = g * jT * w;
  return out;
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
  double x, bmax;
  moneyness(F, K, x, bmax);
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
  const double bs = exp(log_bs(h, t));
  double b;
  if (s > 2.0 && s * s > -2.0 * x) {
    b = bmax - bs * gamma_of(h, t); // above the inflection and s > 2: b >~ 0.4 b_max
  } else {
    b = bs * rho_of(x, h, t);
  }
  P = intrinsic + rfk * b;
  V = rfk * sqT * bs;
}

}  // namespace pivot

/*
 * pivot_oracle.c -- plain, slow, obviously correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
 * CPU legs are the only callers.  Nothing here is shared with the CUDA path.
 *
 * It computes definitions, not the LBR algorithm:
 *
 *  - Normalised Black function (Section 2, Eq. app_normalized_black), written
 *    in x = ln(F/K) <= 0 (the out-of-the-money call form that put-call parity
 *    reduces every row to, Appendix "five-stage LBR construction", stage 1):
 *        b(x,s) = e^{x/2} Phi(x/s + s/2) - e^{-x/2} Phi(x/s - s/2).
 *    Its s-derivative is the normalised vega
 *        b_s(x,s) = exp(-x^2/(2 s^2) - s^2/8) / sqrt(2 pi)
 *    (Appendix "Vega and the option Greeks", Eq. app_vega_closed_form divided
 *    by sqrt(F K T)).  Since b(x,0+) = 0 and b(x,inf) = b_max = e^{x/2}
 *    (Eq. app_b_bounds), the fundamental theorem of calculus gives
 *        b(x,s)         = int_0^s   b_s(x,u) du,
 *        b_max - b(x,s) = int_s^inf b_s(x,u) du,
 *    both integrals of a positive function, so neither cancels.  They are
 *    evaluated by adaptive Gauss-Legendre quadrature after the substitutions
 *    u = s v and u = s / v, scaled by b_s(x,s) so that nothing underflows:
 *        rho(x,s)   = b / b_s       = s int_0^1 exp((1-v^2)(B - A/v^2)) dv,
 *        gamma(x,s) = (b_max-b)/b_s = s int_0^1 exp((1-v^2)(A - B/v^2)) / v^2 dv,
 *    with A = x^2/(2 s^2), B = s^2/8 (each split at v = 1/2, the upper half
 *    integrated in w = 1 - v).  rho is used while B is moderate and gamma
 *    while A is; outside those regimes the other one gives b = b_max - ...
 *
 *  - Implied volatility (Section 2, Eq. iv_inverse_problem): the unique s > 0
 *    with b(x,s) = beta, beta = (P - intrinsic)/sqrt(F K) (Algorithm 1, forward
 *    normalisation with r = 0), found by safeguarded Newton / bisection on
 *    ln b(s) - ln beta (or ln beta_c - ln(b_max - b(s)) when beta is above
 *    b_max/2, beta_c = (U - P)/sqrt(F K)), to about 2 ulp; sigma = s/sqrt(T).
 *    Invalid rows are NaN (Section 3.1; Algorithm 1, forward masking).
 *
 *  - Black-76 price with r = 0 (Eq. app_black76): intrinsic + sqrt(F K) b.
 *
 *  - Implicit-function-theorem adjoint (Eq. implicit_iv, Eq. method_vjp):
 *    dsigma/dP = 1/V, dsigma/dF = -Delta_F/V, dsigma/dK = -Delta_K/V,
 *    dsigma/dT = -sigma/(2T), with the ratios Delta/V written through
 *    M(z) = Phi(z)/phi(z) (F phi(d1) = K phi(d2)), and the low-vega gate of
 *    Section 3.3 (Eq. wellcond_set, Eq. smooth_gate).
 */
#include "pivot_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846264338327950288;
static const double LN_SQRT_2PI = 0.918938533204672741780329736405617640;

/* ---------------------------------------------------------------------------
 * Gauss-Legendre rule on [-1, 1], nodes from Newton's method on the Legendre
 * recurrence (k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}).
 * ------------------------------------------------------------------------- */
#define NGL 20
static double gl_node[NGL], gl_weight[NGL];

static void legendre(double z, double* pn, double* dpn) {
  double p0 = 1.0, p1 = z;
  for (int k = 2; k <= NGL; ++k) {
    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *dpn = NGL * (z * p1 - p0) / (z * z - 1.0);
}

__attribute__((constructor)) static void gl_init(void) {
  for (int i = 0; i < NGL; ++i) {
    double z = cos(PI * (i + 0.75) / (NGL + 0.5)), p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) <= 1e-17) break;
    }
    legendre(z, &p, &dp);
    gl_node[i] = z;
    gl_weight[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* Neumaier compensated summation */
typedef struct { double s, c; } csum;
static void csum_add(csum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double csum_get(const csum* a) { return a->s + a->c; }

typedef double (*integrand_fn)(double v, const double* par);

static double gl_panel(integrand_fn f, const double* par, double a, double b) {
  double m = 0.5 * (a + b), h = 0.5 * (b - a);
  csum acc = {0.0, 0.0};
  for (int i = 0; i < NGL; ++i) csum_add(&acc, gl_weight[i] * f(m + h * gl_node[i], par));
  return h * csum_get(&acc);
}

/* Recursive bisection.  A panel is accepted once the 20-point rule on the
 * whole panel agrees with the sum over its halves to an absolute tolerance or
 * to 1e-12 relative: the composite rule on the halves is then many orders of
 * magnitude more accurate still (Gauss-Legendre converges geometrically in the
 * panel width for analytic integrands), while the test stays above the
 * rounding noise of the integrand values.  A global evaluation budget keeps
 * every call finite. */
typedef struct { double tol; long budget; csum acc; } adapt_t;

static void gl_adapt(integrand_fn f, const double* par, double a, double b, double whole,
                     int depth, adapt_t* st) {
  double m = 0.5 * (a + b);
  double l = gl_panel(f, par, a, m), r = gl_panel(f, par, m, b);
  st->budget -= 2 * NGL;
  double err = fabs(l + r - whole);
  if (err <= st->tol || err <= 1e-12 * fabs(l + r) || depth >= 40 || st->budget <= 0 ||
      !(m > a && m < b)) {
    csum_add(&st->acc, l);
    csum_add(&st->acc, r);
    return;
  }
  gl_adapt(f, par, a, m, l, depth + 1, st);
  gl_adapt(f, par, m, b, r, depth + 1, st);
}

/* integrate over consecutive panels [brk[i], brk[i+1]] */
static double gl_integrate(integrand_fn f, const double* par, const double* brk, int nbrk) {
  double whole[160];
  double est = 0.0;
  for (int i = 0; i + 1 < nbrk; ++i) {
    whole[i] = gl_panel(f, par, brk[i], brk[i + 1]);
    est += fabs(whole[i]);
  }
  adapt_t st = {1e-18 * est, 400000, {0.0, 0.0}};
  for (int i = 0; i + 1 < nbrk; ++i) gl_adapt(f, par, brk[i], brk[i + 1], whole[i], 0, &st);
  return csum_get(&st.acc);
}

/* Breakpoints on [0, 1/2], halving towards 0 until the panel next to 0 is
 * narrower than 1e-3 * feature. */
static int breaks_towards_zero(double feature, double* brk) {
  double w[160];
  int n = 0;
  double h = 0.25;
  while (h > 1e-3 * feature && n < 140) {
    w[n++] = h;
    h *= 0.5;
  }
  int m = 0;
  brk[m++] = 0.0;
  for (int i = n - 1; i >= 0; --i) brk[m++] = w[i];
  brk[m++] = 0.5;
  return m;
}

/* Integrands of rho/s and gamma/s, each split at v = 1/2: the part v in
 * [0, 1/2] is integrated in v, the part v in [1/2, 1] in w = 1 - v, so that
 * 1 - v^2 = w (2 - w) is formed without cancellation.  Features: rho's
 * integrand steps up near v ~ sqrt(A), gamma's peaks near v ~ sqrt(B), and
 * both concentrate near v = 1 on a scale ~ 1/(1 + 2(A + B)). */
static double f_rho_v(double v, const double* par) {
  double A = par[0], B = par[1];
  if (v <= 0.0) return A > 0.0 ? 0.0 : exp(B);
  return exp((1.0 - v) * (1.0 + v) * (B - A / (v * v)));
}
static double f_rho_w(double w, const double* par) {
  double A = par[0], B = par[1], v = 1.0 - w;
  return exp(w * (2.0 - w) * (B - A / (v * v)));
}
static double f_gamma_v(double v, const double* par) {
  double A = par[0], B = par[1];
  if (v <= 0.0) return 0.0;
  double e = (1.0 - v) * (1.0 + v) * (A - B / (v * v));
  if (e < -745.0) return 0.0;
  return exp(e) / (v * v);
}
static double f_gamma_w(double w, const double* par) {
  double A = par[0], B = par[1], v = 1.0 - w;
  return exp(w * (2.0 - w) * (A - B / (v * v))) / (v * v);
}

static double split_integral(integrand_fn fv, integrand_fn fw, double A, double B, double feature_v) {
  double par[2] = {A, B};
  double brk[160];
  int nb = breaks_towards_zero(feature_v, brk);
  double iv = gl_integrate(fv, par, brk, nb);
  nb = breaks_towards_zero(1.0 / (1.0 + 2.0 * (A + B)), brk);
  double iw = gl_integrate(fw, par, brk, nb);
  return iv + iw;
}

/* rho = b/b_s, valid while B = s^2/8 is moderate (the integrand reaches e^B) */
static double rho_of(double x, double s) {
  double h = x / s, A = 0.5 * h * h, B = 0.125 * s * s;
  double feat = A > 0.0 ? fmin(sqrt(A), 1.0) : 1.0;
  return s * split_integral(f_rho_v, f_rho_w, A, B, feat);
}
/* gamma = (b_max - b)/b_s, valid while A = x^2/(2 s^2) is moderate */
static double gamma_of(double x, double s) {
  double h = x / s, A = 0.5 * h * h, B = 0.125 * s * s;
  double feat = fmin(sqrt(B), 1.0);
  return s * split_integral(f_gamma_v, f_gamma_w, A, B, feat);
}
static const double REGIME = 600.0; /* keeps e^A, e^B far from overflow */

/* ln b_s(x,s) = -x^2/(2 s^2) - s^2/8 - ln sqrt(2 pi) */
static double log_bs(double x, double s) {
  double h = x / s;
  return -0.5 * h * h - 0.125 * s * s - LN_SQRT_2PI;
}

double oracle_normalised_black(double x, double s) {
  if (!(x <= 0.0) || !(s >= 0.0)) return NAN;
  if (s == 0.0) return 0.0;
  if (isinf(s)) return exp(0.5 * x);
  if (0.125 * s * s <= REGIME) return exp(log_bs(x, s)) * rho_of(x, s);
  return exp(0.5 * x) - exp(log_bs(x, s)) * gamma_of(x, s);
}
double oracle_normalised_black_complement(double x, double s) {
  if (!(x <= 0.0) || !(s >= 0.0)) return NAN;
  if (s == 0.0) return exp(0.5 * x);
  if (isinf(s)) return 0.0;
  double h = x / s;
  if (0.5 * h * h <= REGIME) return exp(log_bs(x, s)) * gamma_of(x, s);
  return exp(0.5 * x) - exp(log_bs(x, s)) * rho_of(x, s);
}
double oracle_log_normalised_black(double x, double s) {
  if (!(x <= 0.0) || !(s >= 0.0)) return NAN;
  if (s == 0.0) return -INFINITY;
  if (isinf(s)) return 0.5 * x;
  if (0.125 * s * s <= REGIME) return log_bs(x, s) + log(rho_of(x, s));
  return log(oracle_normalised_black(x, s));
}

/* ---------------------------------------------------------------------------
 * Mills-type ratio M(z) = Phi(z)/phi(z).
 * z <= 0: M(z) = int_0^inf exp(z v - v^2/2) dv   (substitute w = z - v in
 *         int_{-inf}^z exp((z^2 - w^2)/2) dw); positive integrand.
 * z > 0 : Phi(z) sqrt(2 pi) exp(z^2/2) with Phi(z) = erfc(-z/sqrt 2)/2, no
 *         cancellation.
 * ------------------------------------------------------------------------- */
static double f_mills(double v, const double* par) { return exp(par[0] * v - 0.5 * v * v); }

double oracle_mills(double z) {
  if (isnan(z)) return NAN;
  if (z > 0.0) {
    if (isinf(z)) return INFINITY;
    return 0.5 * erfc(-z / sqrt(2.0)) * exp(0.5 * z * z + LN_SQRT_2PI);
  }
  if (isinf(z)) return 0.0;
  double par[1] = {z};
  double brk[160];
  int n = 0;
  double h = fmin(1.0, 1.0 / fabs(z)) / 64.0;
  brk[n++] = 0.0;
  while (h < 40.0 && n < 150) {
    brk[n++] = h;
    h *= 2.0;
  }
  brk[n++] = 40.0;
  return gl_integrate(f_mills, par, brk, n);
}

/* ---------------------------------------------------------------------------
 * Row preparation shared by the price, the inversion and the adjoint.
 * ------------------------------------------------------------------------- */
static int bad_inputs(double F, double K, double T, int8_t flag) {
  if (!isfinite(F) || !isfinite(K) || !isfinite(T)) return 1;
  if (!(F > 0.0) || !(K > 0.0) || !(T > 0.0)) return 1;
  if (flag != 1 && flag != -1) return 1;
  return 0;
}

/* x = ln(F/K) with relative accuracy near the money: F - K is exact when
 * F and K are within a factor 2 of each other (Sterbenz). */
static double log_moneyness(double F, double K) {
  if (F >= 0.5 * K && F <= 2.0 * K) return log1p((F - K) / K);
  return log(F / K);
}

static double sqrt_FK(double F, double K) {
  double p = F * K;
  if (p > DBL_MIN * 4.0 && p < DBL_MAX / 4.0) return sqrt(p);
  return sqrt(F) * sqrt(K);
}

/* exact-as-possible tv = P - intrinsic: the intrinsic is theta (F - K) when
 * positive; P - F + K (or P - K + F) is formed with error-free TwoSum steps
 * and rounded once at the end */
static void two_sum(double a, double b, double* s, double* e) {
  double t = a + b, bb = t - a;
  *s = t;
  *e = (a - (t - bb)) + (b - bb);
}
static double time_value(double P, double F, double K, int theta) {
  double itm = theta > 0 ? F - K : K - F; /* sign decides; magnitude unused */
  if (!(itm > 0.0)) return P;
  double s1, e1, s2, e2;
  if (theta > 0) { two_sum(P, -F, &s1, &e1); two_sum(s1, K, &s2, &e2); }
  else           { two_sum(P, -K, &s1, &e1); two_sum(s1, F, &s2, &e2); }
  return s2 + (e1 + e2);
}

/* ---------------------------------------------------------------------------
 * Black-76 price (r = 0) and vega.
 * ------------------------------------------------------------------------- */
static void black_row(double F, double K, double T, double sig, int8_t flag, double* P, double* V) {
  if (bad_inputs(F, K, T, flag) || !(sig >= 0.0)) {
    *P = NAN;
    if (V) *V = NAN;
    return;
  }
  int theta = flag;
  double intrinsic = theta > 0 ? fmax(F - K, 0.0) : fmax(K - F, 0.0);
  double upper = theta > 0 ? F : K;
  double x = log_moneyness(F, K);
  double s = sig * sqrt(T);
  double rfk = sqrt_FK(F, K);
  if (s == 0.0) {
    *P = intrinsic;
    if (V) *V = (x == 0.0) ? rfk * sqrt(T) / sqrt(2.0 * PI) : 0.0;
    return;
  }
  if (isinf(s)) {
    *P = upper;
    if (V) *V = 0.0;
    return;
  }
  double xo = -fabs(x);
  double bs = exp(log_bs(xo, s));
  *P = intrinsic + rfk * bs * rho_of(xo, s);
  if (V) *V = rfk * bs * sqrt(T);
}

int oracle_black_price(int64_t n, const double* F, const double* K, const double* T,
                       const double* sigma, const int8_t* flag, double* P, double* vega,
                       int nthreads) {
  if (n < 0) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i)
    black_row(F[i], K[i], T[i], sigma[i], flag[i], &P[i], vega ? &vega[i] : NULL);
  (void)nthreads;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Implied volatility.
 * ------------------------------------------------------------------------- */
typedef struct {
  double x;        /* -|ln(F/K)| */
  double lnb;      /* ln beta   (beta   = tv/sqrt(FK)) */
  double lnbc;     /* ln beta_c (beta_c = (U - P)/sqrt(FK)) */
  double beta, betac; /* the same, unlogged (0 where they underflow) */
  double beta_hi;  /* beta 2^BETA_SCALE_EXP where beta is subnormal (tv 2^BETA_SCALE_EXP / sqrt(FK)), else 0 */
  int upper;       /* solve on the complement */
} solve_t;

/* A subnormal beta is compared with b through this exact power-of-two scaling:
 * ln b - ln beta as a difference of logarithms would carry an absolute error
 * ~ eps |ln beta| ~ 700 eps, which near the money (where d ln b / d ln s ~ 1)
 * is a relative error of ~700 eps in the root. */
#define BETA_SCALE_EXP 600

/* objective g(s), increasing in s, and its s-derivative; returns 0 when the
 * cheap bound alone decided the sign (deriv is then unset) */
static int objective(const solve_t* q, double s, double* g, double* dg) {
  double lbs = log_bs(q->x, s);
  double h = q->x / s;
  /* outside the regime where the scaled integral is safe, b is within a
   * rounding of 0 or b_max and only the sign of g is needed */
  if (!q->upper && 0.125 * s * s > REGIME) { *g = 0.5 * q->x - q->lnb; return 0; }
  if (q->upper && 0.5 * h * h > REGIME) { *g = q->lnbc - 0.5 * q->x; return 0; }
  if (!q->upper) {
    /* rho <= s e^B, so ln b <= ln b_s + ln s + B */
    double bound = lbs + log(s) + 0.125 * s * s;
    if (bound < q->lnb - 1.0) { *g = bound - q->lnb; return 0; }
    double r = rho_of(q->x, s);
    /* ln(b/beta): as the log of one ratio when everything is representable
     * (absolute error ~ eps), else as a sum of logarithms */
    if (lbs > -700.0 && q->beta > 0.0) *g = log(exp(lbs) * r / q->beta);
    else if (lbs > -700.0 && q->beta_hi > 0.0 && r < 1e100)
      *g = log(ldexp(r, BETA_SCALE_EXP) * exp(lbs) / q->beta_hi); /* r 2^600 is exact */
    else *g = lbs + log(r) - q->lnb;
    *dg = 1.0 / r;
    return 1;
  }
  double gm = gamma_of(q->x, s);
  if (lbs > -700.0 && q->betac > 0.0) *g = log(q->betac / (exp(lbs) * gm));
  else *g = q->lnbc - (lbs + log(gm));
  *dg = 1.0 / gm;
  return 1;
}

static double solve_s(const solve_t* q) {
  double lo = 0.0, hi = INFINITY, s = 1.0;
  double gprev = INFINITY;
  for (int it = 0; it < 600; ++it) {
    double g = 0.0, dg = 0.0;
    int have_d = objective(q, s, &g, &dg);
    if (g == 0.0) return s;
    if (g < 0.0) lo = s; else hi = s;
    double sn = NAN;
    if (have_d && isfinite(dg) && dg > 0.0) sn = s - g / dg;
    int newton_ok = sn > lo && sn < hi;
    if (newton_ok && fabs(sn - s) <= 2.0 * DBL_EPSILON * s) return sn;
    if (isfinite(hi) && hi - lo <= 4.0 * DBL_EPSILON * hi) return 0.5 * (lo + hi);
    /* bisect (geometrically) when Newton leaves the bracket or stalls */
    if (!newton_ok || fabs(g) > 0.5 * gprev) {
      if (lo > 0.0 && isfinite(hi)) sn = sqrt(lo) * sqrt(hi);
      else if (isfinite(hi)) sn = hi < 0.5 ? hi * hi : 0.5 * hi; /* roots reach ~1e-320 */
      else sn = 2.0 * s;
      if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
    }
    gprev = fabs(g);
    s = sn;
  }
  return s;
}

static void iv_row(double F, double K, double T, double P, int8_t flag, double* sig, uint8_t* st) {
  if (bad_inputs(F, K, T, flag) || !isfinite(P)) { *sig = NAN; *st = 3; return; }
  int theta = flag;
  double upper = theta > 0 ? F : K;
  double tv = time_value(P, F, K, theta);
  double cv = upper - P;
  if (tv < 0.0) { *sig = NAN; *st = 1; return; }
  if (cv < 0.0) { *sig = NAN; *st = 2; return; }
  if (tv == 0.0) { *sig = 0.0; *st = 4; return; }
  if (cv == 0.0) { *sig = INFINITY; *st = 5; return; }
  double rfk = sqrt_FK(F, K);
  double beta = tv / rfk, betac = cv / rfk;
  solve_t q;
  q.x = -fabs(log_moneyness(F, K));
  q.lnb = beta >= DBL_MIN ? log(beta) : log(tv) - log(rfk);
  q.lnbc = betac >= DBL_MIN ? log(betac) : log(cv) - log(rfk);
  q.beta = beta >= DBL_MIN ? beta : 0.0;
  q.betac = betac >= DBL_MIN ? betac : 0.0;
  q.beta_hi = beta >= DBL_MIN ? 0.0 : ldexp(tv, BETA_SCALE_EXP) / rfk;
  q.upper = q.lnb > q.lnbc; /* beta > b_max/2 */
  double s = solve_s(&q);
  *sig = s / sqrt(T);
  *st = 0;
}

int oracle_iv(int64_t n, const double* F, const double* K, const double* T,
              const double* P, const int8_t* flag, double* sigma, uint8_t* status,
              int nthreads) {
  if (n < 0) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i) {
    uint8_t st;
    iv_row(F[i], K[i], T[i], P[i], flag[i], &sigma[i], &st);
    if (status) status[i] = st;
  }
  (void)nthreads;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Adjoint with the low-vega gate.
 * ------------------------------------------------------------------------- */
static void grad_row(double F, double K, double T, int8_t flag, double sig, double g,
                     double tau, int mode, double out[4]) {
  if (bad_inputs(F, K, T, flag) || isnan(sig) || sig < 0.0 || isnan(g)) {
    out[0] = out[1] = out[2] = out[3] = NAN;
    return;
  }
  if (sig == 0.0 || isinf(sig)) {
    /* the price sits on a bound of the no-arbitrage interval: V = 0, outside
     * every G_tau, and the IFT gives no finite derivative */
    double v = NAN;
    if (mode == 1) v = (g == 0.0) ? 0.0 : NAN;
    if (mode == 2 || mode == 3) v = 0.0;
    out[0] = out[1] = out[2] = out[3] = v;
    return;
  }
  double x = log_moneyness(F, K);
  double sqT = sqrt(T);
  double s = sig * sqT;
  double V = sqrt_FK(F, K) * exp(log_bs(x, s)) * sqT; /* = F phi(d1) sqrt(T) */
  double d1 = x / s + 0.5 * s, d2 = d1 - s;
  double jF, jK;
  if (flag > 0) {
    jF = -oracle_mills(d1) / (F * sqT); /* -Phi(d1) / V */
    jK = oracle_mills(d2) / (K * sqT);  /*  Phi(d2) / V, K phi(d2) = F phi(d1) */
  } else {
    jF = oracle_mills(-d1) / (F * sqT);  /*  Phi(-d1) / V */
    jK = -oracle_mills(-d2) / (K * sqT); /* -Phi(-d2) / V */
  }
  double jP = 1.0 / V;
  double jT = -sig / (2.0 * T);
  int in_g = fabs(V) > tau;
  if (mode == 0 || ((mode == 1 || mode == 2) && in_g)) {
    out[0] = g * jP; out[1] = g * jF; out[2] = g * jK; out[3] = g * jT;
    return;
  }
  if (mode == 1) {
    double v = (g == 0.0) ? 0.0 : NAN;
    out[0] = out[1] = out[2] = out[3] = v;
    return;
  }
  if (mode == 2) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    return;
  }
  /* mode 3: w = V^2/(V^2 + tau^2) on every row; w/V = V/(V^2 + tau^2) */
  double w, wP;
  if (V > tau) {
    double r = tau / V;
    w = 1.0 / (1.0 + r * r);
    wP = w / V;
  } else {
    double r = V / tau;
    w = r * r / (1.0 + r * r);
    wP = (r / tau) / (1.0 + r * r);
  }
  out[0] = g * wP; out[1] = g * jF * w; out[2] = g * jK * w; out[3] = g * jT * w;
}

int oracle_iv_grad(int64_t n, const double* F, const double* K, const double* T,
                   const int8_t* flag, const double* sigma, const double* gbar,
                   double tau, int gate_mode, double* dP, double* dF, double* dK,
                   double* dT, int nthreads) {
  if (n < 0 || gate_mode < 0 || gate_mode > 3 || !(tau >= 0.0)) return 1;
  if (gate_mode == 3 && !(tau > 0.0)) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double o[4];
    grad_row(F[i], K[i], T[i], flag[i], sigma[i], gbar ? gbar[i] : 1.0, tau, gate_mode, o);
    if (dP) dP[i] = o[0];
    if (dF) dF[i] = o[1];
    if (dK) dK[i] = o[2];
    if (dT) dT[i] = o[3];
  }
  (void)nthreads;
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Vector-Jacobian product of the Black-76 price (r = 0) in (sigma, F, K, T),
 * straight from differentiating Eq. app_black76:
 *   dP/dsigma = V = F phi(d1) sqrt(T),       dP/dT = V sigma / (2T),
 *   dP/dF = Phi(d1) (call), Phi(d1) - 1 (put),
 *   dP/dK = -Phi(d2) (call), 1 - Phi(d2) (put),
 * Phi(z) = erfc(-z/sqrt 2)/2.  sigma = 0: one-sided limits of the intrinsic
 * value (1/2 at the money); sigma = +inf: the upper bound F (call) or K (put).
 * ------------------------------------------------------------------------- */
static double Phi(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

static void price_grad_row(double F, double K, double T, double sig, int8_t flag, double g, double out[4]) {
  if (bad_inputs(F, K, T, flag) || !(sig >= 0.0) || isnan(g)) {
    out[0] = out[1] = out[2] = out[3] = NAN;
    return;
  }
  int theta = flag;
  double x = log_moneyness(F, K);
  if (sig == 0.0 || isinf(sig)) {
    double dF, dK, V = 0.0;
    if (sig == 0.0) {
      double itm = theta * x > 0.0 ? 1.0 : (x == 0.0 ? 0.5 : 0.0);
      dF = theta * itm;
      dK = -theta * itm;
      if (x == 0.0) V = sqrt_FK(F, K) * sqrt(T) / sqrt(2.0 * PI);
    } else {
      dF = theta > 0 ? 1.0 : 0.0;
      dK = theta > 0 ? 0.0 : 1.0;
    }
    out[0] = g * V; out[1] = g * dF; out[2] = g * dK; out[3] = 0.0;
    return;
  }
  double sqT = sqrt(T), s = sig * sqT;
  double d1 = x / s + 0.5 * s, d2 = d1 - s;
  double V = F * exp(-0.5 * d1 * d1) / sqrt(2.0 * PI) * sqT;
  double dF = theta > 0 ? Phi(d1) : -Phi(-d1);
  double dK = theta > 0 ? -Phi(d2) : Phi(-d2);
  out[0] = g * V; out[1] = g * dF; out[2] = g * dK; out[3] = g * V * sig / (2.0 * T);
}

int oracle_black_price_grad(int64_t n, const double* F, const double* K, const double* T, const double* sigma,
                            const int8_t* flag, const double* gbar, double* dsigma, double* dF, double* dK,
                            double* dT, int nthreads) {
  if (n < 0) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double o[4];
    price_grad_row(F[i], K[i], T[i], sigma[i], flag[i], gbar ? gbar[i] : 1.0, o);
    if (dsigma) dsigma[i] = o[0];
    if (dF) dF[i] = o[1];
    if (dK) dK[i] = o[2];
    if (dT) dT[i] = o[3];
  }
  (void)nthreads;
  return 0;
}

/* ---------------------------------------------------------------------------
 * The Black-Scholes interface on xi = (S, K, tau, r, q) (Section 2, Eq.
 * app_forward_price and Eq. app_black_scholes; Section 3, Algorithm 1).
 *
 *  - Price: Eq. app_black_scholes equals the discounted Black-76 price in
 *    forward coordinates (Eq. app_black76): V = e^{-r tau} B(F, K, tau, sigma)
 *    with F = S e^{(r - q) tau}.
 *  - Implied volatility: Algorithm 1's forward normalisation, F = S e^{(r-q) tau}
 *    and B = e^{r tau} V, then the Black-76 inversion above.  Rows with a
 *    non-finite r or q are bad inputs (status 3).
 *  - Adjoint: Algorithm 1's backward, Vbar = gbar / V_bs and
 *    xibar = -gbar (dV/dxi) / V_bs, with the Greeks of Eq. app_black_scholes
 *    differentiated directly (theta = +1 call, -1 put, M = Phi/phi):
 *      V_bs     = S e^{-q tau} phi(d1) sqrt(tau)            (vega)
 *      dV/dS    =  theta e^{-q tau} Phi(theta d1)
 *      dV/dK    = -theta e^{-r tau} Phi(theta d2)
 *      dV/dr    =  theta K tau e^{-r tau} Phi(theta d2)
 *      dV/dq    = -theta S tau e^{-q tau} Phi(theta d1)
 *      dV/dtau  =  V_bs sigma/(2 tau) - theta q S e^{-q tau} Phi(theta d1)
 *                 + theta r K e^{-r tau} Phi(theta d2)
 *    and, with S e^{-q tau} phi(d1) = K e^{-r tau} phi(d2), each ratio to V_bs
 *    is a Mills ratio times a plain factor.  The gate of Section 3.3 compares
 *    V_bs (the derivative of the cash price in sigma) with tau_gate.
 * ------------------------------------------------------------------------- */
static int bs_to_black(double S, double T, double r, double q, double Vm, double* F, double* B) {
  if (!isfinite(r) || !isfinite(q)) return 1;
  *F = S * exp((r - q) * T);
  *B = Vm * exp(r * T);
  return 0;
}

int oracle_bs_price(int64_t n, const double* S, const double* K, const double* T, const double* r,
                    const double* q, const double* sigma, const int8_t* flag, double* V, double* vega,
                    int nthreads) {
  if (n < 0) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double F, unused, P, Vb;
    if (bs_to_black(S[i], T[i], r[i], q[i], 0.0, &F, &unused)) {
      V[i] = NAN;
      if (vega) vega[i] = NAN;
      continue;
    }
    black_row(F, K[i], T[i], sigma[i], flag[i], &P, &Vb);
    double disc = exp(-r[i] * T[i]);
    V[i] = disc * P;
    if (vega) vega[i] = disc * Vb;
  }
  (void)nthreads;
  return 0;
}

int oracle_bs_iv(int64_t n, const double* S, const double* K, const double* T, const double* r,
                 const double* q, const double* Vm, const int8_t* flag, double* sigma, uint8_t* status,
                 int nthreads) {
  if (n < 0) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i) {
    uint8_t st;
    double F, B;
    if (bs_to_black(S[i], T[i], r[i], q[i], Vm[i], &F, &B)) {
      sigma[i] = NAN;
      st = 3;
    } else {
      iv_row(F, K[i], T[i], B, flag[i], &sigma[i], &st);
    }
    if (status) status[i] = st;
  }
  (void)nthreads;
  return 0;
}

static void bs_grad_row(double S, double K, double T, double r, double q, int8_t flag, double sig, double g,
                        double tau, int mode, double out[6]) {
  int k;
  if (bad_inputs(S, K, T, flag) || !isfinite(r) || !isfinite(q) || isnan(sig) || sig < 0.0 || isnan(g)) {
    for (k = 0; k < 6; ++k) out[k] = NAN;
    return;
  }
  if (sig == 0.0 || isinf(sig)) {
    double v = NAN;
    if (mode == 1) v = (g == 0.0) ? 0.0 : NAN;
    if (mode == 2 || mode == 3) v = 0.0;
    for (k = 0; k < 6; ++k) out[k] = v;
    return;
  }
  int theta = flag;
  double sqT = sqrt(T);
  double s = sig * sqT;
  double x = log(S / K) + (r - q) * T; /* ln(F/K), Eq. app_black_scholes's d1 numerator */
  double d1 = x / s + 0.5 * s, d2 = d1 - s;
  double Vbs = exp(log(S) - q * T - 0.5 * d1 * d1 - LN_SQRT_2PI) * sqT;
  double M1 = oracle_mills(theta * d1), M2 = oracle_mills(theta * d2);
  double j[6];
  j[0] = 1.0 / Vbs;                                             /* dsigma/dV   */
  j[1] = -theta * M1 / (S * sqT);                               /* dsigma/dS   */
  j[2] = theta * M2 / (K * sqT);                                /* dsigma/dK   */
  j[3] = -sig / (2.0 * T) + theta * (q * M1 - r * M2) / sqT;    /* dsigma/dtau */
  j[4] = -theta * sqT * M2;                                     /* dsigma/dr   */
  j[5] = theta * sqT * M1;                                      /* dsigma/dq   */
  int in_g = fabs(Vbs) > tau;
  if (mode == 0 || ((mode == 1 || mode == 2) && in_g)) {
    for (k = 0; k < 6; ++k) out[k] = g * j[k];
    return;
  }
  if (mode == 1 || mode == 2) {
    double v = (mode == 1 && g != 0.0) ? NAN : 0.0;
    for (k = 0; k < 6; ++k) out[k] = v;
    return;
  }
  double w, wP;
  if (Vbs > tau) {
    double rr = tau / Vbs;
    w = 1.0 / (1.0 + rr * rr);
    wP = w / Vbs;
  } else {
    double rr = Vbs / tau;
    w = rr * rr / (1.0 + rr * rr);
    wP = (rr / tau) / (1.0 + rr * rr);
  }
  out[0] = g * wP;
  for (k = 1; k < 6; ++k) out[k] = g * j[k] * w;
}

int oracle_bs_iv_grad(int64_t n, const double* S, const double* K, const double* T, const double* r,
                      const double* q, const int8_t* flag, const double* sigma, const double* gbar,
                      double tau, int gate_mode, double* dV, double* dS, double* dK, double* dT,
                      double* dr, double* dq, int nthreads) {
  if (n < 0 || gate_mode < 0 || gate_mode > 3 || !(tau >= 0.0)) return 1;
  if (gate_mode == 3 && !(tau > 0.0)) return 1;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double o[6];
    bs_grad_row(S[i], K[i], T[i], r[i], q[i], flag[i], sigma[i], gbar ? gbar[i] : 1.0, tau, gate_mode, o);
    if (dV) dV[i] = o[0];
    if (dS) dS[i] = o[1];
    if (dK) dK[i] = o[2];
    if (dT) dT[i] = o[3];
    if (dr) dr[i] = o[4];
    if (dq) dq[i] = o[5];
  }
  (void)nthreads;
  return 0;
}

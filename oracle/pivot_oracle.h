/*
 * pivot_oracle.h -- plain FP64 CPU oracle for the PIVOT hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Conventions (all arrays are host memory, structure-of-arrays, length n):
 *   F  forward, K strike, T time to expiry (years), P undiscounted Black-76
 *   price (r = 0), sigma annualised volatility, flag +1 call / -1 put.
 *   s = sigma*sqrt(T) is the total volatility, x = ln(F/K).
 * Status codes written by oracle_iv:
 *   0 ok, 1 below intrinsic, 2 above the upper bound (F for calls, K for puts),
 *   3 bad input (non-finite, F/K/T <= 0, flag not +-1),
 *   4 price equals intrinsic (sigma = 0), 5 price equals the upper bound
 *   (sigma = +inf).  Rows with status 1..3 get sigma = NaN.
 * Gate modes of oracle_iv_grad (Section 3.3, Eq. smooth_gate):
 *   0 exact IFT value, 1 NaN off G_tau (0 where the cotangent is 0),
 *   2 hard mask (0 off G_tau), 3 smooth gate w_tau on every row.
 */
#ifndef PIVOT_ORACLE_H
#define PIVOT_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* normalised Black function b(x,s) for x <= 0 (out-of-the-money call form) */
double oracle_normalised_black(double x, double s);
/* its complement b_max(x) - b(x,s) = exp(x/2) - b(x,s), x <= 0 */
double oracle_normalised_black_complement(double x, double s);
/* ln b(x,s), finite even where b underflows */
double oracle_log_normalised_black(double x, double s);
/* Mills-type ratio Phi(z)/phi(z) */
double oracle_mills(double z);

int oracle_black_price(int64_t n, const double* F, const double* K, const double* T,
                       const double* sigma, const int8_t* flag, double* P, double* vega,
                       int nthreads);
int oracle_iv(int64_t n, const double* F, const double* K, const double* T,
              const double* P, const int8_t* flag, double* sigma, uint8_t* status,
              int nthreads);
int oracle_iv_grad(int64_t n, const double* F, const double* K, const double* T,
                   const int8_t* flag, const double* sigma, const double* gbar,
                   double tau, int gate_mode, double* dP, double* dF, double* dK,
                   double* dT, int nthreads);
/* VJP of the Black-76 price in (sigma, F, K, T); gbar may be NULL (= 1) */
int oracle_black_price_grad(int64_t n, const double* F, const double* K, const double* T,
                            const double* sigma, const int8_t* flag, const double* gbar,
                            double* dsigma, double* dF, double* dK, double* dT, int nthreads);
/* Black-Scholes interface on xi = (S, K, T = tau, r, q), V the discounted price:
 * price and vega dV/dsigma; sigma and status; the gated VJP
 * (dV, dS, dK, dT, dr, dq), the gate comparing the cash vega with tau. */
int oracle_bs_price(int64_t n, const double* S, const double* K, const double* T, const double* r,
                    const double* q, const double* sigma, const int8_t* flag, double* V, double* vega,
                    int nthreads);
int oracle_bs_iv(int64_t n, const double* S, const double* K, const double* T, const double* r,
                 const double* q, const double* Vm, const int8_t* flag, double* sigma, uint8_t* status,
                 int nthreads);
int oracle_bs_iv_grad(int64_t n, const double* S, const double* K, const double* T, const double* r,
                      const double* q, const int8_t* flag, const double* sigma, const double* gbar,
                      double tau, int gate_mode, double* dV, double* dS, double* dK, double* dT,
                      double* dr, double* dq, int nthreads);
/* number of threads OpenMP would use for nthreads <= 0 */
int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif

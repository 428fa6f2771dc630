/*
 * pivot.h -- C ABI of the PIVOT implied-volatility hot path on GB300 (sm_103a).
 *
 * The library inverts undiscounted Black-76 prices (forward measure, r = 0)
 * to implied volatilities in "Let's Be Rational" form (normalised Black
 * function, region-wise rational initial guess, Householder(3) refinement) and
 * supplies the implicit-function-theorem adjoint with the low-vega gating
 * contract.  Paper: "PIVOT: Bridging Black-Scholes Implied-Volatility and
 * Price Objectives via Differentiable Jaeckel Operator", Algorithm 1,
 * Section 3 (forward, backward, low-vega gating) and the appendix on the
 * five-stage LBR construction.
 *
 * Common conventions for every entry point
 *   - Arrays are structure-of-arrays of length n in DEVICE memory (cudaMalloc,
 *     torch CUDA tensors or managed memory), owned by the caller.  The
 *     library allocates nothing and keeps no pointer after the call returns.
 *   - float64 arrays must be 8-byte aligned; int8/uint8 arrays need no
 *     alignment.  Input and output arrays must not overlap.
 *   - F: forward (> 0), K: strike (> 0), T: time to expiry in years (> 0),
 *     P: undiscounted option price, sigma: annualised volatility,
 *     flag: +1 call, -1 put.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *     is asynchronous on that stream; results are valid once the stream has
 *     been synchronised.
 *   - Return value: 0 on success; > 0 an argument error (see PIVOT_E_*),
 *     nothing was launched; < 0 the negated cudaError_t of a failed launch.
 *   - n == 0 is valid and launches nothing.
 *   - Per-row problems are values, not return codes: NaN sigma plus a status
 *     code (PIVOT_ROW_*), and NaN gradients for invalid rows.
 */
#ifndef PIVOT_H
#define PIVOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define PIVOT_OK 0
#define PIVOT_E_SIZE 1        /* n < 0 */
#define PIVOT_E_NULL 2        /* a required pointer is NULL */
#define PIVOT_E_GATE 3        /* gate_mode outside 0..3, tau < 0 or NaN, or tau == 0 with the smooth gate */
#define PIVOT_E_OPTS 4        /* bad pivot_opts field */
#define PIVOT_E_NOT_DEVICE 5  /* a pointer is not accessible from the current device */
#define PIVOT_E_ALIGN 6       /* a float64 pointer is not 8-byte aligned */
#define PIVOT_E_MLP 7         /* PIVOT_MODE_LEARNED without weights, or bad training hyper-parameters */
#define PIVOT_E_TOO_MANY 8    /* n above the row limit of pivot_mlp_grad_static */

/* ---- per-row status codes (uint8) --------------------------------------- */
#define PIVOT_ROW_OK 0              /* sigma finite and > 0 */
#define PIVOT_ROW_BELOW_INTRINSIC 1 /* P < intrinsic value: sigma = NaN (Section 3.1) */
#define PIVOT_ROW_ABOVE_UPPER 2     /* P > F (call) or K (put), super-arbitrage: sigma = NaN */
#define PIVOT_ROW_BAD_INPUT 3       /* non-finite input, F, K or T <= 0, flag not +-1: sigma = NaN */
#define PIVOT_ROW_AT_INTRINSIC 4    /* P equals the intrinsic value: sigma = 0 */
#define PIVOT_ROW_AT_UPPER 5        /* P equals the upper bound: sigma = +inf */

/* ---- gate modes of the backward (Section 3.3, Eq. wellcond_set, smooth_gate) ---- */
#define PIVOT_GATE_EXACT 0  /* the exact IFT value on every valid row */
#define PIVOT_GATE_NAN 1    /* exact on G_tau = {|V| > tau}; off G_tau 0 where the cotangent is 0, else NaN */
#define PIVOT_GATE_MASK 2   /* exact on G_tau, 0 off G_tau (hard mask 1{|V| > tau}) */
#define PIVOT_GATE_SMOOTH 3 /* every row times w_tau(V) = V^2 / (V^2 + tau^2) */

/* ---- forward variants ----------------------------------------------------- */
#define PIVOT_MODE_FP64 0    /* plain FP64 throughout */
#define PIVOT_MODE_MIXED 1   /* FP32 guess and first Householder step, FP64 final step */
#define PIVOT_MODE_LEARNED 2 /* MLP initial guess (BF16 tensor cores), FP64 Householder steps */

/* ---- learned initial guess ------------------------------------------------
 * An MLP 2 -> 64 -> 64 -> 64 -> 1 (SiLU) maps (|x|, q = 1/sqrt(-2 ln beta))
 * to ln(s / s_a), s_a = |x| q + sqrt(2 pi) beta, for the out-of-the-money
 * normalised problem b(x, s) = beta.  Weights are BF16 (bit patterns in
 * uint16), biases FP32, accumulation FP32.  Flat FP32 parameter order:
 * w1[64][2], b1[64], w2[64][64], b2[64], w3[64][64], b3[64], w4[64], b4
 * (w[unit][input]).  Not in the paper: the paper keeps LBR's rational seed;
 * this is the surrogate seed the build adds and measures against it. */
#define PIVOT_MLP_HIDDEN 64
#define PIVOT_MLP_NPARAM 8577

typedef struct {
  uint16_t w1[64 * 2];  /* bf16 [unit][input] */
  uint16_t w2[64 * 64]; /* bf16 [unit][input] */
  uint16_t w3[64 * 64]; /* bf16 [unit][input] */
  uint16_t w4[64];      /* bf16 */
  float b1[64], b2[64], b3[64];
  float b4;
  float reserved[3];
} pivot_mlp; /* inference weights, device memory */

typedef struct {
  float param[PIVOT_MLP_NPARAM]; /* FP32 master parameters (flat order above) */
  float grad[PIVOT_MLP_NPARAM];  /* gradient accumulator (zeroed by pivot_mlp_adam) */
  float adam_m[PIVOT_MLP_NPARAM];
  float adam_v[PIVOT_MLP_NPARAM];
  double loss_sum; /* sum of squared errors accumulated by pivot_mlp_grad */
  double rows;     /* rows that entered loss_sum */
  int64_t step;    /* Adam steps taken */
  pivot_mlp net;   /* BF16 copy of the parameters, refreshed by pivot_mlp_init / pivot_mlp_adam */
} pivot_mlp_trainer; /* training state, device memory owned by the caller */

/* ---- per-launch counters (optional) -----------------------------------------
 * pivot_opts.counters, when not NULL, is a device array of PIVOT_COUNTERS_LEN
 * uint64 that the forward kernels ADD to (the caller clears it):
 *   [0..5]   rows by status code PIVOT_ROW_* (0: solved)
 *   [6..17]  solved rows by the kernel's bin, [6 + b] for bin b:
 *            FP64:    0 lower, 1 mid-low, 2 mid-high, 3 upper, 4 mid-low near the
 *                     money (|ln(F/K)| <= 0.1), 5 mid-high near the money, 6 lower
 *                     with beta < 1e-100, 7 lower near the money
 *            MIXED:   0-3 the four regions seeded in float, 4-7 the four regions
 *                     in FP64 (outside the float range), 8 deep lower tail seeded
 *                     in float from ln beta, 9 mid-low and 10 mid-high near the
 *                     money in float, 11 lower near the money in float
 *            LEARNED: 0 lower, 1 b - beta, 2 upper (MLP seed), 3 deep lower tail
 *                     (float seed from ln beta), 4 lower and 5 b - beta near the
 *                     money (MLP seed)
 *   [18]     rows of the accelerated form (MIXED float-seeded, LEARNED) not
 *            accepted and solved again from LBR's rational seed in FP64
 *   [19..23] reserved (left unchanged)
 * Counting costs a few shared-memory atomics per warp; a NULL pointer costs
 * nothing.  Not in the paper: the invalid-domain and region rates it reports
 * per dataset come from these. */
#define PIVOT_COUNTERS_LEN 24

typedef struct {
  int32_t mode;          /* PIVOT_MODE_* ; default PIVOT_MODE_FP64 */
  int32_t householder;   /* Householder(3) iterations after the initial guess, 0 = default (2), max 4;
                            MIXED and LEARNED: the last one in FP64, the others in float */
  const pivot_mlp* mlp;  /* PIVOT_MODE_LEARNED: device pointer to the weights, else ignored */
  double fallback;       /* PIVOT_MODE_LEARNED: float steps moving the MLP seed by more than this
                            (relative), or a final FP64 step moving the float iterate by more than
                            1e-5, send the row to the rational-guess FP64 path; 0 = default 0.25 */
  uint64_t* counters;    /* NULL, or PIVOT_COUNTERS_LEN device uint64 counters (above), 8-byte aligned */
} pivot_opts;

/*
 * pivot_black_price -- undiscounted Black-76 price with r = 0 (Eq. app_black76)
 * and vega V = F phi(d1) sqrt(T) (Eq. app_vega_closed_form).
 *   in : F, K, T, sigma (n float64), flag (n int8)
 *   out: P_out (n float64); vega_out (n float64, may be NULL)
 * sigma = 0 gives the intrinsic value, sigma = +inf the upper bound; invalid
 * rows (non-finite, F/K/T <= 0, sigma < 0, bad flag) give NaN.
 */
int pivot_black_price(int64_t n, const double* F, const double* K, const double* T,
                      const double* sigma, const int8_t* flag, double* P_out,
                      double* vega_out, void* stream);

/*
 * pivot_black_price_backward -- vector-Jacobian product of the Black-76 price
 * (r = 0) in (sigma, F, K, T) (Eq. app_black76; vega Eq. app_vega_closed_form):
 *   dsigma = gbar V,  dF = gbar dP/dF,  dK = gbar dP/dK,  dT = gbar V sigma / (2T),
 * with dP/dF = Phi(d1) (call) or -Phi(-d1) (put), dP/dK = -Phi(d2) (call) or
 * Phi(-d2) (put).  This is the smooth price node through which an IV-space
 * loss reaches a pricer (Section 3.2, "Differentiable IV inside the loss").
 *   in : F, K, T, sigma (n float64), flag (n int8), gbar (n float64; NULL = 1)
 *   out: dsigma, dF, dK, dT (n float64 each, any may be NULL)
 * sigma = 0 gives the one-sided limits (delta of the intrinsic value, V = 0
 * except at the money); invalid rows give NaN.
 */
int pivot_black_price_backward(int64_t n, const double* F, const double* K, const double* T,
                               const double* sigma, const int8_t* flag, const double* gbar,
                               double* dsigma, double* dF, double* dK, double* dT, void* stream);

/*
 * pivot_iv_forward -- implied volatility, Algorithm 1 (forward): normalise to
 * (x, beta) with beta = (P - intrinsic)/sqrt(F K), solve b(x, s) = beta in LBR
 * form (appendix stages 1-5), return sigma = s / sqrt(T).
 *   in : F, K, T, P (n float64), flag (n int8)
 *   out: sigma_out (n float64); status_out (n uint8, may be NULL)
 *   opts: may be NULL (plain FP64, 2 Householder steps)
 */
int pivot_iv_forward(int64_t n, const double* F, const double* K, const double* T,
                     const double* P, const int8_t* flag, double* sigma_out,
                     uint8_t* status_out, const pivot_opts* opts, void* stream);

/*
 * pivot_iv_backward -- vector-Jacobian product of sigma(P, F, K, T), Algorithm 1
 * (backward) and Eq. method_vjp:
 *   dP = gbar / V,  dF = -gbar (dP_B/dF) / V,  dK = -gbar (dP_B/dK) / V,
 *   dT = -gbar sigma / (2 T),
 * recomputed from the saved (F, K, T, flag, sigma) only (Section 3.2), then
 * gated per gate_mode with threshold tau (cash vega units).
 *   in : F, K, T, sigma (n float64), flag (n int8),
 *        gbar (n float64 upstream cotangent; NULL means 1 on every row, i.e.
 *        the diagonal of the Jacobian), tau >= 0, gate_mode PIVOT_GATE_*
 *   out: dP, dF, dK, dT (n float64 each, any may be NULL to skip)
 * Rows with NaN sigma give NaN.  Rows with sigma = 0 or +inf sit on a bound of
 * the price interval (V = 0, outside every G_tau): NaN in the exact mode,
 * otherwise the off-G_tau value of the gate.
 */
int pivot_iv_backward(int64_t n, const double* F, const double* K, const double* T,
                      const int8_t* flag, const double* sigma, const double* gbar,
                      double tau, int32_t gate_mode, double* dP, double* dF, double* dK,
                      double* dT, void* stream);

/*
 * pivot_iv_forward_backward -- both of the above in one pass over HBM: the
 * forward result and its gated adjoint, same conventions.  sigma_out is
 * required; status_out and each gradient output may be NULL.
 */
int pivot_iv_forward_backward(int64_t n, const double* F, const double* K, const double* T,
                              const double* P, const int8_t* flag, const double* gbar,
                              double tau, int32_t gate_mode, double* sigma_out,
                              uint8_t* status_out, double* dP, double* dF, double* dK,
                              double* dT, const pivot_opts* opts, void* stream);

/*
 * Black-Scholes interface on the paper's tuple xi = (S, K, tau, r, q) (Section 2,
 * Eq. app_forward_price and Eq. app_black_scholes; Section 3, Algorithm 1).
 * Row inputs: spot S, strike K, time to expiry T (the paper's tau, years),
 * risk-free rate r and dividend yield / cost of carry q (continuous, any
 * finite sign), the DISCOUNTED market price V, flag +1 call / -1 put; all
 * float64 except the int8 flag, device memory of one device.
 * Forward (Algorithm 1): F = S e^{(r-q) T}, B = e^{r T} V, then the Black-76
 * inversion of pivot_iv_forward on (F, K, T, B); the status codes refer to B
 * against the Black-76 bounds, i.e. V against the discounted intrinsic value
 * e^{-r T} max(theta (F - K), 0) and the discounted upper bound (S e^{-q T}
 * for calls, K e^{-r T} for puts).  A non-finite r or q is a bad input.
 * Backward (Algorithm 1, Eq. method_vjp): dV = gbar / V_bs and
 * d(S, K, T, r, q) = -gbar (dV/d(S, K, T, r, q)) / V_bs, V_bs = dV/dsigma the
 * cash vega; the gate of Section 3.3 compares V_bs with tau.
 * PIVOT_MODE_LEARNED is not offered on this form (PIVOT_E_OPTS): its seed was
 * trained on Black-76 rows only; FP64 and MIXED are.
 */

/* V = e^{-r T} B(F, K, T, sigma) and, if vega_out is not NULL, dV/dsigma. */
int pivot_bs_price(int64_t n, const double* S, const double* K, const double* T, const double* r,
                   const double* q, const double* sigma, const int8_t* flag, double* V_out,
                   double* vega_out, void* stream);

/* sigma (required) and status (may be NULL) per row; opts as for pivot_iv_forward. */
int pivot_bs_iv_forward(int64_t n, const double* S, const double* K, const double* T, const double* r,
                        const double* q, const double* V, const int8_t* flag, double* sigma_out,
                        uint8_t* status_out, const pivot_opts* opts, void* stream);

/* The gated VJP from the saved (S, K, T, r, q, flag, sigma); gbar, tau and
 * gate_mode as for pivot_iv_backward; each output may be NULL. */
int pivot_bs_iv_backward(int64_t n, const double* S, const double* K, const double* T, const double* r,
                         const double* q, const int8_t* flag, const double* sigma, const double* gbar,
                         double tau, int32_t gate_mode, double* dV, double* dS, double* dK, double* dT,
                         double* dr, double* dq, void* stream);

/* Both in one pass over HBM. */
int pivot_bs_iv_forward_backward(int64_t n, const double* S, const double* K, const double* T,
                                 const double* r, const double* q, const double* V, const int8_t* flag,
                                 const double* gbar, double tau, int32_t gate_mode, double* sigma_out,
                                 uint8_t* status_out, double* dV, double* dS, double* dK, double* dT,
                                 double* dr, double* dq, const pivot_opts* opts, void* stream);

/*
 * pivot_mills_ratio -- Y(z) = Phi(z)/phi(z), the ratio through which the
 * adjoint writes Delta/V (Eq. implicit_iv with F phi(d1) = K phi(d2)) and the
 * normalised Black function writes b/b_s (Section 2, Eq. app_normalized_black).
 *   in : z (n float64)   out: y (n float64)
 * Exposed so that the FP64 Mills-ratio table behind it can be checked on its own.
 */
int pivot_mills_ratio(int64_t n, const double* z, double* y, void* stream);

/*
 * pivot_elementary -- the library's table-driven FP64 logarithm (fn = 0) and
 * exponential (fn = 1), which the solver uses for ln b, ln beta, 1/b_s and
 * the seeds (P. T. P. Tang's method; within 1 ulp), and (fn = 2) the
 * -Phi^{-1}(x) of the lower- and upper-region guesses (appendix stage 4),
 * x in (0, 1/2]: from 1e-37 on the float inverse normal CDF (seed accuracy,
 * relative error ~1e-6), below it the library's FP64 normcdfinv; (fn = 3) 1/x
 * by the solver's fast quotient (the hardware reciprocal estimate refined by
 * two Newton-Raphson steps, within 1 ulp, for normal x of magnitude below
 * 2^1021; the IEEE division elsewhere); and (fn = 4) the guesses' cube root
 * (float cube root of the scaled mantissa, ~1e-7 relative, for positive
 * normal x; the library's FP64 cbrt elsewhere).
 *   in : x (n float64)   out: y (n float64)
 * Exposed so that they can be checked on their own; fn outside 0..4 is
 * PIVOT_E_OPTS.
 */
int pivot_elementary(int32_t fn, int64_t n, const double* x, double* y, void* stream);

/*
 * Training of the learned initial guess with the library's own kernels
 * (BF16 tensor-core forward and backward, FP32 accumulation).  The training
 * pairs are the operator's own: quotes (F, K, T, P, flag) and the sigma that
 * pivot_iv_forward returned for them; rows whose sigma is not finite and > 0
 * are skipped.  Loss: mean over the rows of (MLP(|x|, q) - ln(s / s_a))^2.
 *
 * pivot_mlp_init  -- parameters uniform in +-1/sqrt(fan_in) from `seed`
 *                    (counter-based), moments and gradient zeroed, BF16 copy written.
 * pivot_mlp_grad  -- adds d(sum of squared errors)/d(param) over n rows to
 *                    trainer->grad and the loss to trainer->loss_sum / rows.
 * pivot_mlp_adam  -- one Adam step on trainer->param with grad / rows (mean
 *                    loss), then zeroes grad, loss_sum and rows and refreshes
 *                    trainer->net.
 * The trainer must not be used by two calls that overlap on the GPU.
 */
int pivot_mlp_init(pivot_mlp_trainer* trainer, uint64_t seed, void* stream);
int pivot_mlp_grad(pivot_mlp_trainer* trainer, int64_t n, const double* F, const double* K,
                   const double* T, const double* P, const int8_t* flag, const double* sigma,
                   void* stream);
int pivot_mlp_adam(pivot_mlp_trainer* trainer, double lr, double beta1, double beta2, double eps,
                   void* stream);

/*
 * pivot_mlp_grad_static -- the gradient pass of pivot_mlp_grad without any
 * device allocation, for callers that cannot allocate device memory: code
 * that runs inside a host framework which owns every device buffer (a
 * cudaMalloc there would bypass its allocator and its memory budget), or
 * that works on a device whose memory is already fully handed out.  The paper
 * has no counterpart; it exists for deployment.
 *   in : net (the BF16 weights, e.g. &trainer->net), n rows of F, K, T, P
 *        (float64), flag (int8), sigma (float64) as for pivot_mlp_grad
 *   out: grad_out (PIVOT_MLP_NPARAM float32, the gradient of the sum of
 *        squared errors over the rows, in the flat parameter order),
 *        loss_out (2 float64: that sum, and the number of rows in it)
 * Scratch: the FP32 accumulator (PIVOT_MLP_NPARAM floats) and the two sums
 * live in one static device array of the library (34,328 bytes per device
 * that loads the library, held until the process exits).  Each call clears
 * it first and copies the result out; calls that overlap on the GPU (two
 * streams, two host threads) share the array and race.  n is limited to
 * 2^26 rows per call (FP32 sums over more rows lose their last digits):
 * larger n returns PIVOT_E_TOO_MANY and launches nothing.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.  The
 * address is kept for the life of the process: do not call this entry point
 * after a cudaDeviceReset of a device it has already been used on.
 */
int pivot_mlp_grad_static(const pivot_mlp* net, int64_t n, const double* F, const double* K,
                          const double* T, const double* P, const int8_t* flag, const double* sigma,
                          float* grad_out, double* loss_out, void* stream);

/* sizeof(pivot_mlp_trainer) and offsetof(pivot_mlp_trainer, net), for bindings. */
int64_t pivot_mlp_trainer_bytes(int64_t* net_offset);

/*
 * pivot_iv_guess -- the initial guess s^(0) alone (before any Householder
 * step), for measuring seeds against the root: opts NULL or PIVOT_MODE_FP64
 * gives LBR's four-region rational guess (appendix stage 4), PIVOT_MODE_LEARNED
 * the MLP seed.  Rows that need no solve get NaN.
 *   in : F, K, T, P (n float64), flag (n int8)   out: s_out (n float64)
 */
int pivot_iv_guess(int64_t n, const double* F, const double* K, const double* T, const double* P,
                   const int8_t* flag, const pivot_opts* opts, double* s_out, void* stream);

/*
 * Throughput probes (diagnostics; the paper has no counterpart).  The kernels
 * above are bound by the FP64 pipe, so their roofline fractions are stated
 * against measured unit rates as well as against unit counts x clocks.
 *
 * pivot_probe_units -- one launch of blocks_per_sm x (SM count) blocks of 256
 *   threads, each thread running 8 independent dependency chains for
 *   iters x 8 rounds of one operation:
 *     unit 0: FP64 fma (a = a b + c), 1: FP32 fma, 2: MUFU ex2.approx (float),
 *     3: MUFU tanh.approx (float).
 *   sink: device memory of 8 x (grid) bytes or more (written only if a chain
 *   reaches an impossible value); *lane_ops (HOST double) receives the number of
 *   lane operations the launch performs (an fma counts once: 2 FLOP).
 *   Errors: PIVOT_E_OPTS for unit outside 0..3, blocks_per_sm outside 1..32 or
 *   iters < 1; PIVOT_E_NULL for a NULL lane_ops.
 *
 * pivot_probe_stream -- the fused forward+backward's HBM traffic with no
 *   arithmetic: reads F, K, T, P (float64) and flag (int8), writes sigma = P,
 *   dP = F, dF = K, dK = T, dT = P (float64) and status = flag (uint8), 74 bytes
 *   per row, grid-stride over blocks_per_sm x (SM count) blocks of 256 threads.
 *   width 1: 64-bit accesses, one row per thread; width 2: 128-bit accesses of
 *   two consecutive rows per thread (every float64 array 16-byte aligned, the
 *   int8 arrays 2-byte aligned, else PIVOT_E_ALIGN).  All arrays required.
 */
int pivot_probe_units(int32_t unit, int32_t blocks_per_sm, int64_t iters, void* sink, double* lane_ops,
                      void* stream);
int pivot_probe_stream(int32_t width, int64_t n, const double* F, const double* K, const double* T,
                       const double* P, const int8_t* flag, double* sigma, uint8_t* status, double* dP,
                       double* dF, double* dK, double* dT, int32_t blocks_per_sm, void* stream);

/* Human-readable text for a return code. */
const char* pivot_error_string(int code);

/* ABI version (major * 10000 + minor * 100 + patch).  200: pivot_opts gained `counters`. */
int pivot_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PIVOT_H */

// pivot_capi.cu -- kernels and the extern "C" entry points declared in
// include/pivot.h (plain FP64 path).
//
// One row per thread: every step of Algorithm 1 (normalise, LBR boundary,
// rational guess, Householder(3) steps, denormalise, adjoint, gate) runs in
// registers between one coalesced read of the row and one write of its
// results, so a forward+backward touches HBM once per element (the fused
// design of Section 4.1, "Throughput and forward accuracy").
#include <cstdint>
#include <cuda_runtime.h>

#include "pivot.h"
#include "pivot_device.cuh"
#include "pivot_internal.cuh"

namespace {

using namespace pivot::detail;

__global__ void __launch_bounds__(kBlock) k_black_price(int64_t n, const double* __restrict__ F,
                                                        const double* __restrict__ K, const double* __restrict__ T,
                                                        const double* __restrict__ sigma,
                                                        const int8_t* __restrict__ flag, double* __restrict__ P,
                                                        double* __restrict__ V) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    double p, v;
    pivot::black_price_row(F[i], K[i], T[i], sigma[i], flag[i], p, v);
    P[i] = p;
    if (V) V[i] = v;
  }
}

__global__ void __launch_bounds__(kBlock) k_black_price_backward(
    int64_t n, const double* __restrict__ F, const double* __restrict__ K, const double* __restrict__ T,
    const double* __restrict__ sigma, const int8_t* __restrict__ flag, const double* __restrict__ gbar,
    double* __restrict__ dsigma, double* __restrict__ dF, double* __restrict__ dK, double* __restrict__ dT) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double g = gbar ? gbar[i] : 1.0;
    const pivot::PriceGrad d = pivot::black_price_vjp_row(F[i], K[i], T[i], sigma[i], flag[i], g);
    if (dsigma) dsigma[i] = d.dsigma;
    if (dF) dF[i] = d.dF;
    if (dK) dK[i] = d.dK;
    if (dT) dT[i] = d.dT;
  }
}

__global__ void __launch_bounds__(kBlock) k_elementary(int fn, int64_t n, const double* __restrict__ x,
                                                        double* __restrict__ y) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = fn == 0   ? pivot::log_fp64(x[i])
           : fn == 1 ? pivot::exp_fp64(x[i])
           : fn == 2 ? pivot::neg_ncdfinv<double>(x[i], true)
           : fn == 3 ? pivot::div_fast(1.0, x[i])
                     : pivot::Math<double>::cbrt_(x[i]);
}

__global__ void __launch_bounds__(kBlock) k_mills_ratio(int64_t n, const double* __restrict__ z,
                                                        double* __restrict__ y) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = pivot::mills_y<double>(z[i]);
}

__global__ void __launch_bounds__(kBlock) k_iv_backward(int64_t n, const double* __restrict__ F,
                                                        const double* __restrict__ K, const double* __restrict__ T,
                                                        const int8_t* __restrict__ flag,
                                                        const double* __restrict__ sigma,
                                                        const double* __restrict__ gbar, double tau, int mode,
                                                        double* __restrict__ dP, double* __restrict__ dF,
                                                        double* __restrict__ dK, double* __restrict__ dT) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double g = gbar ? gbar[i] : 1.0;
    const pivot::Grad d = pivot::gated_adjoint(F[i], K[i], T[i], flag[i], sigma[i], g, tau, mode);
    if (dP) dP[i] = d.dP;
    if (dF) dF[i] = d.dF;
    if (dK) dK[i] = d.dK;
    if (dT) dT[i] = d.dT;
  }
}

// Black-Scholes price on xi = (S, K, tau, r, q): e^{-r tau} B(S e^{(r-q) tau}, K, tau, sigma)
// (Eq. app_black_scholes in forward coordinates, Eq. app_black76), and the cash vega.
__global__ void __launch_bounds__(kBlock) k_bs_price(int64_t n, const double* __restrict__ S,
                                                     const double* __restrict__ K, const double* __restrict__ T,
                                                     const double* __restrict__ r, const double* __restrict__ q,
                                                     const double* __restrict__ sigma,
                                                     const int8_t* __restrict__ flag, double* __restrict__ V,
                                                     double* __restrict__ vega) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    double er, ec, p, v;
    const double tau = T[i], rr = r[i];
    pivot::bs_factors(tau, rr, q[i], er, ec);
    pivot::black_price_row(S[i] * ec, K[i], tau, sigma[i], flag[i], p, v);
    const double disc = exp(-rr * tau);
    V[i] = disc * p;
    if (vega) vega[i] = disc * v;
  }
}

__global__ void __launch_bounds__(kBlock) k_bs_iv_backward(Args a) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    double er, ec;
    const double tau = a.T[i], rr = a.r[i], qq = a.q[i];
    pivot::bs_factors(tau, rr, qq, er, ec);
    write_grad_bs(a, i, a.F[i] * ec, a.K[i], tau, a.flag[i], a.sigma[i], rr, qq, er, ec);
  }
}

// ---------------------------------------------------------------------------
// Forward (and fused forward+backward) with per-tile compaction and region
// binning.  The input is cut into chunks of kThreads consecutive rows, dealt to
// the persistent blocks in grid-stride order.  A block's tile is a set of solve
// slots (kCap), filled from as many chunks as they can take:
//  phase 1: passes of up to kCap/kThreads chunks, one row per thread and chunk
//           (coalesced loads), with the cheap stage-1 tests; rows that need no
//           solve (invalid, or at a bound of the price interval) are finished
//           at once, the others take the next free slot (one warp-aggregated
//           atomic) with their time value and its complement.  Passes go on
//           while the free slots can hold one more chunk whatever it holds,
//           so a batch where most rows end in stage 1 still fills the tile.
//  phase 2: the slots are consumed densely: normalisation, LBR boundary node
//           and region of each row, kept in shared memory, counted per region.
//  phase 3: the rows are laid out region after region and consumed in that
//           order, so a warp runs one region's guess and Householder
//           objective with all of its lanes.  Each bin is consumed in whole
//           warps: its last, partial warp of rows (with their nodes) is carried
//           to the block's next tile and joins that tile's bin in front, so
//           that no warp runs with idle lanes or two regions' code, except in
//           the block's last tile, which takes every row.  sigma and the gated
//           adjoint are written here.
// ---------------------------------------------------------------------------
// Region bins.  FP64 form: the 4 regions, plus bins 4, 5 for middle-region
// rows and bin 7 for lower-region rows near the money (|x| <= kTaylorX), the
// only rows whose b may take the Taylor series of rho: kept apart, a warp runs
// one of the two forms of rho (and, in the adjoint, one form of the Mills
// ratios); and bin 6 for lower-region rows with beta below kDeepBeta, whose
// guess takes the scaled cube root and, below ~1e-290, ln beta from the
// row's time value.
// Mixed form: 4 float-seeded region bins, 4 FP64 bins for rows outside the
// float range (b_max - beta below kMixedFloor, |x| above kMixedMaxAbsX, or
// beta below kMixedFloor near the money), bin kDeepBin (lower-tail rows with
// beta below kMixedFloor and |x| >= kDeepMinAbsX, seeded in float from
// ln beta), and 3 near-the-money float bins (middle 9, 10; lower 11).
constexpr int kMaxBins = 12;
// Rows a bin may carry from one tile to the next (its last, partial warp).
constexpr int kCarryPerBin = 31;
// Chunks one tile may draw from (bounds the table of their first rows).
constexpr int kMaxChunks = 32;

// Shared memory of the binned kernel, in row slots: kCarry slots hold the
// rows carried over from earlier tiles (bin b in [31 b, 31 b + 31)), then
// kCap slots the current tile's solved rows.  Per slot: six node fields
// (+ e^{r tau}, e^{(r-q) tau} in the Black-Scholes form) and the phase-3
// order; per tile slot: the row's chunk and lane (a 16-bit code); per carry
// slot: the row's global index and a move record.  Slots per tile: 1,792 for
// the FP64 Black-76 form, 1,536 for its mixed form (12 bins), 1,280 / 1,024
// for the Black-Scholes forms, so that 2 blocks of 256 threads fit an SM
// (~128 registers a thread).
template <bool kBS, bool kMixed>
struct TileCfg {
  static constexpr int kBins = kMixed ? 12 : 8;
  static constexpr int kCarry = kCarryPerBin * kBins;
  static constexpr int kThreads = 256;  // also the rows of a chunk
  static constexpr int kMinBlocks = 2;
  static constexpr int kCap = kBS ? (kMixed ? 1024 : 1280) : (kMixed ? 1536 : 1792);
  static constexpr int kMaxPass = kCap / kThreads;                 // chunks per phase-1 pass
  static constexpr int kRows2 = (kCap + kThreads - 1) / kThreads;  // slots per thread in phase 2
  static constexpr int kSlots = kCarry + kCap;
  static constexpr size_t kSmem = size_t(kBS ? 8 : 6) * kSlots * sizeof(double) + size_t(kCarry) * sizeof(int64_t) +
                                  size_t(kSlots) * sizeof(uint16_t) + size_t(kCap) * sizeof(uint16_t) +
                                  2 * size_t(kCarry) * sizeof(uint16_t);
};
constexpr int kDeepBin = 8;
constexpr double kMixedFloor = 1e-30;
constexpr double kMixedMaxAbsX = 80.0;
constexpr double kDeepMinAbsX = 0.1;

// Row inputs in forward coordinates.  The Black-Scholes form (kBS) reads the
// spot S from a.F and the discounted price V from a.P and maps them with the
// factors phase 1 left in shared memory; the products are the same in every
// phase, so all phases see one F and one B.
template <bool kBS>
__device__ __forceinline__ void row_fp(const Args& a, int64_t i, int r, const double* s_er, const double* s_ec,
                                       double& F, double& P) {
  if (kBS) {
    F = a.F[i] * s_ec[r];
    P = a.P[i] * s_er[r];
  } else {
    F = a.F[i];
    P = a.P[i];
  }
}

// kSmall: chunks of a.chunk_rows < kThreads rows, so that a small batch spreads over more
// blocks; a separate instantiation with its own argument type, so that the full-chunk kernels
// of large batches keep their code and their parameters
struct ArgsChunked : Args {
  int chunk_rows; // 32..kThreads, a multiple of 32
};
template <bool kSmall>
struct BinnedArgs {
  using type = Args;
};
template <>
struct BinnedArgs<true> {
  using type = ArgsChunked;
};
__device__ __forceinline__ int chunk_rows_of(const Args&, int full) { return full; }
__device__ __forceinline__ int chunk_rows_of(const ArgsChunked& a, int) { return a.chunk_rows; }

template <bool kBackward, bool kMixed, bool kBS, bool kSmall = false>
__global__ void __launch_bounds__(TileCfg<kBS, kMixed>::kThreads, TileCfg<kBS, kMixed>::kMinBlocks)
    k_iv_binned(typename BinnedArgs<kSmall>::type a) {
  using Cfg = TileCfg<kBS, kMixed>;
  constexpr int kThreads = Cfg::kThreads;
  constexpr int kMaxPass = Cfg::kMaxPass;
  constexpr int kRows2 = Cfg::kRows2;
  constexpr int kCap = Cfg::kCap;
  constexpr int kBins = Cfg::kBins;
  constexpr int kCarry = Cfg::kCarry;
  constexpr int kSlots = Cfg::kSlots;
  // per row slot (carry slots first, then the tile's): its node, in structure-of-arrays form
  extern __shared__ double smem[];
  double* s_x = smem;
  double* s_rsq = s_x + kSlots;   // 1/sqrt(F K); b_max = min(F, K) rsq is formed from it
  double* s_e = s_rsq + kSlots;
  double* s_bn = s_e + kSlots;
  double* s_bsn = s_bn + kSlots;
  double* s_bb = s_bsn + kSlots;
  double* s_er = s_bb + kSlots;                      // kBS only
  double* s_ec = s_er + (kBS ? kSlots : 0);          // kBS only
  int64_t* s_gidx = reinterpret_cast<int64_t*>(s_ec + (kBS ? kSlots : 0));  // global row of a carry slot
  uint16_t* s_order = reinterpret_cast<uint16_t*>(s_gidx + kCarry);         // phase 2 -> 3: slots in bin order
  uint16_t* s_code = s_order + kSlots;    // tile slot -> (chunk of the tile << 8) | row in the chunk
  uint16_t* s_mv_src = s_code + kCap;     // leftover rows: tile slot ...
  uint16_t* s_mv_dst = s_mv_src + kCarry; // ... -> carry slot
  __shared__ int64_t s_cbase[kMaxChunks];  // first row of each chunk of the tile
  __shared__ int s_nsolve, s_nmv;
  __shared__ int s_cnt[kMaxBins];   // rows per bin, carried ones included
  __shared__ int s_full[kMaxBins];  // rows per bin consumed by this tile
  __shared__ int s_ccnt[kMaxBins];  // rows per bin carried into the next tile
  __shared__ int s_off[kMaxBins + 1];
  __shared__ unsigned long long s_count[PIVOT_COUNTERS_LEN];  // a.counters: this block's sums

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const bool counting = a.counters != nullptr;
  if (counting && tid < PIVOT_COUNTERS_LEN) s_count[tid] = 0;
  // global row of a slot
  auto row_of = [&](int r) -> int64_t {
    if (r < kCarry) return s_gidx[r];
    const int c = s_code[r - kCarry];
    return s_cbase[c >> 8] + (c & 0xff);
  };
  // rows per chunk: kThreads, or fewer (a multiple of 32) on a batch too small to give every
  // resident block a full chunk; threads at or beyond it take no row in phase 1
  const int crows = chunk_rows_of(a, kThreads);
  const bool has_row = !kSmall || tid < crows;
  const int64_t nchunks = (a.n + crows - 1) / crows;
  int64_t cursor = blockIdx.x;  // this block's next chunk
  if (tid < kBins) s_ccnt[tid] = 0;
  while (cursor < nchunks) {
    if (tid < kBins) s_cnt[tid] = s_ccnt[tid];  // carried rows come first in their bins
    if (tid == 0) {
      s_nsolve = 0;
      s_nmv = 0;
    }
    __syncthreads();
    // ---- phase 1: passes over this block's next chunks while the free slots can take them
    int nsolve = 0, nch = 0;
    while (cursor < nchunks) {
      int take = (kCap - nsolve) / kThreads;
      if (take > kMaxChunks - nch) take = kMaxChunks - nch;
      // a pass costs a round trip to memory and two barriers: none for a single chunk once the
      // tile holds rows (mixed stress 3.00 -> 2.97 ms)
      if (take < 2 && nch > 0) break;
      // the pass's loads first, all in flight at once: the stores of one row's outputs would
      // otherwise keep the next row's loads behind them (the output arrays may alias the inputs
      // as far as the compiler knows), one memory round trip per chunk instead of per pass
      double rF[kMaxPass], rK[kMaxPass], rT[kMaxPass], rP[kMaxPass], rr[kBS ? kMaxPass : 1], rq[kBS ? kMaxPass : 1];
      int rfl[kMaxPass];
#pragma unroll
      for (int j = 0; j < kMaxPass; ++j) {
        const int64_t i = has_row ? (cursor + int64_t(j) * gridDim.x) * crows + tid : a.n;
        rF[j] = rK[j] = rT[j] = rP[j] = 0.0;
        rfl[j] = 0;
        if (kBS) rr[kBS ? j : 0] = rq[kBS ? j : 0] = 0.0;
        if (j < take && i < a.n) {
          rF[j] = a.F[i];
          rK[j] = a.K[i];
          rT[j] = a.T[i];
          rP[j] = a.P[i];
          rfl[j] = a.flag[i];
          if (kBS) {
            rr[kBS ? j : 0] = a.r[i];
            rq[kBS ? j : 0] = a.q[i];
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kMaxPass; ++j) {
        if (j >= take) break;  // uniform over the block
        const int64_t c = cursor + int64_t(j) * gridDim.x;
        const int64_t i = has_row ? c * crows + tid : a.n;
        if (tid == 0 && c < nchunks) s_cbase[nch + j] = c * crows;
        bool solve = false;
        int row_status = -1;
        double tv = 0.0, cv = 0.0, er = 1.0, ec = 1.0, Fs = 0.0, Ks = 0.0;
        if (i < a.n) {
          const double K = rK[j], T = rT[j];
          double F = rF[j], P = rP[j];
          if (kBS) {
            pivot::bs_factors(T, rr[kBS ? j : 0], rq[kBS ? j : 0], er, ec);
            F *= ec;
            P *= er;
          }
          const int fl = rfl[j];
          const pivot::Quote q = pivot::classify_quote(F, K, T, P, fl);
          row_status = q.status;
          // every row's status here, in row order (a solved row's stays 0): one coalesced byte
          if (a.status) a.status[i] = uint8_t(q.status);
          if (q.status != 0) {
            a.sigma[i] = q.sigma;
            if (kBackward) {
              // outside the open price interval, or invalid: the degenerate gradient of its status
              const double g = a.gbar ? a.gbar[i] : 1.0;
              const double v = pivot::degenerate_grad(q.status <= 3 || pivot::nan64(g), g, a.mode).dP;
              if (a.dP) a.dP[i] = v;
              if (a.dF) a.dF[i] = v;
              if (a.dK) a.dK[i] = v;
              if (a.dT) a.dT[i] = v;
              if (kBS) {
                if (a.dr) a.dr[i] = v;
                if (a.dq) a.dq[i] = v;
              }
            }
          } else {
            solve = true;
            tv = q.tv;
            cv = q.cv;
            Fs = F;
            Ks = K;
          }
        }
        const int r = kCarry + warp_append(solve, &s_nsolve, lane);
        if (solve) {
          // the time value and its complement, and F and K in the slots phase 2 fills from them
          s_bb[r] = tv;
          s_e[r] = cv;
          s_x[r] = Fs;
          s_rsq[r] = Ks;
          s_code[r - kCarry] = uint16_t(((nch + j) << 8) | tid);
          if (kBS) {
            s_er[r] = er;
            s_ec[r] = ec;
          }
        }
        if (counting) {
#pragma unroll
          for (int k = 1; k < 6; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, row_status == k);
            if (lane == 0 && m) atomicAdd(&s_count[k], (unsigned long long)__popc(m));
          }
        }
      }
      cursor += int64_t(take) * gridDim.x;
      nch += take;
      __syncthreads();
      nsolve = s_nsolve;
      __syncthreads();  // every thread has read the count before the next pass adds to it
    }
    const bool last = cursor >= nchunks;  // the block's last tile takes every row
    // ---- phase 2
    int reg[kRows2], pos[kRows2], row[kRows2];
#pragma unroll
    for (int j = 0; j < kRows2; ++j) {
      const int qi = j * kThreads + tid;
      int rg = -1;
      row[j] = 0;
      if (qi < nsolve) {
        const int r = kCarry + qi;
        const double F = s_x[r], K = s_rsq[r];  // left by phase 1 (forward F in the Black-Scholes form)
        double x, bmax, rsq;
        pivot::moneyness(F, K, x, bmax, rsq);
        const double beta = s_bb[r] * rsq, betac = s_e[r] * rsq;
        s_rsq[r] = rsq;
        bool fp64_row = true;
        // range tests on bit patterns (beta, beta_c and -x are non-negative): integer instructions
        const bool beta_f = pivot::gt_pos(beta, kMixedFloor), betac_f = pivot::gt_pos(betac, kMixedFloor);
        const bool x_f = pivot::gt_pos(kMixedMaxAbsX, -x);
        if (kMixed && !beta_f && betac_f && x_f && !pivot::gt_pos(kDeepMinAbsX, -x) &&
            pivot::pos_normal(beta)) {
          // deep lower tail: beta below the float range but ln beta is not (at |x| >= 0.1 such a
          // beta lies below b_l, in the lower region)
          fp64_row = false;
          rg = kDeepBin;
          s_x[r] = x;
          s_bb[r] = beta;
        } else if (kMixed && beta_f && betac_f && x_f) {
          // float node and region; the float copies are exact in double storage
          pivot::Node<float> nf;
          rg = pivot::classify<float>(float(x), float(bmax), float(beta), float(betac), nf);
          if (nf.bsn > 0.0f && nf.bn >= 0.0f) {
            fp64_row = false;
            // x, b_max and beta (or beta_c) in double for the final FP64 step and the
            // adjoint; the float node packed two floats to a slot (no conversions)
            s_x[r] = x;
            s_bb[r] = (rg == pivot::kUpper) ? betac : beta;
            *reinterpret_cast<float2*>(&s_e[r]) = make_float2(nf.e, nf.bn);
            *reinterpret_cast<float2*>(&s_bn[r]) = make_float2(nf.bsn, nf.x);
            *reinterpret_cast<float2*>(&s_bsn[r]) = make_float2(nf.bmax, nf.bb);
          }
        }
        if (fp64_row) {
          pivot::Node<double> nd;
          rg = pivot::classify<double>(x, bmax, beta, betac, nd) + (kMixed ? 4 : 0);
          s_x[r] = nd.x;
          s_e[r] = nd.e;
          s_bn[r] = nd.bn;
          s_bsn[r] = nd.bsn;
          s_bb[r] = nd.bb;
        }
        // lower and middle rows near the money to their own bins (FP64 form: 0, 1, 2 -> 7, 4, 5;
        // mixed float: 0, 1, 2 -> 11, 9, 10)
        if (pivot::le_pos(-x, pivot::kTaylorX)) {
          if (!kMixed && (rg == pivot::kMidLow || rg == pivot::kMidHigh)) rg += 3;
          else if (!kMixed && rg == pivot::kLower) rg = 7;
          if (kMixed && !fp64_row && (rg == pivot::kMidLow || rg == pivot::kMidHigh)) rg += 8;
          else if (kMixed && !fp64_row && rg == pivot::kLower) rg = 11;
        }
        if (!kMixed && (rg == pivot::kLower || rg == 7) && pivot::gt_pos(pivot::kDeepBeta, beta)) rg = 6;
        row[j] = r;
      }
      reg[j] = rg;
      pos[j] = 0;
#pragma unroll
      for (int k = 0; k < kBins; ++k) {
        const int p = warp_append(rg == k, &s_cnt[k], lane);
        if (rg == k) pos[j] = p;
      }
    }
    __syncthreads();
    if (tid == 0) {
      s_off[0] = 0;
      for (int k = 0; k < kBins; ++k) {
        const int full = last ? s_cnt[k] : (s_cnt[k] & ~31);
        s_full[k] = full;
        s_off[k + 1] = s_off[k] + full;
      }
      if (counting) {
        s_count[0] += nsolve;
        for (int k = 0; k < kBins; ++k) s_count[kCountBin0 + k] += s_full[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRows2; ++j) {
      const int b = reg[j];
      if (b >= 0) {
        const int p = pos[j], full = s_full[b];
        if (p < full) {
          s_order[s_off[b] + p] = uint16_t(row[j]);
        } else {
          // the bin's partial warp: to carry slot p - full of the bin (p - full <= 30)
          const int m = atomicAdd(&s_nmv, 1);
          s_mv_src[m] = uint16_t(row[j]);
          s_mv_dst[m] = uint16_t(kCarryPerBin * b + p - full);
        }
      }
    }
    // carried rows hold the first positions of their bins; those not consumed stay in place
    for (int c = tid; c < kCarry; c += kThreads) {
      const int b = c / kCarryPerBin, p = c - b * kCarryPerBin;
      if (p < s_ccnt[b] && p < s_full[b]) s_order[s_off[b] + p] = uint16_t(c);
    }
    __syncthreads();
    // ---- phase 3
    const int total = s_off[kBins];
    const int nmv = s_nmv;  // final since the barrier above; the next tile resets it
    for (int qi = tid; qi < total; qi += kThreads) {
      const int r = s_order[qi];  // slot
      int bin = 0;
#pragma unroll
      for (int k = 1; k < kBins; ++k) bin += (qi >= s_off[k]) ? 1 : 0;
      const int64_t i = row_of(r);
      const double K = a.K[i], T = a.T[i];
      double F, P;
      row_fp<kBS>(a, i, r, s_er, s_ec, F, P);
      const int fl = a.flag[i];
      const bool deep = kMixed && bin == kDeepBin;
      const int rg = kMixed ? (deep || bin == 11 ? int(pivot::kLower) : bin > kDeepBin ? bin - 8 : (bin & 3))
                            : (bin < 4 ? bin : bin >= 6 ? int(pivot::kLower) : bin - 3);
      const bool float_row = kMixed && (bin < 4 || bin >= kDeepBin);
      const double bb = s_bb[r];
      const double rsq = s_rsq[r];
      const double bmax = pivot::bmax_of(F, K, rsq);
      double s = 0.0;
      pivot::Last last;
      // FP64 bins, and float-seeded rows whose float solve was not accepted, meet at one FP64 solve
      bool fp64 = !float_row;
      if (float_row) {
        if (deep) {
          s = pivot::solve_deep_mixed64(s_x[r], bmax, bb, last);
        } else {
          pivot::Node<float> nf;
          const float2 p0 = *reinterpret_cast<const float2*>(&s_e[r]);
          const float2 p1 = *reinterpret_cast<const float2*>(&s_bn[r]);
          const float2 p2 = *reinterpret_cast<const float2*>(&s_bsn[r]);
          nf.e = p0.x;
          nf.bn = p0.y;
          nf.bsn = p1.x;
          nf.x = p1.y;
          nf.bmax = p2.x;
          nf.bb = p2.y;
          s = pivot::solve_mixed64(rg, nf, s_x[r], bmax, bb, a.steps, last);
        }
        fp64 = !pivot::pos_finite(s);
        if (counting && fp64) atomicAdd(&s_count[kCountReject], 1ull);
      }
      if (fp64) {
        pivot::Node<double> nd;
        int rg64 = rg;
        if (float_row) {
          // not accepted: the FP64 node from the row's inputs (its shared slots hold the float node)
          const pivot::Quote q = pivot::classify_quote(F, K, T, P, fl);
          double x, bmax_w, rsq_w;
          pivot::moneyness(F, K, x, bmax_w, rsq_w);
          rg64 = pivot::classify<double>(x, bmax_w, q.tv * rsq_w, q.cv * rsq_w, nd);
        } else {
          nd.x = s_x[r];
          nd.bmax = bmax;
          nd.e = s_e[r];
          nd.bn = s_bn[r];
          nd.bsn = s_bsn[r];
          nd.bb = bb;
        }
        // ln beta for the lower region's objective
        const double lnbeta = (rg64 == pivot::kLower) ? pivot::log_beta(nd.bb, F, K, T, P, fl) : 0.0;
        // (the mixed form's FP64 rows lie mostly below the float range: the library's Phi^{-1})
        s = pivot::solve64<!kMixed>(rg64, nd, lnbeta, a.steps, last);
      }
      const double inv_sqT = rsqrt(T);
      const double sig = s * inv_sqT;
      a.sigma[i] = sig;
      if (kBackward) {
        // the adjoint at the solved s, reusing x and 1/sqrt(T) of this row
        const double g = a.gbar ? a.gbar[i] : 1.0;
        const double gate_tau = kBS ? a.tau * s_er[r] : a.tau;  // G_tau on the cash vega e^{-r tau} V
        // (no gbar: the same launch-uniform branch on every row, and no products by 1)
        const pivot::Grad d =
            pivot::nan64(g) ? pivot::degenerate_grad(true, g, a.mode)
            : a.gbar ? pivot::adjoint_reuse<false>(F, K, fl, sig, s, s_x[r], bmax, inv_sqT, rsq, g, gate_tau, a.mode,
                                                   last)
                     : pivot::adjoint_reuse<true>(F, K, fl, sig, s, s_x[r], bmax, inv_sqT, rsq, g, gate_tau, a.mode,
                                                  last);
        if (kBS) {
          const pivot::BSGrad o = pivot::bs_grad(d, F, K, T, a.r[i], a.q[i], s_er[r], s_ec[r]);
          if (a.dP) a.dP[i] = o.dV;
          if (a.dF) a.dF[i] = o.dS;
          if (a.dK) a.dK[i] = o.dK;
          if (a.dT) a.dT[i] = o.dT;
          if (a.dr) a.dr[i] = o.dr;
          if (a.dq) a.dq[i] = o.dq;
        } else {
          if (a.dP) a.dP[i] = d.dP;
          if (a.dF) a.dF[i] = d.dF;
          if (a.dK) a.dK[i] = d.dK;
          if (a.dT) a.dT[i] = d.dT;
        }
      }
    }
    __syncthreads();
    // the partial warps' rows to their carry slots, now that phase 3 has read the slots they
    // take; the next tile's first barrier orders these copies before its phase 1
    for (int m = tid; m < nmv; m += kThreads) {
      const int src = s_mv_src[m], dst = s_mv_dst[m];
      s_x[dst] = s_x[src];
      s_rsq[dst] = s_rsq[src];
      s_e[dst] = s_e[src];
      s_bn[dst] = s_bn[src];
      s_bsn[dst] = s_bsn[src];
      s_bb[dst] = s_bb[src];
      if (kBS) {
        s_er[dst] = s_er[src];
        s_ec[dst] = s_ec[src];
      }
      s_gidx[dst] = row_of(src);
    }
    if (tid < kBins) s_ccnt[tid] = s_cnt[tid] - s_full[tid];
  }
  if (counting) {
    __syncthreads();
    if (tid < PIVOT_COUNTERS_LEN && s_count[tid]) atomicAdd(&a.counters[tid], s_count[tid]);
  }
}

int check_opts(const pivot_opts* o, int* steps, int* mode) {
  *steps = kDefaultSteps;
  *mode = PIVOT_MODE_FP64;
  if (o == nullptr) return PIVOT_OK;
  if (o->mode != PIVOT_MODE_FP64 && o->mode != PIVOT_MODE_MIXED && o->mode != PIVOT_MODE_LEARNED)
    return PIVOT_E_OPTS;
  if (o->householder < 0 || o->householder > 4) return PIVOT_E_OPTS;
  if (o->mode == PIVOT_MODE_LEARNED) {
    if (o->mlp == nullptr) return PIVOT_E_MLP;
    if (!(o->fallback >= 0.0) || !(o->fallback < 1.0)) return PIVOT_E_MLP;
  }
  if (o->householder > 0) *steps = o->householder;
  *mode = o->mode;
  return PIVOT_OK;
}

// persistent grid for the binned kernels: resident blocks x SMs, capped by the chunks
template <bool kBackward, bool kMixed, bool kBS, bool kSmall>
int launch_binned_as(const Args& a, int64_t crows, void* stream) {
  // occupancy of this instantiation, looked up once per device
  static thread_local int configured_device = -1;
  static thread_local int64_t cap = 0;
  constexpr size_t smem = TileCfg<kBS, kMixed>::kSmem;
  constexpr int kThreads = TileCfg<kBS, kMixed>::kThreads;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return launch_status();
  if (configured_device != dev) {
    const void* f = reinterpret_cast<const void*>(k_iv_binned<kBackward, kMixed, kBS, kSmall>);
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int b = 0, num_sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kThreads, smem);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    cap = int64_t(b < 1 ? 1 : b) * num_sms;
    configured_device = dev;
  }
  if (crows <= 0) {
    // rows per chunk: a full block's worth, or on a small batch the multiple of 32 that spreads
    // it over up to every resident block (a 4,096-row batch: 128 blocks of 32 rows, not 16 of 256)
    crows = (a.n + cap - 1) / cap;
    crows = ((crows + 31) / 32) * 32;
    if (crows > kThreads) crows = kThreads;
    if (crows < 32) crows = 32;
    if (crows < kThreads) return launch_binned_as<kBackward, kMixed, kBS, true>(a, crows, stream);
  }
  const int64_t chunks = (a.n + crows - 1) / crows;  // every block gets at least one
  const unsigned grid = unsigned(chunks < cap ? chunks : cap);
  if (kSmall) {
    ArgsChunked b;
    static_cast<Args&>(b) = a;
    b.chunk_rows = int(crows);
    k_iv_binned<kBackward, kMixed, kBS, true><<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(b);
  } else {
    k_iv_binned<kBackward, kMixed, kBS, false><<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
  }
  return launch_status();
}
template <bool kBackward, bool kMixed, bool kBS = false>
int launch_binned(const Args& a, void* stream) {
  return launch_binned_as<kBackward, kMixed, kBS, false>(a, 0, stream);
}

}  // namespace

extern "C" {

int pivot_black_price(int64_t n, const double* F, const double* K, const double* T, const double* sigma,
                      const int8_t* flag, double* P_out, double* vega_out, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true},     {K, true, true},     {T, true, true},       {sigma, true, true},
                    {flag, true, false}, {P_out, true, true}, {vega_out, false, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_black_price<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, F, K, T, sigma, flag, P_out,
                                                                                  vega_out);
  return launch_status();
}

int pivot_black_price_backward(int64_t n, const double* F, const double* K, const double* T,
                               const double* sigma, const int8_t* flag, const double* gbar, double* dsigma,
                               double* dF, double* dK, double* dT, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true},        {K, true, true},      {T, true, true},  {sigma, true, true},
                    {flag, true, false},    {gbar, false, true},  {dsigma, false, true}, {dF, false, true},
                    {dK, false, true},      {dT, false, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_black_price_backward<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, F, K, T, sigma, flag,
                                                                                           gbar, dsigma, dF, dK, dT);
  return launch_status();
}

int pivot_iv_forward(int64_t n, const double* F, const double* K, const double* T, const double* P,
                     const int8_t* flag, double* sigma_out, uint8_t* status_out, const pivot_opts* opts,
                     void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  int steps, mode;
  int rc = check_opts(opts, &steps, &mode);
  if (rc != PIVOT_OK) return rc;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true},         {K, true, true},           {T, true, true},
                    {P, true, true},         {flag, true, false},       {sigma_out, true, true},
                    {status_out, false, false}};
  rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  Args a{n, F, K, T, P, flag, nullptr, 0.0, 0, steps, sigma_out, status_out, nullptr, nullptr, nullptr, nullptr};
  rc = check_counters(opts, dev, &a.counters);
  if (rc != PIVOT_OK) return rc;
  if (mode == PIVOT_MODE_LEARNED) {
    int d2 = dev;
    rc = check_ptr(opts->mlp, true, true, &d2);
    if (rc != PIVOT_OK) return rc;
    return launch_learned(a, opts->mlp, opts->fallback, false, stream);
  }
  return mode == PIVOT_MODE_MIXED ? launch_binned<false, true>(a, stream) : launch_binned<false, false>(a, stream);
}

int pivot_iv_backward(int64_t n, const double* F, const double* K, const double* T, const int8_t* flag,
                      const double* sigma, const double* gbar, double tau, int32_t gate_mode, double* dP,
                      double* dF, double* dK, double* dT, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  int rc = check_gate(tau, gate_mode);
  if (rc != PIVOT_OK) return rc;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true},      {K, true, true},   {T, true, true},   {flag, true, false},
                    {sigma, true, true},  {gbar, false, true}, {dP, false, true}, {dF, false, true},
                    {dK, false, true},    {dT, false, true}};
  rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_iv_backward<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, F, K, T, flag, sigma, gbar, tau,
                                                                                  gate_mode, dP, dF, dK, dT);
  return launch_status();
}

int pivot_iv_forward_backward(int64_t n, const double* F, const double* K, const double* T, const double* P,
                              const int8_t* flag, const double* gbar, double tau, int32_t gate_mode,
                              double* sigma_out, uint8_t* status_out, double* dP, double* dF, double* dK,
                              double* dT, const pivot_opts* opts, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  int steps, mode;
  int rc = check_opts(opts, &steps, &mode);
  if (rc == PIVOT_OK) rc = check_gate(tau, gate_mode);
  if (rc != PIVOT_OK) return rc;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true},         {K, true, true},       {T, true, true},    {P, true, true},
                    {flag, true, false},     {gbar, false, true},   {sigma_out, true, true},
                    {status_out, false, false}, {dP, false, true},  {dF, false, true},  {dK, false, true},
                    {dT, false, true}};
  rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  Args a{n, F, K, T, P, flag, gbar, tau, gate_mode, steps, sigma_out, status_out, dP, dF, dK, dT};
  rc = check_counters(opts, dev, &a.counters);
  if (rc != PIVOT_OK) return rc;
  if (mode == PIVOT_MODE_LEARNED) {
    int d2 = dev;
    rc = check_ptr(opts->mlp, true, true, &d2);
    if (rc != PIVOT_OK) return rc;
    return launch_learned(a, opts->mlp, opts->fallback, true, stream);
  }
  return mode == PIVOT_MODE_MIXED ? launch_binned<true, true>(a, stream) : launch_binned<true, false>(a, stream);
}

// ---- Black-Scholes interface on xi = (S, K, tau, r, q) ----------------------------------------

int pivot_bs_price(int64_t n, const double* S, const double* K, const double* T, const double* r,
                   const double* q, const double* sigma, const int8_t* flag, double* V_out, double* vega_out,
                   void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{S, true, true},      {K, true, true},         {T, true, true},         {r, true, true},
                    {q, true, true},      {sigma, true, true},     {flag, true, false},     {V_out, true, true},
                    {vega_out, false, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_bs_price<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, S, K, T, r, q, sigma, flag, V_out,
                                                                               vega_out);
  return launch_status();
}

int pivot_bs_iv_forward(int64_t n, const double* S, const double* K, const double* T, const double* r,
                        const double* q, const double* V, const int8_t* flag, double* sigma_out,
                        uint8_t* status_out, const pivot_opts* opts, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  int steps, mode;
  int rc = check_opts(opts, &steps, &mode);
  if (rc != PIVOT_OK) return rc;
  if (mode == PIVOT_MODE_LEARNED) return PIVOT_E_OPTS;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{S, true, true},    {K, true, true},         {T, true, true},          {r, true, true},
                    {q, true, true},    {V, true, true},         {flag, true, false},      {sigma_out, true, true},
                    {status_out, false, false}};
  rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  Args a{n, S, K, T, V, flag, nullptr, 0.0, 0, steps, sigma_out, status_out, nullptr, nullptr, nullptr, nullptr,
         r, q, nullptr, nullptr};
  rc = check_counters(opts, dev, &a.counters);
  if (rc != PIVOT_OK) return rc;
  return mode == PIVOT_MODE_MIXED ? launch_binned<false, true, true>(a, stream)
                                  : launch_binned<false, false, true>(a, stream);
}

int pivot_bs_iv_backward(int64_t n, const double* S, const double* K, const double* T, const double* r,
                         const double* q, const int8_t* flag, const double* sigma, const double* gbar, double tau,
                         int32_t gate_mode, double* dV, double* dS, double* dK, double* dT, double* dr, double* dq,
                         void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  int rc = check_gate(tau, gate_mode);
  if (rc != PIVOT_OK) return rc;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{S, true, true},      {K, true, true},     {T, true, true},     {r, true, true},
                    {q, true, true},      {flag, true, false}, {sigma, true, true}, {gbar, false, true},
                    {dV, false, true},    {dS, false, true},   {dK, false, true},   {dT, false, true},
                    {dr, false, true},    {dq, false, true}};
  rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  Args a{n, S, K, T, nullptr, flag, gbar, tau, gate_mode, 0, const_cast<double*>(sigma), nullptr, dV, dS, dK, dT,
         r, q, dr, dq};
  k_bs_iv_backward<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return launch_status();
}

int pivot_bs_iv_forward_backward(int64_t n, const double* S, const double* K, const double* T, const double* r,
                                 const double* q, const double* V, const int8_t* flag, const double* gbar,
                                 double tau, int32_t gate_mode, double* sigma_out, uint8_t* status_out, double* dV,
                                 double* dS, double* dK, double* dT, double* dr, double* dq,
                                 const pivot_opts* opts, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  int steps, mode;
  int rc = check_opts(opts, &steps, &mode);
  if (rc == PIVOT_OK) rc = check_gate(tau, gate_mode);
  if (rc != PIVOT_OK) return rc;
  if (mode == PIVOT_MODE_LEARNED) return PIVOT_E_OPTS;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{S, true, true},         {K, true, true},       {T, true, true},      {r, true, true},
                    {q, true, true},         {V, true, true},       {flag, true, false},  {gbar, false, true},
                    {sigma_out, true, true}, {status_out, false, false}, {dV, false, true}, {dS, false, true},
                    {dK, false, true},       {dT, false, true},     {dr, false, true},    {dq, false, true}};
  rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  Args a{n, S, K, T, V, flag, gbar, tau, gate_mode, steps, sigma_out, status_out, dV, dS, dK, dT, r, q, dr, dq};
  rc = check_counters(opts, dev, &a.counters);
  if (rc != PIVOT_OK) return rc;
  return mode == PIVOT_MODE_MIXED ? launch_binned<true, true, true>(a, stream)
                                  : launch_binned<true, false, true>(a, stream);
}

int pivot_mills_ratio(int64_t n, const double* z, double* y, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{z, true, true}, {y, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_mills_ratio<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, z, y);
  return launch_status();
}

int pivot_elementary(int32_t fn, int64_t n, const double* x, double* y, void* stream) {
  if (fn < 0 || fn > 4) return PIVOT_E_OPTS;
  if (n < 0) return PIVOT_E_SIZE;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{x, true, true}, {y, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_elementary<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(fn, n, x, y);
  return launch_status();
}

const char* pivot_error_string(int code) {
  switch (code) {
    case PIVOT_OK: return "ok";
    case PIVOT_E_SIZE: return "n < 0";
    case PIVOT_E_NULL: return "a required pointer is NULL";
    case PIVOT_E_GATE: return "bad gate_mode or tau";
    case PIVOT_E_OPTS: return "bad pivot_opts";
    case PIVOT_E_NOT_DEVICE: return "a pointer is not device memory of the current device";
    case PIVOT_E_ALIGN: return "a float64 pointer is not 8-byte aligned";
    case PIVOT_E_MLP: return "learned mode without weights, or bad training hyper-parameters";
    case PIVOT_E_TOO_MANY: return "n above the row limit of pivot_mlp_grad_static (2^26)";
    default: break;
  }
  if (code < 0) return cudaGetErrorString(static_cast<cudaError_t>(-code));
  return "unknown error";
}

int pivot_version(void) { return 200; }

}  // extern "C"

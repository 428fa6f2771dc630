// pivot_learned.cu -- PIVOT_MODE_LEARNED: the MLP initial guess on BF16 tensor
// cores (mma.sync, FP32 accumulation), FP64 Householder(3) steps on the LBR
// objectives (appendix stage 5), the gated adjoint, and the training kernels
// of the MLP (forward, backward and Adam, all in this file).
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pivot.h"
#include "pivot_device.cuh"
#include "pivot_internal.cuh"
#include "pivot_mlp.cuh"

namespace {

using namespace pivot::detail;
namespace M = pivot::mlp;

constexpr int kLBlock = 128; // 4 warps
constexpr int kLWarps = kLBlock / 32;
constexpr double kDefaultFallback = 0.25;

// The quote's normalised problem and its MLP features (lane = row); `has`
// false gives neutral features for the lanes that only keep the warp full.
struct LearnedRow {
  double x, bmax, beta, betac, lnb;
  M::Features f;
};

__device__ __forceinline__ LearnedRow learned_row(double F, double K, double T, double P, int fl) {
  LearnedRow r;
  const pivot::Quote q = pivot::classify_quote(F, K, T, P, fl);
  double rsq;
  pivot::moneyness(F, K, r.x, r.bmax, rsq);
  r.beta = q.tv * rsq;
  r.betac = q.cv * rsq;
  r.lnb = pivot::log_beta(r.beta, F, K, T, P, fl);
  r.f = M::features(r.x, r.beta, r.lnb);
  return r;
}

// ---------------------------------------------------------------------------
// Inference (PIVOT_MODE_LEARNED), one 2,048-row tile per block of 256 threads
// (2 blocks per SM):
//  phase 1: rows that need no solve are finished (as in the binned kernel),
//           the others listed; their time value and complement kept.
//  phase 2: warps take the list 32 rows at a time: FP64 normalisation, the
//           MLP seed s0 (features and baseline in float, network on tensor
//           cores with activations in registers), and the row's objective:
//           lower below the inflection b_c, middle up to beta = b_max/2,
//           upper beyond.  Lower-tail rows whose beta is below the float
//           range (|x| >= 0.1) take the float seed from ln beta of the mixed
//           form instead (bin 3); other rows outside the float range (beta_c
//           below 1e-30, |x| > 80, tiny beta near the money) go straight to
//           the fallback list.
//  phase 3: rows objective after objective: `steps - 1` float Householder(3)
//           steps from s0, then the FP64 final step of the mixed form, the
//           gated adjoint.  A row is accepted when the float steps moved s0
//           by at most `fallback` (relative) and the FP64 step moved the
//           float iterate by at most 1e-5 -- its quartic error is then far
//           below double rounding; otherwise it joins the fallback list.
//  phase 4: the fallback rows, densely: LBR's rational seed and FP64 steps.
// ---------------------------------------------------------------------------
constexpr int kIBlock = 256;
constexpr int kIWarps = kIBlock / 32;
constexpr int kITile = 2048;
constexpr int kIRowsPerThread = kITile / kIBlock;
constexpr double kAcceptFinal = 1e-5;
constexpr uint8_t kNoBin = 255;

struct InferSmem {
  M::Weights W;
  double x[kITile], rsq[kITile], bb[kITile];  // rsq = 1/sqrt(F K); b_max = min(F, K) rsq
  float s0[kITile];
  uint16_t list[kITile], order[kITile], pos[kITile], fb[kITile];
  uint8_t bin[kITile];
  int nsolve, nfb, cnt[6], off[7];
  unsigned long long count[PIVOT_COUNTERS_LEN]; // a.counters: this block's sums
};
// bins 0-2: the MLP-seeded objectives (lower, b - beta, upper); bin 3: deep lower-tail rows
// (beta below the float range, |x| >= 0.1), seeded in float from ln beta as in the mixed form;
// bins 4, 5: the rows of bins 0, 1 near the money (|x| <= kTaylorX), the only ones whose b may
// take the Taylor series of rho, so that a warp runs one form of rho
constexpr int kIBins = 6;

template <bool kBackward>
__device__ __forceinline__ void finish_row(const Args& a, int64_t i, double F, double K, double T, int fl, double s,
                                           double x, double bmax, double rsq, const pivot::Last& last) {
  const double inv_sqT = rsqrt(T);
  const double sig = s * inv_sqT;
  a.sigma[i] = sig;
  if (a.status) a.status[i] = 0;
  if (kBackward) {
    const double g = a.gbar ? a.gbar[i] : 1.0;
    const pivot::Grad d = isnan(g) ? pivot::degenerate_grad(true, g, a.mode)
                          : a.gbar ? pivot::adjoint_reuse<false>(F, K, fl, sig, s, x, bmax, inv_sqT, rsq, g, a.tau,
                                                                 a.mode, last)
                                   : pivot::adjoint_reuse<true>(F, K, fl, sig, s, x, bmax, inv_sqT, rsq, g, a.tau,
                                                                a.mode, last);
    if (a.dP) a.dP[i] = d.dP;
    if (a.dF) a.dF[i] = d.dF;
    if (a.dK) a.dK[i] = d.dK;
    if (a.dT) a.dT[i] = d.dT;
  }
}

template <bool kBackward>
__global__ void __launch_bounds__(kIBlock, 2) k_iv_learned(Args a, const pivot_mlp* net, double fallback) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  InferSmem& S = *reinterpret_cast<InferSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  M::stage_weights(net, S.W, nullptr);
  const int fsteps = a.steps - 1; // float steps before the FP64 one
  const bool counting = a.counters != nullptr;
  if (counting && tid < PIVOT_COUNTERS_LEN) S.count[tid] = 0;
  for (int64_t base = int64_t(blockIdx.x) * kITile; base < a.n; base += int64_t(gridDim.x) * kITile) {
    if (tid == 0) {
      S.nsolve = 0;
      S.nfb = 0;
      for (int k = 0; k < kIBins; ++k) S.cnt[k] = 0;
    }
    __syncthreads();
    // ---- phase 1: every row's loads first (a row's output stores would otherwise hold the
    // next row's loads back), then the stage-1 tests
    double rF[kIRowsPerThread], rK[kIRowsPerThread], rT[kIRowsPerThread], rP[kIRowsPerThread];
    int rfl[kIRowsPerThread];
#pragma unroll
    for (int j = 0; j < kIRowsPerThread; ++j) {
      const int64_t i = base + j * kIBlock + tid;
      rF[j] = rK[j] = rT[j] = rP[j] = 0.0;
      rfl[j] = 0;
      if (i < a.n) {
        rF[j] = a.F[i];
        rK[j] = a.K[i];
        rT[j] = a.T[i];
        rP[j] = a.P[i];
        rfl[j] = a.flag[i];
      }
    }
#pragma unroll
    for (int j = 0; j < kIRowsPerThread; ++j) {
      const int r = j * kIBlock + tid;
      const int64_t i = base + r;
      bool solve = false;
      int row_status = -1;
      if (i < a.n) {
        const double F = rF[j], K = rK[j], T = rT[j], P = rP[j];
        const int fl = rfl[j];
        const pivot::Quote q = pivot::classify_quote(F, K, T, P, fl);
        row_status = q.status;
        if (q.status != 0) {
          a.sigma[i] = q.sigma;
          if (a.status) a.status[i] = uint8_t(q.status);
          if (kBackward) {
            // outside the open price interval, or invalid: the degenerate gradient of its status
            const double g = a.gbar ? a.gbar[i] : 1.0;
            const double v = pivot::degenerate_grad(q.status <= 3 || pivot::nan64(g), g, a.mode).dP;
            if (a.dP) a.dP[i] = v;
            if (a.dF) a.dF[i] = v;
            if (a.dK) a.dK[i] = v;
            if (a.dT) a.dT[i] = v;
          }
        } else {
          solve = true;
          S.bb[r] = q.tv;
          S.x[r] = q.cv;
        }
      }
      const int slot = warp_append(solve, &S.nsolve, lane);
      if (solve) S.list[slot] = uint16_t(r);
      if (counting) {
#pragma unroll
        for (int k = 1; k < 6; ++k) {
          const unsigned m = __ballot_sync(0xffffffffu, row_status == k);
          if (lane == 0 && m) atomicAdd(&S.count[k], (unsigned long long)__popc(m));
        }
      }
    }
    __syncthreads();
    // ---- phase 2: normalisation, MLP seed, objective
    const int nsolve = S.nsolve;
    for (int c = warp; c * 32 < nsolve; c += kIWarps) {
      const int qi = c * 32 + lane;
      const bool has = qi < nsolve;
      const int r = has ? S.list[qi] : 0;
      bool learned = false;
      float f0 = 0.0f, f1 = 0.5f, bf = 0.0f;
      double x = 0.0, bmax = 0.0, rsq = 0.0, beta = 0.0, betac = 0.0;
      if (has) {
        const int64_t i = base + r;
        const double F = a.F[i], K = a.K[i];
        pivot::moneyness(F, K, x, bmax, rsq);
        beta = S.bb[r] * rsq;
        betac = S.x[r] * rsq;
        learned = beta > 1e-30 && betac > 1e-30 && x > -80.0;
        if (learned) {
          bf = float(beta);
          f0 = float(-x);
          f1 = rsqrtf(-2.0f * logf(bf));
        }
      }
      const float o = M::forward_regs(f0, f1, S.W); // every lane of the warp takes part
      int bin = -1;
      if (has) {
        S.x[r] = x;
        S.rsq[r] = rsq;
        if (!learned && !(beta > 1e-30) && betac > 1e-30 && x <= -0.1 && x > -80.0 && pivot::pos_normal(beta)) {
          bin = 3;
          S.bb[r] = beta;
        }
        if (learned) {
          const float s0 = fmaf(f0, f1, M::kSqrt2PiF * bf) * __expf(o);
          const float e = erfcxf(sqrtf(f0));
          const bool low = bf <= 0.5f * float(bmax) * (1.0f - e);
          bin = low ? 0 : (beta <= betac ? 1 : 2);
          if (bin < 2 && x >= -pivot::kTaylorX) bin += 4;
          if (!(s0 > 0.0f && s0 < INFINITY)) bin = -1;
          S.s0[r] = s0;
          S.bb[r] = (bin == 2) ? betac : beta;
        }
        if (bin < 0) S.fb[atomicAdd(&S.nfb, 1)] = uint16_t(r);
        S.bin[r] = bin < 0 ? kNoBin : uint8_t(bin);
      }
#pragma unroll
      for (int k = 0; k < kIBins; ++k) {
        const int p = warp_append(bin == k, &S.cnt[k], lane);
        if (bin == k) S.pos[r] = uint16_t(p);
      }
    }
    __syncthreads();
    if (tid == 0) {
      S.off[0] = 0;
      for (int k = 0; k < kIBins; ++k) S.off[k + 1] = S.off[k] + S.cnt[k];
    }
    __syncthreads();
    for (int qi = tid; qi < nsolve; qi += kIBlock) {
      const int r = S.list[qi];
      const int b = S.bin[r];
      if (b != kNoBin) S.order[S.off[b] + S.pos[r]] = uint16_t(r);
    }
    __syncthreads();
    // ---- phase 3: float steps from the seed, the FP64 final step, accept or defer
    const int total = S.off[kIBins];
    for (int qi = tid; qi < total; qi += kIBlock) {
      const int r = S.order[qi];
      int b = 0;
#pragma unroll
      for (int k = 1; k < kIBins; ++k) b += (qi >= S.off[k]) ? 1 : 0;
      if (b == 3) {
        // deep lower tail
        pivot::Last last;
        const int64_t i = base + r;
        const double F = a.F[i], K = a.K[i];
        const double x = S.x[r], rsq = S.rsq[r], bmax = pivot::bmax_of(F, K, rsq);
        const double s = pivot::solve_deep_mixed64(x, bmax, S.bb[r], last);
        if (pivot::pos_finite(s)) {
          finish_row<kBackward>(a, i, F, K, a.T[i], a.flag[i], s, x, bmax, rsq, last);
        } else {
          S.fb[atomicAdd(&S.nfb, 1)] = uint16_t(r);
        }
        continue;
      }
      const int bn = b >= 4 ? b - 4 : b;
      const int rg = bn == 0 ? pivot::kLower : bn == 1 ? pivot::kMidHigh : pivot::kUpper;
      const int64_t i = base + r;
      const double F = a.F[i], K = a.K[i];
      const double x = S.x[r], bb = S.bb[r], rsq = S.rsq[r], bmax = pivot::bmax_of(F, K, rsq);
      const float xf = float(x), bbf = float(bb);
      const float lnb = (rg == pivot::kMidHigh) ? 0.0f : logf(bbf);
      const float lnbetac = (rg == pivot::kUpper) ? lnb : 0.0f;
      const float inv_lnbeta = (rg == pivot::kLower) ? 1.0f / lnb : 0.0f;
      const float s0 = S.s0[r];
      float sf = s0;
      for (int k = 0; k < fsteps; ++k) sf = pivot::householder_step<float>(xf, bbf, lnbetac, inv_lnbeta, rg, sf);
      bool ok = sf > 0.0f && sf < INFINITY && fabsf(sf - s0) <= float(fallback) * sf;
      pivot::Last last;
      double s = 0.0;
      if (ok) {
        s = pivot::step64_final(x, bmax, bb, rg, double(sf), sf, xf, last);
        ok = fabs(s - double(sf)) <= kAcceptFinal * s;
      }
      if (ok) {
        finish_row<kBackward>(a, i, F, K, a.T[i], a.flag[i], s, x, bmax, rsq, last);
      } else {
        S.fb[atomicAdd(&S.nfb, 1)] = uint16_t(r);
      }
    }
    __syncthreads();
    // ---- phase 4: fallback rows on LBR's rational seed, FP64 steps
    const int nfb = S.nfb;
    for (int qi = tid; qi < nfb; qi += kIBlock) {
      const int r = S.fb[qi];
      const int64_t i = base + r;
      const double F = a.F[i], K = a.K[i], T = a.T[i], P = a.P[i];
      const int fl = a.flag[i];
      const pivot::Quote q = pivot::classify_quote(F, K, T, P, fl);
      double x, bmax, rsq;
      pivot::moneyness(F, K, x, bmax, rsq);
      pivot::Node<double> nd;
      const int rg = pivot::classify<double>(x, bmax, q.tv * rsq, q.cv * rsq, nd);
      const double lnb = (rg == pivot::kLower) ? pivot::log_beta(nd.bb, F, K, T, P, fl) : 0.0;
      pivot::Last last;
      const double s = pivot::solve64(rg, nd, lnb, a.steps, last);
      finish_row<kBackward>(a, i, F, K, T, fl, s, x, bmax, rsq, last);
    }
    __syncthreads();
    if (counting && tid == 0) {
      S.count[0] += S.nsolve;
      for (int k = 0; k < kIBins; ++k) S.count[kCountBin0 + k] += S.cnt[k];
      S.count[kCountReject] += nfb;
    }
  }
  if (counting) {
    __syncthreads();
    if (tid < PIVOT_COUNTERS_LEN && S.count[tid]) atomicAdd(&a.counters[tid], S.count[tid]);
  }
}

// ---------------------------------------------------------------------------
// Initial guesses alone (diagnostics: how far each seed is from the root).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_guess_rational(int64_t n, const double* __restrict__ F,
                                                           const double* __restrict__ K, const double* __restrict__ T,
                                                           const double* __restrict__ P, const int8_t* __restrict__ flag,
                                                           double* __restrict__ s_out) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const pivot::Quote q = pivot::classify_quote(F[i], K[i], T[i], P[i], flag[i]);
    double s = __longlong_as_double(0x7ff8000000000000LL);
    if (q.status == 0) {
      double x, bmax, rsq;
      pivot::moneyness(F[i], K[i], x, bmax, rsq);
      pivot::Node<double> nd;
      const int rg = pivot::classify<double>(x, bmax, q.tv * rsq, q.cv * rsq, nd);
      const double lnb = (rg == pivot::kLower) ? pivot::log_beta(nd.bb, F[i], K[i], T[i], P[i], flag[i]) : 0.0;
      s = pivot::region_guess<double>(rg, nd, lnb);
    }
    s_out[i] = s;
  }
}

__global__ void __launch_bounds__(kLBlock) k_guess_mlp(int64_t n, const double* __restrict__ F,
                                                       const double* __restrict__ K, const double* __restrict__ T,
                                                       const double* __restrict__ P, const int8_t* __restrict__ flag,
                                                       const pivot_mlp* net, double* __restrict__ s_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  M::Weights& W = *reinterpret_cast<M::Weights*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  M::stage_weights(net, W, nullptr);
  __syncthreads();
  for (int64_t c0 = (int64_t(blockIdx.x) * kLWarps + warp) * 32; c0 < n; c0 += int64_t(gridDim.x) * kLWarps * 32) {
    const int64_t i = c0 + lane;
    bool has = false;
    LearnedRow row;
    float f0 = 0.0f, f1 = 0.5f;
    if (i < n) {
      const pivot::Quote q = pivot::classify_quote(F[i], K[i], T[i], P[i], flag[i]);
      if (q.status == 0) {
        has = true;
        row = learned_row(F[i], K[i], T[i], P[i], flag[i]);
        f0 = row.f.f0;
        f1 = row.f.f1;
      }
    }
    const float o = M::forward_regs(f0, f1, W);
    if (i < n) s_out[i] = has ? row.f.sa * exp(double(o)) : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// ---------------------------------------------------------------------------
// Training: parameters, gradient pass, Adam.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ void write_net_param(pivot_mlp* net, int i, float p) {
  const uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(p));
  if (i < M::OB1) net->w1[i - M::OW1] = b;
  else if (i < M::OW2) net->b1[i - M::OB1] = p;
  else if (i < M::OB2) net->w2[i - M::OW2] = b;
  else if (i < M::OW3) net->b2[i - M::OB2] = p;
  else if (i < M::OB3) net->w3[i - M::OW3] = b;
  else if (i < M::OW4) net->b3[i - M::OB3] = p;
  else if (i < M::OB4) net->w4[i - M::OW4] = b;
  else net->b4 = p;
}

__global__ void k_mlp_init(pivot_mlp_trainer* tr, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M::NPARAM; i += gridDim.x * blockDim.x) {
    const int fan_in = (i < M::OW2) ? 2 : M::H;
    const double u = double(splitmix64(seed * 0x100000001B3ull + uint64_t(i)) >> 11) * (1.0 / 9007199254740992.0);
    const float p = float((2.0 * u - 1.0) * rsqrt(double(fan_in)));
    tr->param[i] = p;
    tr->grad[i] = 0.0f;
    tr->adam_m[i] = 0.0f;
    tr->adam_v[i] = 0.0f;
    write_net_param(&tr->net, i, p);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    tr->loss_sum = 0.0;
    tr->rows = 0.0;
    tr->step = 0;
  }
}

struct TrainSmem {
  M::Weights W;
  M::WeightsT WT;
  M::TrainTiles tiles[kLWarps];
};

// The MLP gradient pass over n rows (forward + backward on tensor cores): the
// gradient of the sum of squared errors is added to grad[], the sum to
// *loss_sum and the row count to *rows.  Shared by pivot_mlp_grad (the
// trainer's own accumulators) and pivot_mlp_grad_static (the library's
// static scratch).
__device__ __forceinline__ void mlp_grad_rows(const pivot_mlp* net, int64_t n, const double* __restrict__ F,
                                              const double* __restrict__ K, const double* __restrict__ T,
                                              const double* __restrict__ P, const int8_t* __restrict__ flag,
                                              const double* __restrict__ sigma, float* grad, double* loss_sum,
                                              double* rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  M::stage_weights(net, S.W, &S.WT);
  __syncthreads();
  float sq = 0.0f;
  int nvalid = 0;
  for (int64_t c0 = (int64_t(blockIdx.x) * kLWarps + warp) * 32; c0 < n; c0 += int64_t(gridDim.x) * kLWarps * 32) {
    const int64_t i = c0 + lane;
    bool valid = false;
    float f0 = 0.0f, f1 = 0.5f, y = 0.0f;
    if (i < n) {
      const double sg = sigma[i];
      const pivot::Quote q = pivot::classify_quote(F[i], K[i], T[i], P[i], flag[i]);
      if (q.status == 0 && sg > 0.0 && sg < INFINITY) {
        const LearnedRow row = learned_row(F[i], K[i], T[i], P[i], flag[i]);
        const double target = log(sg * sqrt(T[i]) / row.f.sa);
        if (row.f.sa > 0.0 && fabs(target) < 1e30) {
          valid = true;
          f0 = row.f.f0;
          f1 = row.f.f1;
          y = float(target);
        }
      }
    }
    sq += M::train_warp(f0, f1, y, valid, S.W, S.WT, S.tiles[warp], grad);
    nvalid += valid ? 1 : 0;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, off);
    nvalid += __shfl_xor_sync(0xffffffffu, nvalid, off);
  }
  if (lane == 0) {
    atomicAdd(loss_sum, double(sq));
    atomicAdd(rows, double(nvalid));
  }
}

__global__ void __launch_bounds__(kLBlock, 1) k_mlp_grad(pivot_mlp_trainer* tr, int64_t n, const double* __restrict__ F,
                                                         const double* __restrict__ K, const double* __restrict__ T,
                                                         const double* __restrict__ P, const int8_t* __restrict__ flag,
                                                         const double* __restrict__ sigma) {
  mlp_grad_rows(&tr->net, n, F, K, T, P, flag, sigma, tr->grad, &tr->loss_sum, &tr->rows);
}

__global__ void k_mlp_adam(pivot_mlp_trainer* tr, double lr, double beta1, double beta2, double eps) {
  const double rows = tr->rows;
  const double inv = rows > 0.0 ? 1.0 / rows : 0.0;
  const double t = double(tr->step + 1);
  const double c1 = 1.0 / (1.0 - pow(beta1, t)), c2 = 1.0 / (1.0 - pow(beta2, t));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M::NPARAM; i += gridDim.x * blockDim.x) {
    const double g = double(tr->grad[i]) * inv;
    const double m = beta1 * double(tr->adam_m[i]) + (1.0 - beta1) * g;
    const double v = beta2 * double(tr->adam_v[i]) + (1.0 - beta2) * g * g;
    tr->adam_m[i] = float(m);
    tr->adam_v[i] = float(v);
    const float p = float(double(tr->param[i]) - lr * (m * c1) / (sqrt(v * c2) + eps));
    tr->param[i] = p;
    tr->grad[i] = 0.0f;
    write_net_param(&tr->net, i, p);
  }
}

__global__ void k_mlp_adam_finish(pivot_mlp_trainer* tr) {
  tr->step += 1;
  tr->loss_sum = 0.0;
  tr->rows = 0.0;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

namespace pivot {
namespace detail {

int launch_learned(const Args& a, const pivot_mlp* mlp, double fallback, bool backward, void* stream) {
  const size_t smem = sizeof(InferSmem);
  static thread_local int configured_device = -1;
  static thread_local int grid_cap = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return launch_status();
  if (configured_device != dev) {
    cudaFuncSetAttribute(k_iv_learned<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    cudaFuncSetAttribute(k_iv_learned<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int b0 = 0, b1 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_iv_learned<false>, kIBlock, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_iv_learned<true>, kIBlock, smem);
    const int b = (b0 < b1 ? b0 : b1) > 0 ? (b0 < b1 ? b0 : b1) : 1;
    grid_cap = b * sm_count();
    configured_device = dev;
  }
  const int64_t tiles = (a.n + kITile - 1) / kITile;
  const unsigned grid = unsigned(tiles < grid_cap ? tiles : grid_cap);
  const double fb = fallback > 0.0 ? fallback : kDefaultFallback;
  if (backward)
    k_iv_learned<true><<<grid, kIBlock, smem, static_cast<cudaStream_t>(stream)>>>(a, mlp, fb);
  else
    k_iv_learned<false><<<grid, kIBlock, smem, static_cast<cudaStream_t>(stream)>>>(a, mlp, fb);
  return launch_status();
}

}  // namespace detail
}  // namespace pivot

extern "C" {

int64_t pivot_mlp_trainer_bytes(int64_t* net_offset) {
  if (net_offset) *net_offset = int64_t(offsetof(pivot_mlp_trainer, net));
  return int64_t(sizeof(pivot_mlp_trainer));
}

int pivot_iv_guess(int64_t n, const double* F, const double* K, const double* T, const double* P,
                   const int8_t* flag, const pivot_opts* opts, double* s_out, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  const bool learned = opts && opts->mode == PIVOT_MODE_LEARNED;
  if (opts && opts->mode != PIVOT_MODE_FP64 && !learned) return PIVOT_E_OPTS;
  if (learned && opts->mlp == nullptr) return PIVOT_E_MLP;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true}, {K, true, true}, {T, true, true}, {P, true, true}, {flag, true, false},
                    {s_out, true, true}, {learned ? opts->mlp : nullptr, learned, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!learned) {
    k_guess_rational<<<grid_for(n), kBlock, 0, st>>>(n, F, K, T, P, flag, s_out);
    return launch_status();
  }
  const size_t smem = sizeof(M::Weights);
  cudaFuncSetAttribute(k_guess_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int64_t chunks = (n + 32 * kLWarps - 1) / (32 * kLWarps);
  const int64_t cap = int64_t(4) * sm_count();
  k_guess_mlp<<<unsigned(chunks < cap ? chunks : cap), kLBlock, smem, st>>>(n, F, K, T, P, flag, opts->mlp, s_out);
  return launch_status();
}

int pivot_mlp_init(pivot_mlp_trainer* trainer, uint64_t seed, void* stream) {
  int dev = -1;
  const Ptr ps[] = {{trainer, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  k_mlp_init<<<34, 256, 0, static_cast<cudaStream_t>(stream)>>>(trainer, seed);
  return launch_status();
}

int pivot_mlp_grad(pivot_mlp_trainer* trainer, int64_t n, const double* F, const double* K, const double* T,
                   const double* P, const int8_t* flag, const double* sigma, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{trainer, true, true}, {F, true, true}, {K, true, true}, {T, true, true},
                    {P, true, true},       {flag, true, false}, {sigma, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  const size_t smem = sizeof(TrainSmem);
  cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  const int64_t chunks = (n + 32 * kLWarps - 1) / (32 * kLWarps);
  const int64_t cap = sm_count();
  k_mlp_grad<<<unsigned(chunks < cap ? chunks : cap), kLBlock, smem, static_cast<cudaStream_t>(stream)>>>(
      trainer, n, F, K, T, P, flag, sigma);
  return launch_status();
}

int pivot_mlp_adam(pivot_mlp_trainer* trainer, double lr, double beta1, double beta2, double eps, void* stream) {
  if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return PIVOT_E_MLP;
  int dev = -1;
  const Ptr ps[] = {{trainer, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_mlp_adam<<<34, 256, 0, st>>>(trainer, lr, beta1, beta2, eps);
  k_mlp_adam_finish<<<1, 1, 0, st>>>(trainer);
  return launch_status();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// pivot_mlp_grad_static: the gradient pass of pivot_mlp_grad for callers that
// cannot allocate device memory.  Its scratch (the FP32 gradient accumulator
// and the two loss sums) is a fixed array inside the library instead of the
// caller's pivot_mlp_trainer; the result is copied to the caller's outputs.
// ---------------------------------------------------------------------------
namespace {

// rows one call may cover: FP32 sums over more rows lose their last digits
constexpr int64_t kStaticGradMaxRows = int64_t(1) << 26;
// PIVOT_MLP_NPARAM accumulators, padded to an 8-byte boundary, then 2 doubles
constexpr int kStaticLossOffset = ((PIVOT_MLP_NPARAM + 1) / 2) * 2;
constexpr int kStaticScratchFloats = kStaticLossOffset + 4;

static __device__ __align__(256) float g_mlp_grad_scratch[kStaticScratchFloats];

__global__ void k_static_scratch_zero(float* scratch) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kStaticScratchFloats; i += gridDim.x * blockDim.x)
    scratch[i] = 0.0f;
}

__global__ void __launch_bounds__(kLBlock, 1)
    k_mlp_grad_static(const pivot_mlp* net, int64_t n, const double* __restrict__ F, const double* __restrict__ K,
                      const double* __restrict__ T, const double* __restrict__ P, const int8_t* __restrict__ flag,
                      const double* __restrict__ sigma, float* scratch) {
  double* loss = reinterpret_cast<double*>(scratch + kStaticLossOffset);
  mlp_grad_rows(net, n, F, K, T, P, flag, sigma, scratch, loss, loss + 1);
}

__global__ void k_static_scratch_copy_out(const float* scratch, float* grad_out, double* loss_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < PIVOT_MLP_NPARAM; i += gridDim.x * blockDim.x)
    grad_out[i] = scratch[i];
  if (blockIdx.x == 0 && threadIdx.x < 2)
    loss_out[threadIdx.x] = reinterpret_cast<const double*>(scratch + kStaticLossOffset)[threadIdx.x];
}

// device address of the static scratch, looked up once per device with that device current.
// Host threads may make their first call on a device at the same time: each slot is an atomic,
// and a lookup that loses the race stores the same address.  The cache assumes the device's
// context lives as long as the process (after cudaDeviceReset the module, and so the array, may
// be loaded at another address).
int static_scratch(float** out) {
  constexpr int kMaxDevices = 64;
  static std::atomic<float*> addr[kMaxDevices];
  int dev = 0;
  const cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return -int(e0);
  if (dev < 0 || dev >= kMaxDevices) return PIVOT_E_NOT_DEVICE;
  float* p = addr[dev].load(std::memory_order_acquire);
  if (p == nullptr) {
    void* q = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&q, g_mlp_grad_scratch);
    if (e != cudaSuccess) return -int(e);
    p = static_cast<float*>(q);
    addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return PIVOT_OK;
}

}  // namespace

extern "C" int pivot_mlp_grad_static(const pivot_mlp* net, int64_t n, const double* F, const double* K,
                                     const double* T, const double* P, const int8_t* flag, const double* sigma,
                                     float* grad_out, double* loss_out, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if (n > kStaticGradMaxRows) return PIVOT_E_TOO_MANY;
  if (reinterpret_cast<uintptr_t>(net) & 3u || reinterpret_cast<uintptr_t>(grad_out) & 3u) return PIVOT_E_ALIGN;
  int dev = -1;
  const Ptr ps[] = {{net, true, false},     {grad_out, true, false}, {loss_out, true, true},
                    {F, n > 0, true},       {K, n > 0, true},        {T, n > 0, true},
                    {P, n > 0, true},       {flag, n > 0, false},    {sigma, n > 0, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  if (rc != PIVOT_OK) return rc;
  float* scratch = nullptr;
  rc = static_scratch(&scratch);
  if (rc != PIVOT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's sums: clear it first
  k_static_scratch_zero<<<34, 256, 0, st>>>(scratch);
  if (n > 0) {
    const size_t smem = sizeof(TrainSmem);
    cudaFuncSetAttribute(k_mlp_grad_static, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const int64_t chunks = (n + 32 * kLWarps - 1) / (32 * kLWarps);
    const int64_t cap = sm_count();
    k_mlp_grad_static<<<unsigned(chunks < cap ? chunks : cap), kLBlock, smem, st>>>(net, n, F, K, T, P, flag, sigma,
                                                                                    scratch);
  }
  k_static_scratch_copy_out<<<34, 256, 0, st>>>(scratch, grad_out, loss_out);
  return launch_status();
}

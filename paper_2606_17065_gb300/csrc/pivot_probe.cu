// pivot_probe.cu -- throughput probes of the units the hot path runs on: the
// FP64 and FP32 fused multiply-add pipes, the multi-function unit (MUFU), and
// a row stream with the hot path's own HBM layout.  The roofline fractions of
// the inversion kernels are stated against these measured rates beside the
// rates derived from unit counts and clocks.  Diagnostic entry points: the
// paper has no counterpart.
#include <cstdint>
#include <cuda_runtime.h>

#include "pivot.h"
#include "pivot_internal.cuh"

namespace {

using namespace pivot::detail;

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent dependency chains per thread
constexpr int kUnroll = 8;  // chain rounds per loop iteration

// `iters` loop iterations of kUnroll rounds over kChains independent chains
// a <- a * b + c (b just below 1, so every chain stays near c / (1 - b)).  The
// result is stored only when it equals a value it cannot reach, which keeps
// the chains live without a store per thread.
template <typename R>
__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(int64_t iters, R* sink) {
  R a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = R(1) + R(threadIdx.x * kChains + k) * R(1e-6);
  const R b = R(0.999), c = R(1e-3);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == R(-1)) sink[blockIdx.x] = s;
}

// MUFU: ex2.approx (fn 0) or tanh.approx (fn 1) chains in float.  ex2 of a
// negated value in (0, 1] stays in [1/2, 1); tanh shrinks its argument slowly.
template <int kFn>
__global__ void __launch_bounds__(kProbeThreads) k_probe_mufu(int64_t iters, float* sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 0.5f + float(threadIdx.x * kChains + k) * 1e-6f;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        if (kFn == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[k]) : "f"(-a[k]));
        else asm volatile("tanh.approx.f32 %0, %1;" : "=f"(a[k]) : "f"(a[k]));
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

// The row stream of the fused forward+backward: read F, K, T, P (float64) and
// flag (int8), write sigma, dP, dF, dK, dT (float64) and status (uint8), 74
// bytes per row, with no arithmetic between.  kVec2: each thread moves two
// consecutive rows with 128-bit loads and stores of every float64 array (and
// 16-bit ones of the int8 arrays); otherwise one row per thread with 64-bit
// accesses.  The caller's arrays are 16-byte aligned for kVec2 (checked on the
// host), and an odd last row is moved by the scalar form.
template <bool kVec2>
__global__ void __launch_bounds__(kProbeThreads) k_probe_stream(int64_t n, const double* __restrict__ F,
                                                                const double* __restrict__ K,
                                                                const double* __restrict__ T,
                                                                const double* __restrict__ P,
                                                                const int8_t* __restrict__ flag,
                                                                double* __restrict__ sigma, uint8_t* __restrict__ st,
                                                                double* __restrict__ dP, double* __restrict__ dF,
                                                                double* __restrict__ dK, double* __restrict__ dT) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (kVec2) {
    const int64_t npair = n >> 1;
#pragma unroll 1
    for (int64_t p = t0; p < npair; p += stride) {
      const double2 f = reinterpret_cast<const double2*>(F)[p];
      const double2 k = reinterpret_cast<const double2*>(K)[p];
      const double2 t = reinterpret_cast<const double2*>(T)[p];
      const double2 q = reinterpret_cast<const double2*>(P)[p];
      const char2 fl = reinterpret_cast<const char2*>(flag)[p];
      reinterpret_cast<double2*>(sigma)[p] = q;
      reinterpret_cast<double2*>(dP)[p] = f;
      reinterpret_cast<double2*>(dF)[p] = k;
      reinterpret_cast<double2*>(dK)[p] = t;
      reinterpret_cast<double2*>(dT)[p] = q;
      reinterpret_cast<uchar2*>(st)[p] = make_uchar2(uint8_t(fl.x), uint8_t(fl.y));
    }
    if (t0 == 0 && (n & 1)) {
      const int64_t i = n - 1;
      sigma[i] = P[i];
      dP[i] = F[i];
      dF[i] = K[i];
      dK[i] = T[i];
      dT[i] = P[i];
      st[i] = uint8_t(flag[i]);
    }
  } else {
#pragma unroll 1
    for (int64_t i = t0; i < n; i += stride) {
      const double f = F[i], k = K[i], t = T[i], q = P[i];
      const int8_t fl = flag[i];
      sigma[i] = q;
      dP[i] = f;
      dF[i] = k;
      dK[i] = t;
      dT[i] = q;
      st[i] = uint8_t(fl);
    }
  }
}

int probe_grid(int blocks_per_sm, unsigned* grid) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return -int(e);
  *grid = unsigned(sms * blocks_per_sm);
  return PIVOT_OK;
}

}  // namespace

extern "C" {

int pivot_probe_units(int32_t unit, int32_t blocks_per_sm, int64_t iters, void* sink, double* lane_ops,
                      void* stream) {
  if (unit < 0 || unit > 3 || blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1) return PIVOT_E_OPTS;
  if (lane_ops == nullptr) return PIVOT_E_NULL;
  int dev = -1;
  const Ptr ps[] = {{sink, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK) rc = select_device(dev);
  unsigned grid = 0;
  if (rc == PIVOT_OK) rc = probe_grid(blocks_per_sm, &grid);
  if (rc != PIVOT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (unit) {
    case 0: k_probe_fma<double><<<grid, kProbeThreads, 0, st>>>(iters, static_cast<double*>(sink)); break;
    case 1: k_probe_fma<float><<<grid, kProbeThreads, 0, st>>>(iters, static_cast<float*>(sink)); break;
    case 2: k_probe_mufu<0><<<grid, kProbeThreads, 0, st>>>(iters, static_cast<float*>(sink)); break;
    default: k_probe_mufu<1><<<grid, kProbeThreads, 0, st>>>(iters, static_cast<float*>(sink)); break;
  }
  *lane_ops = double(grid) * kProbeThreads * double(iters) * kUnroll * kChains;
  return launch_status();
}

int pivot_probe_stream(int32_t width, int64_t n, const double* F, const double* K, const double* T, const double* P,
                       const int8_t* flag, double* sigma, uint8_t* status, double* dP, double* dF, double* dK,
                       double* dT, int32_t blocks_per_sm, void* stream) {
  if (n < 0) return PIVOT_E_SIZE;
  if ((width != 1 && width != 2) || blocks_per_sm < 1 || blocks_per_sm > 32) return PIVOT_E_OPTS;
  if (n == 0) return PIVOT_OK;
  int dev = -1;
  const Ptr ps[] = {{F, true, true},      {K, true, true},  {T, true, true},  {P, true, true},
                    {flag, true, false},  {sigma, true, true}, {status, true, false},
                    {dP, true, true},     {dF, true, true}, {dK, true, true}, {dT, true, true}};
  int rc = check_all(ps, &dev);
  if (rc == PIVOT_OK && width == 2) {
    const void* v[] = {F, K, T, P, sigma, dP, dF, dK, dT};
    for (const void* p : v)
      if (reinterpret_cast<uintptr_t>(p) & 15u) rc = PIVOT_E_ALIGN;
    if ((reinterpret_cast<uintptr_t>(flag) | reinterpret_cast<uintptr_t>(status)) & 1u) rc = PIVOT_E_ALIGN;
  }
  if (rc == PIVOT_OK) rc = select_device(dev);
  unsigned grid = 0;
  if (rc == PIVOT_OK) rc = probe_grid(blocks_per_sm, &grid);
  if (rc != PIVOT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (width == 2)
    k_probe_stream<true><<<grid, kProbeThreads, 0, st>>>(n, F, K, T, P, flag, sigma, status, dP, dF, dK, dT);
  else
    k_probe_stream<false><<<grid, kProbeThreads, 0, st>>>(n, F, K, T, P, flag, sigma, status, dP, dF, dK, dT);
  return launch_status();
}

}  // extern "C"

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

namespace {

constexpr int kBlock = 256;
constexpr int kDefaultSteps = 2;

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

__global__ void __launch_bounds__(kBlock) k_iv_forward(int64_t n, const double* __restrict__ F,
                                                       const double* __restrict__ K, const double* __restrict__ T,
                                                       const double* __restrict__ P, const int8_t* __restrict__ flag,
                                                       double* __restrict__ sigma, uint8_t* __restrict__ status,
                                                       int steps) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const pivot::Prepared p = pivot::prepare(F[i], K[i], T[i], P[i], flag[i]);
    double sig = p.sigma;
    if (p.status == 0) sig = pivot::solve_s(p, steps, nullptr) / p.sqrtT;
    sigma[i] = sig;
    if (status) status[i] = uint8_t(p.status);
  }
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

__global__ void __launch_bounds__(kBlock) k_iv_forward_backward(
    int64_t n, const double* __restrict__ F, const double* __restrict__ K, const double* __restrict__ T,
    const double* __restrict__ P, const int8_t* __restrict__ flag, const double* __restrict__ gbar, double tau,
    int mode, double* __restrict__ sigma, uint8_t* __restrict__ status, double* __restrict__ dP,
    double* __restrict__ dF, double* __restrict__ dK, double* __restrict__ dT, int steps) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double f = F[i], k = K[i], tt = T[i];
    const int fl = flag[i];
    const pivot::Prepared p = pivot::prepare(f, k, tt, P[i], fl);
    double sig = p.sigma;
    if (p.status == 0) sig = pivot::solve_s(p, steps, nullptr) / p.sqrtT;
    sigma[i] = sig;
    if (status) status[i] = uint8_t(p.status);
    const double g = gbar ? gbar[i] : 1.0;
    const pivot::Grad d = pivot::gated_adjoint(f, k, tt, fl, sig, g, tau, mode);
    if (dP) dP[i] = d.dP;
    if (dF) dF[i] = d.dF;
    if (dK) dK[i] = d.dK;
    if (dT) dT[i] = d.dT;
  }
}

// ---------------------------------------------------------------------------
// host-side argument checks
// ---------------------------------------------------------------------------
int check_ptr(const void* p, bool required, bool f64, int* device) {
  if (p == nullptr) return required ? PIVOT_E_NULL : PIVOT_OK;
  if (f64 && (reinterpret_cast<uintptr_t>(p) & 7u)) return PIVOT_E_ALIGN;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return PIVOT_E_NOT_DEVICE;
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PIVOT_E_NOT_DEVICE;
  if (*device < 0) *device = a.device;
  else if (a.device != *device) return PIVOT_E_NOT_DEVICE;
  return PIVOT_OK;
}

struct Ptr {
  const void* p;
  bool required;
  bool f64;
};

template <int N>
int check_all(const Ptr (&ps)[N], int* device) {
  for (int i = 0; i < N; ++i) {
    const int rc = check_ptr(ps[i].p, ps[i].required, ps[i].f64, device);
    if (rc != PIVOT_OK) return rc;
  }
  return PIVOT_OK;
}

int check_gate(double tau, int32_t mode) {
  if (mode < PIVOT_GATE_EXACT || mode > PIVOT_GATE_SMOOTH) return PIVOT_E_GATE;
  if (!(tau >= 0.0) || !(tau < INFINITY)) return PIVOT_E_GATE;
  if (mode == PIVOT_GATE_SMOOTH && !(tau > 0.0)) return PIVOT_E_GATE;
  return PIVOT_OK;
}

int check_opts(const pivot_opts* o, int* steps, int* mode) {
  *steps = kDefaultSteps;
  *mode = PIVOT_MODE_FP64;
  if (o == nullptr) return PIVOT_OK;
  if (o->mode != PIVOT_MODE_FP64) return PIVOT_E_OPTS;  // other modes: separate entry points
  if (o->householder < 0 || o->householder > 4) return PIVOT_E_OPTS;
  if (o->householder > 0) *steps = o->householder;
  *mode = o->mode;
  return PIVOT_OK;
}

unsigned grid_for(int64_t n) {
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  const int64_t cap = int64_t(1) << 20;
  return unsigned(blocks < cap ? blocks : cap);
}

int launch_status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PIVOT_OK : -int(e);
}

int select_device(int device) {
  if (device < 0) return PIVOT_OK;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return PIVOT_E_NOT_DEVICE;
  if (cur != device && cudaSetDevice(device) != cudaSuccess) return PIVOT_E_NOT_DEVICE;
  return PIVOT_OK;
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
  k_iv_forward<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(n, F, K, T, P, flag, sigma_out,
                                                                                 status_out, steps);
  return launch_status();
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
  k_iv_forward_backward<<<grid_for(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(
      n, F, K, T, P, flag, gbar, tau, gate_mode, sigma_out, status_out, dP, dF, dK, dT, steps);
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
    default: break;
  }
  if (code < 0) return cudaGetErrorString(static_cast<cudaError_t>(-code));
  return "unknown error";
}

int pivot_version(void) { return 100; }

}  // extern "C"

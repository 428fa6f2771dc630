// pivot_internal.cuh -- kernel plumbing shared by the translation units of
// the library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pivot.h"
#include "pivot_device.cuh"

namespace pivot {
namespace detail {

constexpr int kBlock = 256;
constexpr int kDefaultSteps = 2;

struct Args {
  int64_t n;
  const double *F, *K, *T, *P;
  const int8_t* flag;
  const double* gbar;
  double tau;
  int mode;
  int steps;
  double* sigma;
  uint8_t* status;
  double *dP, *dF, *dK, *dT;
  // Black-Scholes form only: F holds the spot S, P the discounted price V,
  // dP / dF / dT receive dsigma/dV, dsigma/dS, dsigma/dtau; r, q per row
  const double *r, *q;
  double *dr, *dq;
  // PIVOT_COUNTERS_LEN per-launch counters (pivot_opts.counters), or NULL
  unsigned long long* counters;
};

// slots of the counters (include/pivot.h)
constexpr int kCountBin0 = 6;
constexpr int kCountReject = 18;

// Black-Scholes form: the gated adjoint of a finished row in xi coordinates
__device__ __forceinline__ void write_grad_bs(const Args& a, int64_t i, double F, double K, double T, int fl,
                                              double sig, double r, double q, double er, double ec) {
  const double g = a.gbar ? a.gbar[i] : 1.0;
  const pivot::Grad d = pivot::gated_adjoint(F, K, T, fl, sig, g, a.tau * er, a.mode);
  const pivot::BSGrad o = pivot::bs_grad(d, F, K, T, r, q, er, ec);
  if (a.dP) a.dP[i] = o.dV;
  if (a.dF) a.dF[i] = o.dS;
  if (a.dK) a.dK[i] = o.dK;
  if (a.dT) a.dT[i] = o.dT;
  if (a.dr) a.dr[i] = o.dr;
  if (a.dq) a.dq[i] = o.dq;
}

// warp-aggregated append: returns this lane's slot in a shared counter
__device__ __forceinline__ int warp_append(bool take, int* counter, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, take);
  int b0 = 0;
  if (m) {
    const int leader = __ffs(m) - 1;
    if (lane == leader) b0 = atomicAdd(counter, __popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, leader);
  }
  return b0 + __popc(m & ((1u << lane) - 1u));
}

// ---------------------------------------------------------------------------
// host-side argument checks
// ---------------------------------------------------------------------------
inline int check_ptr(const void* p, bool required, bool f64, int* device) {
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
inline int check_all(const Ptr (&ps)[N], int* device) {
  for (int i = 0; i < N; ++i) {
    const int rc = check_ptr(ps[i].p, ps[i].required, ps[i].f64, device);
    if (rc != PIVOT_OK) return rc;
  }
  return PIVOT_OK;
}

inline int check_gate(double tau, int32_t mode) {
  if (mode < PIVOT_GATE_EXACT || mode > PIVOT_GATE_SMOOTH) return PIVOT_E_GATE;
  if (!(tau >= 0.0) || !(tau < INFINITY)) return PIVOT_E_GATE;
  if (mode == PIVOT_GATE_SMOOTH && !(tau > 0.0)) return PIVOT_E_GATE;
  return PIVOT_OK;
}

inline unsigned grid_for(int64_t n) {
  const int64_t blocks = (n + kBlock - 1) / kBlock;
  const int64_t cap = int64_t(1) << 20;
  return unsigned(blocks < cap ? blocks : cap);
}

inline int launch_status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PIVOT_OK : -int(e);
}

inline int select_device(int device) {
  if (device < 0) return PIVOT_OK;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return PIVOT_E_NOT_DEVICE;
  if (cur != device && cudaSetDevice(device) != cudaSuccess) return PIVOT_E_NOT_DEVICE;
  return PIVOT_OK;
}

// the counters of pivot_opts: NULL, or device memory of the call's device
inline int check_counters(const pivot_opts* o, int device, unsigned long long** out) {
  *out = nullptr;
  if (o == nullptr || o->counters == nullptr) return PIVOT_OK;
  int d = device;
  const int rc = check_ptr(o->counters, true, true, &d);
  if (rc != PIVOT_OK) return rc;
  *out = reinterpret_cast<unsigned long long*>(o->counters);
  return PIVOT_OK;
}

// PIVOT_MODE_LEARNED launch (pivot_learned.cu)
int launch_learned(const Args& a, const pivot_mlp* mlp, double fallback, bool backward, void* stream);

}  // namespace detail
}  // namespace pivot

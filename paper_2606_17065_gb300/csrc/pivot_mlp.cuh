// pivot_mlp.cuh -- the learned initial guess: an MLP 2 -> 64 -> 64 -> 64 -> 1
// (SiLU) with BF16 weights and FP32 accumulation, evaluated and trained per
// warp on 32 rows at a time with mma.sync m16n8k16 (BF16 in, FP32 out).
//
// Inputs (|x|, q = 1/sqrt(-2 ln beta)), output o ~ ln(s / s_a) with
// s_a = |x| q + sqrt(2 pi) beta: s_a follows the two closed-form limits of
// b(x, s) = beta (s ~ |x|/sqrt(-2 ln beta) deep out of the money, where
// ln b ~ -x^2/(2 s^2); s ~ sqrt(2 pi) beta at the money for small s, where
// b(0, s) = 2 Phi(s/2) - 1 ~ s/sqrt(2 pi)), so the network only learns a
// bounded correction.  The seed replaces the LBR node and rational guess;
// the FP64 Householder steps that follow are the paper's (appendix stage 5).
//
// Fragment layouts of mma.m16n8k16 with BF16 operands (g = lane/4, t = lane%4):
//   A (16x16, row major): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..], a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]
//   B (16x8, "col"):      b0 = B[2t..2t+1][g],  b1 = B[2t+8..2t+9][g]
//   C (16x8, FP32):       c0, c1 = C[g][2t], C[g][2t+1];  c2, c3 = C[g+8][2t], C[g+8][2t+1]
// A is read from a row-major [m][k] shared array and B from a [n][k] array
// (k contiguous), so every fragment register is one 32-bit shared load.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pivot.h"

namespace pivot {
namespace mlp {

constexpr int H = PIVOT_MLP_HIDDEN; // 64
constexpr int kRows = 32;           // rows per warp
constexpr int LDA = H + 8;          // row-major activations [row][H] (bf16), padded
constexpr int LDT = kRows + 8;      // transposed activations [H][row] (bf16), padded
constexpr int LDW = H + 8;          // weights [n][k] (bf16), padded

// flat FP32 parameter order
constexpr int OW1 = 0, OB1 = OW1 + H * 2, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + H, NPARAM = OB4 + 1;
static_assert(NPARAM == PIVOT_MLP_NPARAM, "parameter count");

constexpr float kSqrt2PiF = 2.50662827463100050242f;

// SiLU through the hardware tanh: sigmoid(z) = (1 + tanh(z/2))/2, one MUFU
// operation instead of an exponential and a division.  tanh.approx has a
// relative error below 2^-10.9, under the BF16 rounding (2^-9) that every
// activation then takes; training and inference use the same function.
__device__ __forceinline__ float tanh_approx(float v) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float sigmoid(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) { return z * sigmoid(z); }
__device__ __forceinline__ float silu_grad(float z) {
  const float sg = sigmoid(z);
  return sg * fmaf(z, 1.0f - sg, 1.0f);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C[MT*16 x NT*8] = A[.. x KS*16] * B, A row-major (lda), B given as Bt[n][k]
// (ldb); epi(row, col, value) receives every element of C.
template <int MT, int NT, int KS, typename Epi>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bt, int ldb,
                                          Epi epi) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    float c[NT][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const __nv_bfloat16* Ar = A + (mt * 16 + g) * lda + ks * 16 + 2 * tq;
      const uint32_t a[4] = {ld32(Ar), ld32(Ar + 8 * lda), ld32(Ar + 8), ld32(Ar + 8 * lda + 8)};
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const __nv_bfloat16* Br = Bt + (nt * 8 + g) * ldb + ks * 16 + 2 * tq;
        mma_16816(c[nt], a, ld32(Br), ld32(Br + 8));
      }
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int r0 = mt * 16 + g, c0 = nt * 8 + 2 * tq;
      epi(r0, c0, c[nt][0]);
      epi(r0, c0 + 1, c[nt][1]);
      epi(r0 + 8, c0, c[nt][2]);
      epi(r0 + 8, c0 + 1, c[nt][3]);
    }
  }
}

// Network weights staged in shared memory.
struct Weights {
  __nv_bfloat16 w2t[H * LDW]; // [unit][input]
  __nv_bfloat16 w3t[H * LDW];
  float w1[H * 2]; // [unit][input], BF16 values held as float
  float w4[H];
  float b1[H], b2[H], b3[H];
  float b4;
};

// Transposed copies for the backward pass (dA = dZ W): [input][unit].
struct WeightsT {
  __nv_bfloat16 w2n[H * LDW];
  __nv_bfloat16 w3n[H * LDW];
};

__device__ __forceinline__ float bf16_bits_to_float(uint16_t v) {
  return __uint_as_float(uint32_t(v) << 16);
}

// cooperative copy of the inference weights into shared memory (all threads of the block)
__device__ __forceinline__ void stage_weights(const pivot_mlp* net, Weights& W, WeightsT* WT) {
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
    const int n = i / H, k = i % H;
    const __nv_bfloat16 v2 = __ushort_as_bfloat16(net->w2[i]);
    const __nv_bfloat16 v3 = __ushort_as_bfloat16(net->w3[i]);
    W.w2t[n * LDW + k] = v2;
    W.w3t[n * LDW + k] = v3;
    if (WT) {
      WT->w2n[k * LDW + n] = v2;
      WT->w3n[k * LDW + n] = v3;
    }
  }
  for (int i = threadIdx.x; i < H * 2; i += blockDim.x) W.w1[i] = bf16_bits_to_float(net->w1[i]);
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    W.w4[i] = bf16_bits_to_float(net->w4[i]);
    W.b1[i] = net->b1[i];
    W.b2[i] = net->b2[i];
    W.b3[i] = net->b3[i];
  }
  if (threadIdx.x == 0) W.b4 = net->b4;
}

// Features of the normalised out-of-the-money problem b(x, s) = beta:
// f0 = |x|, f1 = q = 1/sqrt(-2 ln beta) (beta < b_max <= 1, so ln beta < 0),
// and the closed-form baseline s_a = |x| q + sqrt(2 pi) beta.
struct Features {
  float f0, f1;
  double sa;
};

__device__ __forceinline__ Features features(double x, double beta, double lnbeta) {
  Features f;
  const double q = rsqrt(-2.0 * lnbeta);
  f.f0 = float(-x);
  f.f1 = float(q);
  f.sa = fma(-x, q, 2.50662827463100050242 * beta);
  return f;
}

// Forward pass of the 32 rows of a warp with every activation in registers:
// the FP32 accumulator fragment of one m16n8k16 layer is the BF16 A fragment
// of the next (columns 2t, 2t+1 of n-tiles 2k and 2k+1 are k-tile k's
// a0/a1 and a2/a3 in the same lane), so no shared-memory tile is needed.
// Layer 1 (2 -> 64) is evaluated in FP32 directly in that layout, layer 4
// (64 -> 1) as a dot product reduced over the four lanes of a quad.  Same
// arithmetic as the forward half of train_warp up to the summation order of
// layer 4.
// Lane r holds row r's features and receives its output.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float forward_regs(float f0, float f1, const Weights& W) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
  float out = 0.0f;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = mt * 16 + g, r1 = r0 + 8;
    const float x00 = __shfl_sync(0xffffffffu, f0, r0), x01 = __shfl_sync(0xffffffffu, f1, r0);
    const float x10 = __shfl_sync(0xffffffffu, f0, r1), x11 = __shfl_sync(0xffffffffu, f1, r1);
    // layer 1 straight into the A fragments of layer 2
    uint32_t a[4][4];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int c = ks * 16 + half * 8 + 2 * tq;
        const float z00 = fmaf(W.w1[2 * c], x00, fmaf(W.w1[2 * c + 1], x01, W.b1[c]));
        const float z01 = fmaf(W.w1[2 * c + 2], x00, fmaf(W.w1[2 * c + 3], x01, W.b1[c + 1]));
        const float z10 = fmaf(W.w1[2 * c], x10, fmaf(W.w1[2 * c + 1], x11, W.b1[c]));
        const float z11 = fmaf(W.w1[2 * c + 2], x10, fmaf(W.w1[2 * c + 3], x11, W.b1[c + 1]));
        a[ks][2 * half] = pack_bf16(silu(z00), silu(z01));
        a[ks][2 * half + 1] = pack_bf16(silu(z10), silu(z11));
      }
    }
    // layers 2 and 3
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
      const __nv_bfloat16* Bt = layer == 0 ? W.w2t : W.w3t;
      const float* bias = layer == 0 ? W.b2 : W.b3;
      float c[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const __nv_bfloat16* Br = Bt + (nt * 8 + g) * LDW + ks * 16 + 2 * tq;
          mma_16816(c[nt], a[ks], ld32(Br), ld32(Br + 8));
        }
      }
      if (layer == 0) {
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          const int col = nt * 8 + 2 * tq;
          const int slot = (nt & 1) * 2;
          a[nt >> 1][slot] = pack_bf16(silu(c[nt][0] + bias[col]), silu(c[nt][1] + bias[col + 1]));
          a[nt >> 1][slot + 1] = pack_bf16(silu(c[nt][2] + bias[col]), silu(c[nt][3] + bias[col + 1]));
        }
      } else {
        // layer 4 on the BF16-rounded activations of layer 3
        float o0 = 0.0f, o1 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          const int col = nt * 8 + 2 * tq;
          const float w0 = W.w4[col], w1 = W.w4[col + 1];
          o0 = fmaf(w0, __bfloat162float(__float2bfloat16_rn(silu(c[nt][0] + bias[col]))), o0);
          o0 = fmaf(w1, __bfloat162float(__float2bfloat16_rn(silu(c[nt][1] + bias[col + 1]))), o0);
          o1 = fmaf(w0, __bfloat162float(__float2bfloat16_rn(silu(c[nt][2] + bias[col]))), o1);
          o1 = fmaf(w1, __bfloat162float(__float2bfloat16_rn(silu(c[nt][3] + bias[col + 1]))), o1);
        }
        o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
        o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
        o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
        o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
        // rows r0 (quad g) and r1 back to lane = row
        const int src = 4 * (lane & 7);
        const float v0 = __shfl_sync(0xffffffffu, o0, src);
        const float v1 = __shfl_sync(0xffffffffu, o1, src);
        const int within = lane - mt * 16;
        if (within >= 0 && within < 16) out = W.b4 + (within < 8 ? v0 : v1);
      }
    }
  }
  return out;
}

// Per-warp scratch of the training pass.
struct TrainTiles {
  __nv_bfloat16 RA[kRows * LDA], RB[kRows * LDA]; // row-major tiles
  __nv_bfloat16 TA[H * LDT], TB[H * LDT], TC[H * LDT]; // transposed tiles [unit][row]
  float Z2[kRows * H], Z3[kRows * H];                  // pre-activations, later their gradients
  float feat[kRows][2];
  float dO[kRows];
};

// Forward + backward of the 32 rows of a warp for the loss sum_r valid_r (o_r - y_r)^2;
// gradients are added to grad[] (global, FP32 atomics).  Returns this lane's squared error.
__device__ __forceinline__ float train_warp(float f0, float f1, float y, bool valid, const Weights& W,
                                            const WeightsT& WT, TrainTiles& S, float* grad) {
  const int lane = threadIdx.x & 31;
  S.feat[lane][0] = f0;
  S.feat[lane][1] = f1;
  // ---- forward, keeping what the backward needs
#pragma unroll 4
  for (int j = 0; j < H; ++j) {
    const float z = fmaf(W.w1[2 * j], f0, fmaf(W.w1[2 * j + 1], f1, W.b1[j]));
    const __nv_bfloat16 a = __float2bfloat16_rn(silu(z));
    S.RA[lane * LDA + j] = a;
    S.TA[j * LDT + lane] = a;
  }
  __syncwarp();
  warp_gemm<2, 8, 4>(S.RA, LDA, W.w2t, LDW, [&](int r, int c, float v) {
    const float z = v + W.b2[c];
    const __nv_bfloat16 a = __float2bfloat16_rn(silu(z));
    S.Z2[r * H + c] = z;
    S.RB[r * LDA + c] = a;
    S.TB[c * LDT + r] = a;
  });
  __syncwarp();
  warp_gemm<2, 8, 4>(S.RB, LDA, W.w3t, LDW, [&](int r, int c, float v) {
    const float z = v + W.b3[c];
    S.Z3[r * H + c] = z;
    S.RA[r * LDA + c] = __float2bfloat16_rn(silu(z));
  });
  __syncwarp();
  float o = W.b4;
#pragma unroll 8
  for (int k = 0; k < H; ++k) o = fmaf(W.w4[k], __bfloat162float(S.RA[lane * LDA + k]), o);
  const float err = valid ? (o - y) : 0.0f;
  const float dO = 2.0f * err;
  S.dO[lane] = dO;
  __syncwarp();
  // ---- output layer: dW4[k] = sum_r a3[r][k] dO[r], db4 = sum_r dO[r]
  for (int k = lane; k < H; k += 32) {
    float acc = 0.0f;
#pragma unroll 8
    for (int r = 0; r < kRows; ++r) acc = fmaf(__bfloat162float(S.RA[r * LDA + k]), S.dO[r], acc);
    atomicAdd(grad + OW4 + k, acc);
  }
  float db4 = dO;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) db4 += __shfl_xor_sync(0xffffffffu, db4, off);
  if (lane == 0) atomicAdd(grad + OB4, db4);
  // ---- dZ3 = dO w4 silu'(z3): FP32 into Z3, BF16 row-major into RB (a2 row-major is free), transposed into TC
#pragma unroll 4
  for (int k = 0; k < H; ++k) {
    const float d = dO * W.w4[k] * silu_grad(S.Z3[lane * H + k]);
    S.Z3[lane * H + k] = d;
    const __nv_bfloat16 db = __float2bfloat16_rn(d);
    S.RB[lane * LDA + k] = db;
    S.TC[k * LDT + lane] = db;
  }
  __syncwarp();
  for (int k = lane; k < H; k += 32) {
    float acc = 0.0f;
#pragma unroll 8
    for (int r = 0; r < kRows; ++r) acc += S.Z3[r * H + k];
    atomicAdd(grad + OB3 + k, acc);
  }
  // dW3[out][in] = sum_r a2[r][in] dZ3[r][out]: A = a2^T (TB [in][row]), Bt = dZ3^T (TC [out][row])
  warp_gemm<4, 8, 2>(S.TB, LDT, S.TC, LDT, [&](int in, int out, float v) { atomicAdd(grad + OW3 + out * H + in, v); });
  __syncwarp();
  // dA2[r][in] = sum_out dZ3[r][out] w3[out][in]: A = dZ3 (RB), Bt = w3 as [in][out] (WT.w3n)
  warp_gemm<2, 8, 4>(S.RB, LDA, WT.w3n, LDW, [&](int r, int in, float v) {
    const float d = v * silu_grad(S.Z2[r * H + in]);
    S.Z2[r * H + in] = d;
    const __nv_bfloat16 db = __float2bfloat16_rn(d);
    S.RA[r * LDA + in] = db;
    S.TB[in * LDT + r] = db;
  });
  __syncwarp();
  for (int k = lane; k < H; k += 32) {
    float acc = 0.0f;
#pragma unroll 8
    for (int r = 0; r < kRows; ++r) acc += S.Z2[r * H + k];
    atomicAdd(grad + OB2 + k, acc);
  }
  // dW2[out][in] = sum_r a1[r][in] dZ2[r][out]: A = a1^T (TA), Bt = dZ2^T (TB)
  warp_gemm<4, 8, 2>(S.TA, LDT, S.TB, LDT, [&](int in, int out, float v) { atomicAdd(grad + OW2 + out * H + in, v); });
  __syncwarp();
  // dA1[r][j] = sum_out dZ2[r][out] w2[out][j]; dZ1 = dA1 silu'(z1), z1 recomputed from the features
  warp_gemm<2, 8, 4>(S.RA, LDA, WT.w2n, LDW, [&](int r, int j, float v) {
    const float z = fmaf(W.w1[2 * j], S.feat[r][0], fmaf(W.w1[2 * j + 1], S.feat[r][1], W.b1[j]));
    S.Z3[r * H + j] = v * silu_grad(z);
  });
  __syncwarp();
  for (int j = lane; j < H; j += 32) {
    float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
#pragma unroll 8
    for (int r = 0; r < kRows; ++r) {
      const float d = S.Z3[r * H + j];
      g0 = fmaf(d, S.feat[r][0], g0);
      g1 = fmaf(d, S.feat[r][1], g1);
      gb += d;
    }
    atomicAdd(grad + OW1 + 2 * j, g0);
    atomicAdd(grad + OW1 + 2 * j + 1, g1);
    atomicAdd(grad + OB1 + j, gb);
  }
  __syncwarp();
  return err * err;
}

}  // namespace mlp
}  // namespace pivot

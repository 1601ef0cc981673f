// fv_mlp.cuh -- the learned starting guess of the exact Riemann solver's
// Newton iteration (Sec. 2.1 computes Godunov fluxes from the exact face
// Riemann problem; the paper has no learned component, so every choice here
// is a stated reading): a 6 -> 64 -> 64 -> 1 perceptron with tanh-form GELU
// activations predicts log(p*/pbar) (target 0) or log(p*/p_TR) / s(q)
// (target 1: the two-rarefaction guess's error in units of its weak-shock
// scale) from the face-frame primitives normalised by the pair's mean state.
//
// Inference is warp-collective and runs on the tensor cores with bfloat16
// operands and FP32 accumulation: a warp evaluates its 32 faces as two
// 16-row tiles, layer 1 as m16n8k8 (6 features padded to 8), layer 2 as
// m16n8k16 with layer 1's accumulator fragments re-packed in registers as
// its A fragments, the output layer as an FP32 dot product reduced across
// each quad.  Weights arrive pre-packed in fragment order (fv_mlp_pack) and
// are read from shared memory, one 32- or 64-bit word per lane per mma.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace fvk {

// parameter layout (FP32): W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3
enum : int {
  MLP_H = 64,
  MLP_NIN = 6,
  MP_W1 = 0,
  MP_B1 = MP_W1 + MLP_H * MLP_NIN,
  MP_W2 = MP_B1 + MLP_H,
  MP_B2 = MP_W2 + MLP_H * MLP_H,
  MP_W3 = MP_B2 + MLP_H,
  MP_B3 = MP_W3 + MLP_H,
  MLP_NPARAM = MP_B3 + 1,  // 4673
};

// packed layout (32-bit words): B fragments of W1 (8 n-tiles x 32 lanes),
// B fragments of W2 (4 k-steps x 8 n-tiles x 32 lanes x 2), then FP32
// b1, b2, w3, b3 and the target mode
enum : int {
  PK_W1 = 0,
  PK_W2 = PK_W1 + 8 * 32,
  PK_B1 = PK_W2 + 4 * 8 * 32 * 2,
  PK_B2 = PK_B1 + MLP_H,
  PK_W3 = PK_B2 + MLP_H,
  PK_B3 = PK_W3 + MLP_H,
  PK_TARGET = PK_B3 + 1,
  PK_GATE = PK_TARGET + 1,  // FP32 shock-strength threshold (negative: always)
  PK_WORDS = 2560,
};
static_assert(PK_GATE < PK_WORDS, "packed layout");

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// inference activation: the tanh form with the hardware tanh approximation
// (relative error near 2^-11, below bfloat16's 2^-8 resolution)
template <bool EXACT = false>
__device__ __forceinline__ float gelu_infer(float x) {
  float u = 0.7978845608028654f * (x + 0.044715f * (x * x * x));
  return 0.5f * x * (1.0f + (EXACT ? tanhf(u) : tanh_fast(u)));
}

__device__ __forceinline__ void mma_k8(float c[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_k16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// features of a face-frame pair: the left and right states normalised by
// the pair's mean state (rb, ub, pb the means, ab = sqrt(gamma pb / rb)),
// x = ((rL-rb)/rb, (uL-ub)/ab, (pL-pb)/pb, (rR-rb)/rb, (uR-ub)/ab, (pR-pb)/pb),
// computed in the path's precision T as differences (bfloat16 then keeps
// 2^-9 of a small jump); returns pb
template <typename T>
__device__ __forceinline__ float mlp_features(T gamma, T rL, T uL, T pL, T rR, T uR, T pR, float x[6]) {
  const T rs = rL + rR, ps = pL + pR;
  const T dr = (rL - rR) / rs, dp = (pL - pR) / ps;
  const T du = (uL - uR) / (T(2) * sqrt(gamma * ps / rs));
  x[0] = (float)dr;
  x[1] = (float)du;
  x[2] = (float)dp;
  x[3] = (float)-dr;
  x[4] = (float)-du;
  x[5] = (float)-dp;
  return (float)(T(0.5) * ps);
}

// scale of the two-rarefaction guess's error, s(q) = (q / (1 + q))^3 for
// q > 0 (third order for weak shocks, bounded for strong ones), else 0
__device__ __forceinline__ float shock_scale(float q) {
  if (!(q > 0.0f)) return 0.0f;
  float r = q / (1.0f + q);
  return r * r * r;
}

// shock strength of a pair by the two-rarefaction estimate, in FP32 with the
// hardware exp2/log2: q = p_TR / min(pL, pR) - 1.  The estimate is exact when
// both waves are rarefactions (q <= 0) and accurate to third order in the
// jump for weak shocks, so the network is consulted only where q exceeds the
// packed gate.
__device__ __forceinline__ float shock_strength(float gamma, float rL, float uL, float pL, float rR,
                                                float uR, float pR) {
  const float z = (gamma - 1.0f) / (2.0f * gamma);
  float aL = sqrtf(gamma * pL / rL), aR = sqrtf(gamma * pR / rR);
  float num = aL + aR - 0.5f * (gamma - 1.0f) * (uR - uL);
  float den = aL * exp2f(-z * __log2f(pL)) + aR * exp2f(-z * __log2f(pR));
  float ptr = exp2f(__log2f(fmaxf(num, 0.0f) / den) / z);
  return ptr / fminf(pL, pR) - 1.0f;
}

// the network output for this lane's features; every lane of the warp must
// call it together (mma.sync and full-mask shuffles).  sw: packed weights.
// The two 16-face tiles go one after the other, which halves the live
// fragments (the weights are read from shared memory once per tile).
// EXACT: the library's correctly rounded-ish tanhf in the activations
// instead of the hardware approximation (the check that separates the
// approximation's error from the bfloat16 quantisation; not used in flux
// kernels)
template <bool EXACT = false>
__device__ __forceinline__ float mlp_eval_warp(const uint32_t *__restrict__ sw, const float x[6]) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t q0 = pack_bf16x2(x[0], x[1]), q1 = pack_bf16x2(x[2], x[3]),
                 q2 = pack_bf16x2(x[4], x[5]);
  const float *b1 = reinterpret_cast<const float *>(sw + PK_B1);
  const float *b2 = reinterpret_cast<const float *>(sw + PK_B2);
  const float *w3 = reinterpret_cast<const float *>(sw + PK_W3);
  const uint2 *w2 = reinterpret_cast<const uint2 *>(sw + PK_W2);
  float yr00 = 0.f, yr01 = 0.f, yr10 = 0.f, yr11 = 0.f;  // [tile][row g / g+8]
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    // layer-1 A fragment (m16n8k8): rows g and g+8 of the tile hold the
    // features of faces 16 mt + g and 16 mt + 8 + g, columns 2t, 2t+1
    uint32_t a1f[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int src = 16 * mt + 8 * h + g;
      uint32_t s0 = __shfl_sync(FULL, q0, src), s1 = __shfl_sync(FULL, q1, src),
               s2 = __shfl_sync(FULL, q2, src);
      a1f[h] = t == 0 ? s0 : t == 1 ? s1 : t == 2 ? s2 : 0u;
    }
    // layer 1 + GELU, re-packed as the A fragments of layer 2: n-tile j
    // (hidden units 8j..8j+7) fills k-step j/2, registers 0/1 (j even) or
    // 2/3 (j odd), rows g / g+8
    uint32_t a2f[4][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float c0 = b1[8 * j + 2 * t], c1 = b1[8 * j + 2 * t + 1];
      float c[4] = {c0, c1, c0, c1};
      mma_k8(c, a1f[0], a1f[1], sw[PK_W1 + j * 32 + lane]);
      a2f[j >> 1][(j & 1) * 2 + 0] = pack_bf16x2(gelu_infer<EXACT>(c[0]), gelu_infer<EXACT>(c[1]));
      a2f[j >> 1][(j & 1) * 2 + 1] = pack_bf16x2(gelu_infer<EXACT>(c[2]), gelu_infer<EXACT>(c[3]));
    }
    // layer 2 + GELU + the output layer's partial dot products
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float c0 = b2[8 * j + 2 * t], c1 = b2[8 * j + 2 * t + 1];
      float c[4] = {c0, c1, c0, c1};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint2 bw = w2[(kk * 8 + j) * 32 + lane];
        mma_k16(c, a2f[kk], bw.x, bw.y);
      }
      const float v0 = w3[8 * j + 2 * t], v1 = w3[8 * j + 2 * t + 1];
      y0 += gelu_infer<EXACT>(c[0]) * v0 + gelu_infer<EXACT>(c[1]) * v1;
      y1 += gelu_infer<EXACT>(c[2]) * v0 + gelu_infer<EXACT>(c[3]) * v1;
    }
    y0 += __shfl_xor_sync(FULL, y0, 1);
    y0 += __shfl_xor_sync(FULL, y0, 2);
    y1 += __shfl_xor_sync(FULL, y1, 1);
    y1 += __shfl_xor_sync(FULL, y1, 2);
    if (mt == 0) {
      yr00 = y0;
      yr01 = y1;
    } else {
      yr10 = y0;
      yr11 = y1;
    }
  }
  // face `lane` is row 16 mt + 8 h + g with (mt, h) = (lane >> 4, (lane >> 3) & 1),
  // held by lane 4 (lane & 7)
  const int src = 4 * (lane & 7), which = lane >> 3;
  float v0 = __shfl_sync(FULL, yr00, src), v1 = __shfl_sync(FULL, yr01, src),
        v2 = __shfl_sync(FULL, yr10, src), v3 = __shfl_sync(FULL, yr11, src);
  float y = which == 0 ? v0 : which == 1 ? v1 : which == 2 ? v2 : v3;
  return y + __int_as_float((int)sw[PK_B3]);
}

// stage the packed weights of global memory into shared memory (whole block)
__device__ __forceinline__ void mlp_stage(uint32_t *sw, const uint32_t *__restrict__ gw) {
  for (int i = threadIdx.x; i < PK_WORDS / 4; i += blockDim.x)
    reinterpret_cast<uint4 *>(sw)[i] = reinterpret_cast<const uint4 *>(gw)[i];
  __syncthreads();
}

}  // namespace fvk

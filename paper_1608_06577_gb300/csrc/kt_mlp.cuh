// kt_mlp.cuh -- the learned start of the T^{tau mu} -> e root-find (device side).
//
// A 6 -> 32 -> 32 -> 1 ReLU network predicts z, the correction y = 10 ln(e / e_conf) = r^2 z of
// the conformal closed-form root e_conf = sqrt(4E^2 - 3M^2) - E of Sec. 2.4 (r^2 = M^2/E^2), for
// cells with r^2 > kMlpGateR2 (below it y = 0).  Inference runs inside the first stage's update
// kernel with warp-level BF16 tensor-core MMAs (FP32 accumulation); the second stage applies the
// same z to its own features.  The Newton steps that follow and the residual test are FP64.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "kt_device.cuh"

namespace kt {

constexpr int MLP_IN = 6, MLP_H = 32;
constexpr float kMlpGateR2 = 1e-3f;  // r^2 above which the network's correction is applied
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;  // 1313
constexpr int OFF_W1 = 0, OFF_B1 = 192, OFF_W2 = 224, OFF_B2 = 1248, OFF_W3 = 1280, OFF_B3 = 1312;

// packed inference weights (32-bit words): W1 [32 rows][4 words of bf16x2, k 0..7, k >= 6 zero],
// W2 [32 rows][20 words, 16 used: the pad keeps the fragment loads free of bank conflicts],
// W3 [16 words], then the FP32 biases b1[32], b2[32], b3
constexpr int PK_W1 = 0, PK_W2 = 128, PK_W3 = 128 + 640, PK_B1 = PK_W3 + 16, PK_B2 = PK_B1 + 32,
              PK_B3 = PK_B2 + 32, PK_WORDS = PK_B3 + 1;
constexpr int PK_W2_STRIDE = 20;

// Features of one cell from E = T^tt - pi^tt, M^2 and Pi (FP32), with fixed physics scalings.
// Also returns e_conf / E.
__device__ __forceinline__ void mlp_features(float E, float M2, float Pi, float (&x)[MLP_IN], float& econf_over_E) {
  const float iE = __fdividef(1.f, E);
  float r2 = fminf(fmaxf(M2 * iE * iE, 0.f), 0.999999f);
  float r = sqrtf(r2);
  float ec = __fdividef(3.f * (1.f - r) * (1.f + r), sqrtf(4.f - 3.f * r2) + 1.f);
  x[0] = (__logf(E) - 1.f) * (1.f / 6.f);
  x[1] = r2;
  x[2] = 5.f * Pi * iE;
  x[3] = 0.5f * __logf(1.f - r2);
  x[4] = ec;
  x[5] = r;
  econf_over_E = ec;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
// ReLU and the rounding to BF16 in one conversion: max(x, 0) rounded to nearest (a negative x
// gives zero); lo in the low half
__device__ __forceinline__ uint32_t pack_relu_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// the biases of output columns 2t, 2t + 1 (one 8-byte shared-memory load; w is 16-byte aligned)
__device__ __forceinline__ float2 bias_pair(const uint32_t* w, int off) {
  return *reinterpret_cast<const float2*>(w + off);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Inference for the 32 cells of a warp (lane = cell); all 32 lanes must call it together.
// w: packed weights (shared memory, 16-byte aligned).  Fragment layouts are those of mma.m16n8k16: lane =
// 4 g + t holds rows g, g+8 and columns 2t, 2t+1 (+8) of A and C, and B rows 2t, 2t+1 (+8),
// column g.  The C fragments of one layer are the A fragments of the next.
__device__ __forceinline__ float mlp_warp_infer(const uint32_t* __restrict__ w, const float (&x)[MLP_IN]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t p0 = pack_bf16x2(x[0], x[1]), p1 = pack_bf16x2(x[2], x[3]), p2 = pack_bf16x2(x[4], x[5]);
  uint32_t a1f[2][2];  // layer-1 A: [m-tile][row half], columns 2t, 2t+1 (k >= 8 is zero)
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int src = mt * 16 + g + 8 * h;
      uint32_t w0 = __shfl_sync(full, p0, src), w1 = __shfl_sync(full, p1, src), w2 = __shfl_sync(full, p2, src);
      a1f[mt][h] = (t == 0) ? w0 : ((t == 1) ? w1 : ((t == 2) ? w2 : 0u));
    }
  // layer 1: [32 x 8(k)] x [8 x 32] + b1, ReLU
  uint32_t a2f[2][2][4];  // layer-2 A: [m-tile][k-step][4]
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const uint32_t b0 = w[PK_W1 + (nt * 8 + g) * 4 + t];
    const float2 bi = bias_pair(w, PK_B1 + nt * 8 + 2 * t);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      float c[4] = {bi.x, bi.y, bi.x, bi.y};
      mma_bf16_16816(c, a1f[mt][0], a1f[mt][1], 0u, 0u, b0, 0u);
      const uint32_t lo = pack_relu_bf16x2(c[0], c[1]);
      const uint32_t hi = pack_relu_bf16x2(c[2], c[3]);
      const int ks = nt >> 1, half = nt & 1;
      a2f[mt][ks][half * 2 + 0] = lo;
      a2f[mt][ks][half * 2 + 1] = hi;
    }
  }
  // layer 2: [32 x 32] x [32 x 32] + b2, ReLU
  uint32_t a3f[2][2][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const float2 bi = bias_pair(w, PK_B2 + nt * 8 + 2 * t);
    float c[2][4] = {{bi.x, bi.y, bi.x, bi.y}, {bi.x, bi.y, bi.x, bi.y}};
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const uint32_t b0 = w[PK_W2 + (nt * 8 + g) * PK_W2_STRIDE + ks * 8 + t];
      const uint32_t b1 = w[PK_W2 + (nt * 8 + g) * PK_W2_STRIDE + ks * 8 + 4 + t];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        mma_bf16_16816(c[mt], a2f[mt][ks][0], a2f[mt][ks][1], a2f[mt][ks][2], a2f[mt][ks][3], b0, b1);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int ks = nt >> 1, half = nt & 1;
      a3f[mt][ks][half * 2 + 0] = pack_relu_bf16x2(c[mt][0], c[mt][1]);
      a3f[mt][ks][half * 2 + 1] = pack_relu_bf16x2(c[mt][2], c[mt][3]);
    }
  }
  // layer 3: [32 x 32] x [32 x 8 (column 0 used)] + b3
  const float b3 = __uint_as_float(w[PK_B3]);
  float c3[2][4] = {{b3, b3, b3, b3}, {b3, b3, b3, b3}};
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const uint32_t b0 = (g == 0) ? w[PK_W3 + ks * 8 + t] : 0u;
    const uint32_t b1 = (g == 0) ? w[PK_W3 + ks * 8 + 4 + t] : 0u;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
      mma_bf16_16816(c3[mt], a3f[mt][ks][0], a3f[mt][ks][1], a3f[mt][ks][2], a3f[mt][ks][3], b0, b1);
  }
  // column 0 of row r of m-tile mt sits in lane 4 (r mod 8), register 0 (r < 8) or 2
  const int mt = lane >> 4, r = lane & 15, src = 4 * (r & 7);
  const float v00 = __shfl_sync(full, c3[0][0], src), v02 = __shfl_sync(full, c3[0][2], src);
  const float v10 = __shfl_sync(full, c3[1][0], src), v12 = __shfl_sync(full, c3[1][2], src);
  return (mt == 0) ? ((r < 8) ? v00 : v02) : ((r < 8) ? v10 : v12);
}

// FP32 parameters -> packed inference weights (one block; defined in kt_mlp.cu)
__global__ void mlp_pack_kernel(const float* __restrict__ params, uint32_t* packed);

// copy the packed weights into shared memory (whole block)
__device__ __forceinline__ void mlp_load_shared(uint32_t* sm, const uint32_t* __restrict__ packed) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  for (int i = tid; i < PK_WORDS; i += nt) sm[i] = packed[i];
}

}  // namespace kt

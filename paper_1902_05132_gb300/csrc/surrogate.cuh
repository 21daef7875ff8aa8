// Learned surrogate of the reaction components (mixed + surrogate form).
//
// One small MLP per reaction component (l, l', a, b) stands in for the
// Sommerfeld integral u^{ab}_{l l'}(rho, zt, zs) of eq. generalcomponentsimag
// (after the alpha integral): zt is the target's distance to the reference
// interface of arrow a, zs the image depth of arrow b.  The network maps the
// box-normalized inputs to y = 4 pi R u, R = sqrt(rho^2 + (zt + zs)^2) the
// distance to the image point, which removes the 1/R decay and leaves an
// O(1) smooth function.  Architecture: 3 -> 64 -> 64 -> 64 -> 2, GELU;
// weights and layer inputs rounded to BF16, products accumulated in FP32.
// The quadrature stays the reference: a held-out check per cell of a
// 4 x 4 x 4 grid over the input box decides where the surrogate may be used.
#pragma once
#include <cuda_bf16.h>

#define SURR_H 64
#define SURR_NPAR (SURR_H * 3 + SURR_H + SURR_H * SURR_H + SURR_H + SURR_H * SURR_H + SURR_H + 2 * SURR_H + 2)
#define SURR_CELLS 64
// parameter offsets: W1 [64][3], b1, W2 [64][64], b2, W3 [64][64], b3, W4 [2][64], b4
#define SURR_W1 0
#define SURR_B1 (SURR_W1 + SURR_H * 3)
#define SURR_W2 (SURR_B1 + SURR_H)
#define SURR_B2 (SURR_W2 + SURR_H * SURR_H)
#define SURR_W3 (SURR_B2 + SURR_H)
#define SURR_B3 (SURR_W3 + SURR_H * SURR_H)
#define SURR_W4 (SURR_B3 + SURR_H)
#define SURR_B4 (SURR_W4 + 2 * SURR_H)

// Box of the inputs and the trained networks (device pointers; w == nullptr:
// no surrogate).
struct SurrView {
  const __nv_bfloat16* w;           // [slot][SURR_NPAR], slot = ((l L1 + l') 2 + a) 2 + b
  const unsigned char* ok;          // [slot][SURR_CELLS]: held-out error within the bound
  double rho_max, z_min, z_max;
};

// Counter-based generator (the splitmix64 finalizer applied to seed + counter):
// uniform double in [0, 1) for draw `i` of stream `seed`.
__host__ __device__ inline unsigned long long surr_mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__host__ __device__ inline double surr_uniform(unsigned long long seed, long i) {
  return (double)(surr_mix64(seed * 0x632BE59BD9B4E019ULL + (unsigned long long)i) >> 11) * (1.0 / 9007199254740992.0);
}

__host__ __device__ inline float surr_gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__host__ __device__ inline float surr_gelu_d(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}
__device__ inline float surr_bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// normalized inputs in [-1, 1] and the cell of a point (false if outside the box)
__device__ inline bool surr_inputs(const SurrView& S, double rho, double zt, double zs, float* x, int* cell) {
  if (!(rho >= 0.0 && rho <= S.rho_max && zt >= S.z_min && zt <= S.z_max && zs >= S.z_min && zs <= S.z_max))
    return false;
  double u0 = rho / S.rho_max, u1 = (zt - S.z_min) / (S.z_max - S.z_min), u2 = (zs - S.z_min) / (S.z_max - S.z_min);
  x[0] = (float)(2.0 * u0 - 1.0);
  x[1] = (float)(2.0 * u1 - 1.0);
  x[2] = (float)(2.0 * u2 - 1.0);
  int c0 = min(3, (int)(u0 * 4.0)), c1 = min(3, (int)(u1 * 4.0)), c2 = min(3, (int)(u2 * 4.0));
  *cell = (c0 * 4 + c1) * 4 + c2;
  return true;
}

// Forward pass of one network for one input (BF16 weights from global memory,
// FP32 accumulation, layer inputs rounded to BF16 as in training).
__device__ inline float2 surr_forward(const __nv_bfloat16* __restrict__ W, const float* x) {
  float a[SURR_H], b[SURR_H];
#pragma unroll 4
  for (int j = 0; j < SURR_H; ++j) {
    float s = __bfloat162float(W[SURR_B1 + j]);
    for (int i = 0; i < 3; ++i) s = fmaf(__bfloat162float(W[SURR_W1 + j * 3 + i]), surr_bf(x[i]), s);
    a[j] = surr_bf(surr_gelu(s));
  }
  for (int j = 0; j < SURR_H; ++j) {
    float s = __bfloat162float(W[SURR_B2 + j]);
    const __nv_bfloat16* wr = W + SURR_W2 + j * SURR_H;
#pragma unroll 16
    for (int i = 0; i < SURR_H; ++i) s = fmaf(__bfloat162float(wr[i]), a[i], s);
    b[j] = surr_bf(surr_gelu(s));
  }
  for (int j = 0; j < SURR_H; ++j) {
    float s = __bfloat162float(W[SURR_B3 + j]);
    const __nv_bfloat16* wr = W + SURR_W3 + j * SURR_H;
#pragma unroll 16
    for (int i = 0; i < SURR_H; ++i) s = fmaf(__bfloat162float(wr[i]), b[i], s);
    a[j] = surr_bf(surr_gelu(s));
  }
  float o[2];
  for (int k = 0; k < 2; ++k) {
    float s = __bfloat162float(W[SURR_B4 + k]);
    const __nv_bfloat16* wr = W + SURR_W4 + k * SURR_H;
#pragma unroll 16
    for (int i = 0; i < SURR_H; ++i) s = fmaf(__bfloat162float(wr[i]), a[i], s);
    o[k] = s;
  }
  return make_float2(o[0], o[1]);
}

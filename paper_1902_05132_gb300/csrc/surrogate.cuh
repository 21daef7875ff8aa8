// Learned surrogate of the reaction components (mixed + surrogate form).
//
// One small MLP per reaction component (l, l', a, b) stands in for the
// Sommerfeld integral u^{ab}_{l l'}(rho, zt, zs) of eq. generalcomponentsimag
// (after the alpha integral): zt is the target's distance to the reference
// interface of arrow a, zs the image depth of arrow b.  The network maps the
// box-normalized inputs to y = 4 pi R u, R = sqrt(rho^2 + (zt + zs)^2) the
// distance to the image point, which removes the 1/R decay and leaves an
// O(1) smooth function.  Architecture: 3 -> 64 -> 64 -> 64 (GELU), then a
// linear output layer 64 -> 2 (Re, Im) chosen by the cell of an 8 x 8 x 8 grid
// over the input box.
//  * Training: the three hidden layers and a shared output layer by Adam on
//    the standardized outputs (weights and layer inputs rounded to BF16, FP32
//    accumulation); then the output layer of every cell by ridge-regularized
//    least squares (FP64 normal equations over that cell's training samples,
//    features from the inference arithmetic below).
//  * Inference: every weight and layer input carried as a BF16 hi/lo pair
//    (x = hi + lo, a 16-bit significand), FP32 multiply-accumulate.
// The quadrature stays the reference: a held-out check per cell decides where
// the surrogate may be used.
#pragma once
#include <cuda_bf16.h>

#define SURR_H 64
#define SURR_NPAR (SURR_H * 3 + SURR_H + SURR_H * SURR_H + SURR_H + SURR_H * SURR_H + SURR_H + 2 * SURR_H + 2)
#define SURR_GRID 8                    // cells per input axis
#define SURR_CELLS (SURR_GRID * SURR_GRID * SURR_GRID)
// parameter offsets: W1 [64][3], b1, W2 [64][64], b2, W3 [64][64], b3, W4 [2][64], b4
#define SURR_W1 0
#define SURR_B1 (SURR_W1 + SURR_H * 3)
#define SURR_W2 (SURR_B1 + SURR_H)
#define SURR_B2 (SURR_W2 + SURR_H * SURR_H)
#define SURR_W3 (SURR_B2 + SURR_H)
#define SURR_B3 (SURR_W3 + SURR_H * SURR_H)
#define SURR_W4 (SURR_B3 + SURR_H)
#define SURR_B4 (SURR_W4 + 2 * SURR_H)
// inference parameters of one component: the hidden layers (W1 .. b3), then
// one output layer per cell, [cell][k][65] (64 weights and the bias of
// output k); stored twice, BF16 hi parts then BF16 lo parts
#define SURR_NTRUNK SURR_W4
#define SURR_HEAD_N (SURR_H + 1)
#define SURR_NHEAD (SURR_CELLS * 2 * SURR_HEAD_N)
#define SURR_NINF (SURR_NTRUNK + SURR_NHEAD)

// Box of the inputs and the trained networks (device pointers; w == nullptr:
// no surrogate).
struct SurrView {
  const __nv_bfloat16* w;           // [slot][2][SURR_NINF], slot = ((l L1 + l') 2 + a) 2 + b
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
  const int g = SURR_GRID;
  int c0 = min(g - 1, (int)(u0 * g)), c1 = min(g - 1, (int)(u1 * g)), c2 = min(g - 1, (int)(u2 * g));
  *cell = (c0 * g + c1) * g + c2;
  return true;
}

// The value a BF16 hi/lo pair carries: hi = bf16(x), lo = bf16(x - hi).
__device__ inline float surr_hilo(float x) {
  float h = surr_bf(x);
  return h + surr_bf(x - h);
}
__device__ inline float surr_w(const __nv_bfloat16* __restrict__ hi, const __nv_bfloat16* __restrict__ lo, int i) {
  return __bfloat162float(hi[i]) + __bfloat162float(lo[i]);
}

// Hidden layers of one network for one input (inference arithmetic):
// f[0..63] = GELU(W3 GELU(W2 GELU(W1 x + b1) + b2) + b3), every operand a
// BF16 hi/lo pair, FP32 accumulation.  `hi` and `lo` point at the component's
// inference parameters.
__device__ inline void surr_features(const __nv_bfloat16* __restrict__ hi, const __nv_bfloat16* __restrict__ lo,
                                     const float* x, float* f) {
  float a[SURR_H];
  float xi[3] = {surr_hilo(x[0]), surr_hilo(x[1]), surr_hilo(x[2])};
#pragma unroll 4
  for (int j = 0; j < SURR_H; ++j) {
    float s = surr_w(hi, lo, SURR_B1 + j);
    for (int i = 0; i < 3; ++i) s = fmaf(surr_w(hi, lo, SURR_W1 + j * 3 + i), xi[i], s);
    a[j] = surr_hilo(surr_gelu(s));
  }
  for (int j = 0; j < SURR_H; ++j) {
    float s = surr_w(hi, lo, SURR_B2 + j);
    const int r = SURR_W2 + j * SURR_H;
#pragma unroll 16
    for (int i = 0; i < SURR_H; ++i) s = fmaf(surr_w(hi, lo, r + i), a[i], s);
    f[j] = surr_hilo(surr_gelu(s));
  }
  for (int j = 0; j < SURR_H; ++j) {
    float s = surr_w(hi, lo, SURR_B3 + j);
    const int r = SURR_W3 + j * SURR_H;
#pragma unroll 16
    for (int i = 0; i < SURR_H; ++i) s = fmaf(surr_w(hi, lo, r + i), f[i], s);
    a[j] = surr_hilo(surr_gelu(s));
  }
  for (int j = 0; j < SURR_H; ++j) f[j] = a[j];
}

// The same forward pass with the hidden layers already summed to FP32 (hi +
// lo, exact) and laid out as in the inference parameters (e.g. staged in
// shared memory); the cell's output layer is read from the component's
// inference parameters `W` (hi and lo parts).  Same operations in the same
// order as surr_forward: bit-identical results.  Fully unrolled so that the
// layer activations stay in registers.
__device__ __forceinline__ float2 surr_forward_f32(const float* __restrict__ w, const __nv_bfloat16* __restrict__ W,
                                                   const float* x, int cell) {
  float a[SURR_H], f[SURR_H];
  const float xi0 = surr_hilo(x[0]), xi1 = surr_hilo(x[1]), xi2 = surr_hilo(x[2]);
#pragma unroll
  for (int j = 0; j < SURR_H; ++j) {
    float s = w[SURR_B1 + j];
    s = fmaf(w[SURR_W1 + j * 3 + 0], xi0, s);
    s = fmaf(w[SURR_W1 + j * 3 + 1], xi1, s);
    s = fmaf(w[SURR_W1 + j * 3 + 2], xi2, s);
    a[j] = surr_hilo(surr_gelu(s));
  }
#pragma unroll
  for (int j = 0; j < SURR_H; ++j) {
    float s = w[SURR_B2 + j];
    const float4* r = reinterpret_cast<const float4*>(w + SURR_W2 + j * SURR_H);
#pragma unroll
    for (int i = 0; i < SURR_H / 4; ++i) {
      const float4 v = r[i];
      s = fmaf(v.x, a[4 * i], s);
      s = fmaf(v.y, a[4 * i + 1], s);
      s = fmaf(v.z, a[4 * i + 2], s);
      s = fmaf(v.w, a[4 * i + 3], s);
    }
    f[j] = surr_hilo(surr_gelu(s));
  }
#pragma unroll
  for (int j = 0; j < SURR_H; ++j) {
    float s = w[SURR_B3 + j];
    const float4* r = reinterpret_cast<const float4*>(w + SURR_W3 + j * SURR_H);
#pragma unroll
    for (int i = 0; i < SURR_H / 4; ++i) {
      const float4 v = r[i];
      s = fmaf(v.x, f[4 * i], s);
      s = fmaf(v.y, f[4 * i + 1], s);
      s = fmaf(v.z, f[4 * i + 2], s);
      s = fmaf(v.w, f[4 * i + 3], s);
    }
    a[j] = surr_hilo(surr_gelu(s));
  }
  const __nv_bfloat16* hi = W;
  const __nv_bfloat16* lo = W + SURR_NINF;
  float o[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r = SURR_NTRUNK + (cell * 2 + k) * SURR_HEAD_N;
    float s = surr_w(hi, lo, r + SURR_H);
#pragma unroll
    for (int i = 0; i < SURR_H; ++i) s = fmaf(surr_w(hi, lo, r + i), a[i], s);
    o[k] = s;
  }
  return make_float2(o[0], o[1]);
}

// Forward pass of one component's network for one input in `cell`.
__device__ inline float2 surr_forward(const __nv_bfloat16* __restrict__ W, const float* x, int cell) {
  const __nv_bfloat16* hi = W;
  const __nv_bfloat16* lo = W + SURR_NINF;
  float f[SURR_H];
  surr_features(hi, lo, x, f);
  float o[2];
  for (int k = 0; k < 2; ++k) {
    const int r = SURR_NTRUNK + (cell * 2 + k) * SURR_HEAD_N;
    float s = surr_w(hi, lo, r + SURR_H);
#pragma unroll 16
    for (int i = 0; i < SURR_H; ++i) s = fmaf(surr_w(hi, lo, r + i), f[i], s);
    o[k] = s;
  }
  return make_float2(o[0], o[1]);
}

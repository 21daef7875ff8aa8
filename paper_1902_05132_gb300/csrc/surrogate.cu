// Training of the learned surrogate of the reaction components
// (fmm_layered_surrogate_train) and its held-out check.
//
// Data: for every reaction component of the medium, points drawn uniformly in
// the box [0, rho_max] x [z_min, z_max]^2 of (rho, zt, zs) with the values of
// the component computed by the library's quadrature (the plain path of the
// near field, eq. generalcomponentsimag), plus an independent held-out set.
// Training: all components at once, minibatches of 1024 points per component
// and step; one CTA runs forward and backward for 32 points (weights and layer
// inputs rounded to BF16, FP32 products and sums) and writes its partial
// gradients; a second kernel adds the partials of a component in a fixed
// order and takes an Adam step on FP32 master weights, then rounds them to the
// BF16 copy that inference reads.  Loss: mean squared error of y = 4 pi R u.
// Check: relative RMS error of the held-out points of every cell of a
// 4 x 4 x 4 grid over the box; a cell is used only if it is within the bound.
#include <cmath>
#include <string>
#include <vector>

#include "fmm_internal.h"

namespace {

constexpr int kSB = 32;          // points per CTA
constexpr int kNCH = 32;         // CTAs per component and step: minibatch 1024
constexpr int kTPB = 128;
constexpr int kNP = SURR_NPAR;

// Forward and backward of one CTA's points; partial gradients to gpart.
__global__ void __launch_bounds__(kTPB) k_surr_train(const float* __restrict__ X, const float* __restrict__ Y,
                                                    long nper, const float* __restrict__ wf_all,
                                                    float* __restrict__ gpart, unsigned long long seed, int step) {
  const int si = blockIdx.y, ch = blockIdx.x, H = SURR_H;
  const float* wf = wf_all + (long)si * kNP;
  extern __shared__ float sm[];
  float* W = sm;                               // kNP, BF16-rounded
  float* xs = W + kNP;                         // [kSB][3]
  float* ys = xs + kSB * 3;                    // [kSB][2], then the output gradient
  float* h1 = ys + kSB * 2;
  float* a1 = h1 + kSB * H;
  float* h2 = a1 + kSB * H;
  float* a2 = h2 + kSB * H;
  float* h3 = a2 + kSB * H;
  float* a3 = h3 + kSB * H;
  float* d = a3 + kSB * H;
  float* e = d + kSB * H;
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) W[i] = surr_bf(wf[i]);
  for (int s = threadIdx.x; s < kSB; s += blockDim.x) {
    unsigned long long r = surr_mix64(seed + (unsigned long long)step * 0x9E3779B97F4A7C15ULL +
                                      ((unsigned long long)si << 40) + (unsigned long long)(ch * kSB + s));
    long idx = (long)(r % (unsigned long long)nper) + (long)si * nper;
    for (int i = 0; i < 3; ++i) xs[s * 3 + i] = surr_bf(X[3 * idx + i]);
    for (int k = 0; k < 2; ++k) ys[s * 2 + k] = Y[2 * idx + k];
  }
  __syncthreads();
  // forward
  for (int q = threadIdx.x; q < kSB * H; q += blockDim.x) {
    int s = q / H, j = q % H;
    float v = W[SURR_B1 + j];
    for (int i = 0; i < 3; ++i) v = fmaf(W[SURR_W1 + j * 3 + i], xs[s * 3 + i], v);
    h1[q] = v;
    a1[q] = surr_bf(surr_gelu(v));
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kSB * H; q += blockDim.x) {
    int s = q / H, j = q % H;
    float v = W[SURR_B2 + j];
    for (int i = 0; i < H; ++i) v = fmaf(W[SURR_W2 + j * H + i], a1[s * H + i], v);
    h2[q] = v;
    a2[q] = surr_bf(surr_gelu(v));
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kSB * H; q += blockDim.x) {
    int s = q / H, j = q % H;
    float v = W[SURR_B3 + j];
    for (int i = 0; i < H; ++i) v = fmaf(W[SURR_W3 + j * H + i], a2[s * H + i], v);
    h3[q] = v;
    a3[q] = surr_bf(surr_gelu(v));
  }
  __syncthreads();
  const float inv_b = 1.0f / (float)(kSB * kNCH);
  for (int q = threadIdx.x; q < kSB * 2; q += blockDim.x) {
    int s = q / 2, k = q % 2;
    float v = W[SURR_B4 + k];
    for (int i = 0; i < H; ++i) v = fmaf(W[SURR_W4 + k * H + i], a3[s * H + i], v);
    ys[q] = 2.0f * (v - ys[q]) * inv_b;       // d loss / d output
  }
  __syncthreads();
  float* G = gpart + ((long)si * kNCH + ch) * kNP;
  // output layer gradients, delta of layer 3
  for (int p = threadIdx.x; p < 2 * H + 2; p += blockDim.x) {
    float g = 0.0f;
    if (p < 2 * H) {
      int k = p / H, i = p % H;
      for (int s = 0; s < kSB; ++s) g = fmaf(ys[s * 2 + k], a3[s * H + i], g);
      G[SURR_W4 + p] = g;
    } else {
      for (int s = 0; s < kSB; ++s) g += ys[s * 2 + (p - 2 * H)];
      G[SURR_B4 + p - 2 * H] = g;
    }
  }
  for (int q = threadIdx.x; q < kSB * H; q += blockDim.x) {
    int s = q / H, i = q % H;
    float v = W[SURR_W4 + i] * ys[s * 2] + W[SURR_W4 + H + i] * ys[s * 2 + 1];
    d[q] = v * surr_gelu_d(h3[q]);
  }
  __syncthreads();
  // layer 3 gradients, delta of layer 2
  for (int p = threadIdx.x; p < H * H + H; p += blockDim.x) {
    float g = 0.0f;
    if (p < H * H) {
      int j = p / H, i = p % H;
      for (int s = 0; s < kSB; ++s) g = fmaf(d[s * H + j], a2[s * H + i], g);
      G[SURR_W3 + p] = g;
    } else {
      int j = p - H * H;
      for (int s = 0; s < kSB; ++s) g += d[s * H + j];
      G[SURR_B3 + j] = g;
    }
  }
  for (int q = threadIdx.x; q < kSB * H; q += blockDim.x) {
    int s = q / H, i = q % H;
    float v = 0.0f;
    for (int j = 0; j < H; ++j) v = fmaf(W[SURR_W3 + j * H + i], d[s * H + j], v);
    e[q] = v * surr_gelu_d(h2[q]);
  }
  __syncthreads();
  // layer 2 gradients, delta of layer 1
  for (int p = threadIdx.x; p < H * H + H; p += blockDim.x) {
    float g = 0.0f;
    if (p < H * H) {
      int j = p / H, i = p % H;
      for (int s = 0; s < kSB; ++s) g = fmaf(e[s * H + j], a1[s * H + i], g);
      G[SURR_W2 + p] = g;
    } else {
      int j = p - H * H;
      for (int s = 0; s < kSB; ++s) g += e[s * H + j];
      G[SURR_B2 + j] = g;
    }
  }
  for (int q = threadIdx.x; q < kSB * H; q += blockDim.x) {
    int s = q / H, i = q % H;
    float v = 0.0f;
    for (int j = 0; j < H; ++j) v = fmaf(W[SURR_W2 + j * H + i], e[s * H + j], v);
    d[q] = v * surr_gelu_d(h1[q]);
  }
  __syncthreads();
  // layer 1 gradients
  for (int p = threadIdx.x; p < H * 3 + H; p += blockDim.x) {
    float g = 0.0f;
    if (p < H * 3) {
      int j = p / 3, i = p % 3;
      for (int s = 0; s < kSB; ++s) g = fmaf(d[s * H + j], xs[s * 3 + i], g);
      G[SURR_W1 + p] = g;
    } else {
      int j = p - H * 3;
      for (int s = 0; s < kSB; ++s) g += d[s * H + j];
      G[SURR_B1 + j] = g;
    }
  }
}

// Adam step: partial gradients added in CTA order (deterministic).
__global__ void k_surr_adam(long n, const int* __restrict__ slots, const float* __restrict__ gpart,
                            float* __restrict__ wf, float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ w16, float lr, float c1, float c2) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long si = i / kNP, p = i % kNP;
  float g = 0.0f;
  for (int c = 0; c < kNCH; ++c) g += gpart[(si * kNCH + c) * kNP + p];
  float mi = 0.9f * m[i] + 0.1f * g;
  float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  float w = wf[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  wf[i] = w;
  w16[(long)slots[si] * kNP + p] = __float2bfloat16_rn(w);
}

// Held-out errors: acc[(si * 64 + cell) * 3 + {0,1,2}] += |err|^2, |y|^2, 1
__global__ void k_surr_heldout(long n, long nper, const int* __restrict__ slots, const float* __restrict__ X,
                               const float* __restrict__ Y, const __nv_bfloat16* __restrict__ w16,
                               double* __restrict__ acc) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int si = (int)(e / nper);
  float x[3] = {X[3 * e], X[3 * e + 1], X[3 * e + 2]};
  float2 o = surr_forward(w16 + (long)slots[si] * kNP, x);
  float y0 = Y[2 * e], y1 = Y[2 * e + 1];
  int c[3];
  for (int i = 0; i < 3; ++i) c[i] = min(3, max(0, (int)((x[i] + 1.0f) * 2.0f)));
  int cell = (c[0] * 4 + c[1]) * 4 + c[2];
  double* a = acc + ((long)si * SURR_CELLS + cell) * 3;
  double dr = (double)o.x - y0, di = (double)o.y - y1;
  atomicAdd(a, dr * dr + di * di);
  atomicAdd(a + 1, (double)y0 * y0 + (double)y1 * y1);
  atomicAdd(a + 2, 1.0);
}

}  // namespace

void launch_coef(int L1, const Rule& R, cplx* coef, cudaStream_t st);
RuleView make_rule_view(const Rule& R, const cplx* coef);
void launch_surr_samples(long n, long nper, const int* slots, int L1, SurrView box, RuleView R,
                         unsigned long long seed, float* X, float* Y, cudaStream_t st);

static void surr_train_impl(fmm_layered* h, double rho_max, double z_min, double z_max, long nper, int steps,
                            double bound, unsigned long long seed, cudaStream_t st) {
  SurrState& S = h->surr;
  const int L1 = h->L1;
  std::vector<int> slots;
  for (int l = 0; l < L1; ++l)
    for (int lp = 0; lp < L1; ++lp)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          bool ok_a = (a == AR_UP) ? (l < L1 - 1) : (l > 0);
          bool ok_b = (b == AR_UP) ? (lp < L1 - 1) : (lp > 0);
          if (ok_a && ok_b) slots.push_back(((l * L1 + lp) * 2 + a) * 2 + b);
        }
  const int ns = (int)slots.size();
  const int nslot_all = L1 * L1 * 4;
  S.trained = false;
  // quadrature long enough for the smallest vertical distance zt + zs = 2 z_min
  rule_extend(h, h->rule.near_tmax(2.0 * z_min), st);
  const int Q = h->rule.Q();
  S.coef.ensure(sizeof(cplx) * (size_t)nslot_all * Q);
  launch_coef(L1, h->rule, S.coef.as<cplx>(), st);
  RuleView R = make_rule_view(h->rule, S.coef.as<cplx>());
  SurrView box{};
  box.rho_max = rho_max;
  box.z_min = z_min;
  box.z_max = z_max;
  S.slots.ensure(sizeof(int) * ns);
  FMM_CHECK(cudaMemcpyAsync(S.slots.ptr, slots.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  const long nh = std::max<long>(nper / 8, 256);
  S.X.ensure(sizeof(float) * 3 * (size_t)ns * nper);
  S.Y.ensure(sizeof(float) * 2 * (size_t)ns * nper);
  S.Xh.ensure(sizeof(float) * 3 * (size_t)ns * nh);
  S.Yh.ensure(sizeof(float) * 2 * (size_t)ns * nh);
  launch_surr_samples((long)ns * nper, nper, S.slots.as<int>(), L1, box, R, seed, S.X.as<float>(), S.Y.as<float>(), st);
  launch_surr_samples((long)ns * nh, nh, S.slots.as<int>(), L1, box, R, seed ^ 0x5DEECE66DULL, S.Xh.as<float>(),
                      S.Yh.as<float>(), st);
  FMM_CHECK(cudaGetLastError());
  // Glorot-uniform initial weights, zero biases
  const long npt = (long)ns * kNP;
  std::vector<float> w0((size_t)npt, 0.0f);
  auto init = [&](int si, int off, int fan_out, int fan_in) {
    double lim = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < fan_out * fan_in; ++i)
      w0[(size_t)si * kNP + off + i] = (float)((2.0 * surr_uniform(seed + 17 + si, off + i) - 1.0) * lim);
  };
  for (int si = 0; si < ns; ++si) {
    init(si, SURR_W1, SURR_H, 3);
    init(si, SURR_W2, SURR_H, SURR_H);
    init(si, SURR_W3, SURR_H, SURR_H);
    init(si, SURR_W4, 2, SURR_H);
  }
  S.wf.ensure(sizeof(float) * npt);
  S.m.ensure(sizeof(float) * npt);
  S.v.ensure(sizeof(float) * npt);
  S.w16.ensure(sizeof(__nv_bfloat16) * (size_t)nslot_all * kNP);
  S.gpart.ensure(sizeof(float) * (size_t)ns * kNCH * kNP);
  FMM_CHECK(cudaMemcpyAsync(S.wf.ptr, w0.data(), sizeof(float) * npt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemsetAsync(S.m.ptr, 0, sizeof(float) * npt, st));
  FMM_CHECK(cudaMemsetAsync(S.v.ptr, 0, sizeof(float) * npt, st));
  FMM_CHECK(cudaMemsetAsync(S.w16.ptr, 0, sizeof(__nv_bfloat16) * (size_t)nslot_all * kNP, st));
  const size_t smem = sizeof(float) * (kNP + kSB * 5 + 8 * kSB * SURR_H);
  FMM_CHECK(cudaFuncSetAttribute(k_surr_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  float c1 = 1.0f, c2 = 1.0f;
  for (int t = 0; t < steps; ++t) {
    LAUNCH(k_surr_train<<<dim3(kNCH, ns), kTPB, smem, st>>>(S.X.as<float>(), S.Y.as<float>(), nper, S.wf.as<float>(),
                                                             S.gpart.as<float>(), seed, t));
    c1 *= 0.9f;
    c2 *= 0.999f;
    const float lr = (float)(2e-3 * 0.5 * (1.0 + std::cos(M_PI * t / steps)) + 1e-5);
    LAUNCH(k_surr_adam<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(npt, S.slots.as<int>(), S.gpart.as<float>(),
                                                                      S.wf.as<float>(), S.m.as<float>(), S.v.as<float>(),
                                                                      S.w16.as<__nv_bfloat16>(), lr, 1.0f - c1, 1.0f - c2));
  }
  FMM_CHECK(cudaGetLastError());
  // held-out check per cell
  S.acc.ensure(sizeof(double) * (size_t)ns * SURR_CELLS * 3);
  FMM_CHECK(cudaMemsetAsync(S.acc.ptr, 0, sizeof(double) * (size_t)ns * SURR_CELLS * 3, st));
  LAUNCH(k_surr_heldout<<<(unsigned)(((long)ns * nh + 127) / 128), 128, 0, st>>>(
      (long)ns * nh, nh, S.slots.as<int>(), S.Xh.as<float>(), S.Yh.as<float>(), S.w16.as<__nv_bfloat16>(),
      S.acc.as<double>()));
  std::vector<double> acc((size_t)ns * SURR_CELLS * 3);
  FMM_CHECK(cudaMemcpyAsync(acc.data(), S.acc.ptr, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  S.cell_err.assign((size_t)nslot_all * SURR_CELLS, -1.0);
  S.cell_ok.assign((size_t)nslot_all * SURR_CELLS, 0);
  for (int si = 0; si < ns; ++si)
    for (int c = 0; c < SURR_CELLS; ++c) {
      const double* a = &acc[((size_t)si * SURR_CELLS + c) * 3];
      if (a[2] < 8 || a[1] <= 0.0) continue;              // too few held-out points to judge
      double err = std::sqrt(a[0] / a[1]);
      size_t k = (size_t)slots[si] * SURR_CELLS + c;
      S.cell_err[k] = err;
      S.cell_ok[k] = err <= bound ? 1 : 0;
    }
  S.ok.ensure(S.cell_ok.size());
  FMM_CHECK(cudaMemcpyAsync(S.ok.ptr, S.cell_ok.data(), S.cell_ok.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  S.rho_max = rho_max;
  S.z_min = z_min;
  S.z_max = z_max;
  S.bound = bound;
  S.trained = true;
}

SurrView surrogate_view(const fmm_layered* h) {
  SurrView v{};
  const SurrState& S = h->surr;
  if (!(h->flags & FMM_SURROGATE) || !S.trained) return v;
  v.w = (const __nv_bfloat16*)S.w16.ptr;
  v.ok = (const unsigned char*)S.ok.ptr;
  v.rho_max = S.rho_max;
  v.z_min = S.z_min;
  v.z_max = S.z_max;
  return v;
}

extern "C" int fmm_layered_surrogate_train(fmm_layered_t* h, double rho_max, double z_min, double z_max,
                                           long samples_per_component, int steps, double bound,
                                           unsigned long long seed, void* stream) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (h->L1 < 2 || !(rho_max > 0) || !(z_min > 0) || !(z_max > z_min) || !std::isfinite(rho_max + z_max) ||
      samples_per_component < 1024 || steps < 1 || !(bound > 0)) {
    h->err = "invalid argument (two or more layers, rho_max > 0, 0 < z_min < z_max, >= 1024 samples, steps >= 1, "
             "bound > 0)";
    return FMM_ERR_ARG;
  }
  try {
    surr_train_impl(h, rho_max, z_min, z_max, samples_per_component, steps, bound, seed, (cudaStream_t)stream);
  } catch (FmmError& e) {
    h->err = e.msg;
    h->surr.trained = false;
    return e.code;
  }
  return FMM_OK;
}

extern "C" int fmm_layered_surrogate_set_bound(fmm_layered_t* h, double bound) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  SurrState& S = h->surr;
  if (!S.trained || !(bound > 0)) {
    h->err = "no trained surrogate, or bound <= 0";
    return FMM_ERR_ARG;
  }
  for (size_t i = 0; i < S.cell_err.size(); ++i) S.cell_ok[i] = (S.cell_err[i] >= 0.0 && S.cell_err[i] <= bound) ? 1 : 0;
  if (cudaMemcpy(S.ok.ptr, S.cell_ok.data(), S.cell_ok.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    h->err = "copy of the cell verdicts failed";
    return FMM_ERR_CUDA;
  }
  S.bound = bound;
  return FMM_OK;
}

extern "C" int fmm_layered_surrogate_report(const fmm_layered_t* h, double* cell_err, unsigned char* cell_ok) {
  if (!h || !h->surr.trained) return FMM_ERR_ARG;
  const size_t n = h->surr.cell_err.size();
  if (cell_err) for (size_t i = 0; i < n; ++i) cell_err[i] = h->surr.cell_err[i];
  if (cell_ok) for (size_t i = 0; i < n; ++i) cell_ok[i] = h->surr.cell_ok[i];
  return FMM_OK;
}

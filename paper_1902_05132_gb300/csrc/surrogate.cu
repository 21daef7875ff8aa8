// Training of the learned surrogate of the reaction components
// (fmm_layered_surrogate_train), its held-out check, and the gradient entry
// point used to check the training kernels.
//
// Data: for every reaction component of the medium, points drawn uniformly in
// the box [0, rho_max] x [z_min, z_max]^2 of (rho, zt, zs), stratified by the
// cells of an 8 x 8 x 8 grid, with the values of the component computed by the
// library's quadrature (the plain path of the near field, eq.
// generalcomponentsimag), plus an independent held-out set.
// Training, in three steps:
//  1. the outputs y = 4 pi R u of each component are standardized (mean and
//     standard deviation per component and output);
//  2. Adam on the hidden layers and a shared output layer, all components at
//     once, minibatches of 1024 points per component and step; one CTA runs
//     forward and backward for 32 points (weights and layer inputs rounded to
//     BF16, FP32 products and sums) and writes its partial gradients; a second
//     kernel adds the partials of a component in a fixed order and takes the
//     Adam step on FP32 master weights.  Loss: mean squared error;
//  3. the output layer of every cell by least squares: the normal equations
//     of the cell's training samples over the 64 hidden features (computed
//     with the inference arithmetic) and a constant are summed in FP64 by one
//     CTA per (component, cell) and solved on the host (Cholesky, ridge
//     1e-10 of the mean diagonal); the standardization is folded into them.
// Check: relative RMS error of the held-out points of every cell; a cell is
// used only if it is within the bound.
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
// seq != 0: CTA ch takes points ch*32 .. ch*32+31 of the component (one fixed
// minibatch) instead of drawing them.
__global__ void __launch_bounds__(kTPB) k_surr_train(const float* __restrict__ X, const float* __restrict__ Y,
                                                    long nper, const float* __restrict__ wf_all,
                                                    float* __restrict__ gpart, unsigned long long seed, int step,
                                                    int seq) {
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
    long idx = (seq ? (long)(ch * kSB + s) : (long)(r % (unsigned long long)nper)) + (long)si * nper;
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
__device__ inline float surr_gsum(const float* __restrict__ gpart, long si, long p) {
  float g = 0.0f;
  for (int c = 0; c < kNCH; ++c) g += gpart[(si * kNCH + c) * kNP + p];
  return g;
}

__global__ void k_surr_adam(long n, const float* __restrict__ gpart, float* __restrict__ wf, float* __restrict__ m,
                            float* __restrict__ v, float lr, float c1, float c2) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long si = i / kNP, p = i % kNP;
  const float g = surr_gsum(gpart, si, p);
  float mi = 0.9f * m[i] + 0.1f * g;
  float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  wf[i] = wf[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// Gradient of one minibatch: the partials added in the order the Adam step uses.
__global__ void k_surr_gsum(long n, const float* __restrict__ gpart, float* __restrict__ g) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) g[i] = surr_gsum(gpart, i / kNP, i % kNP);
}

// y <- (y - mean) / sd per component and output (mu_sd[si][4] = mean0, mean1, sd0, sd1)
__global__ void k_surr_standardize(long n, long nper, const double* __restrict__ mu_sd, float* __restrict__ Y) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double* a = mu_sd + 4 * (e / nper);
  Y[2 * e] = (float)((Y[2 * e] - a[0]) / a[2]);
  Y[2 * e + 1] = (float)((Y[2 * e + 1] - a[1]) / a[3]);
}

// Normal equations of the output layer of one (component, cell): the upper
// triangle of F^T F (F = [features, 1], 65 columns, entries (i, j), i <= j, in
// row order) and F^T y (65 x 2), summed in FP64 over the cell's training
// samples; one CTA per (cell, component), 128 samples per round.
constexpr int kGN = SURR_HEAD_N;                       // 65
constexpr int kGTRI = kGN * (kGN + 1) / 2;             // 2145
constexpr int kGENT = kGTRI + 2 * kGN;                 // 2275
constexpr int kGPT = (kGENT + kTPB - 1) / kTPB;        // entries per thread

__global__ void __launch_bounds__(kTPB) k_surr_gram(long nper, const int* __restrict__ slots,
                                                   const float* __restrict__ X, const float* __restrict__ Y,
                                                   const __nv_bfloat16* __restrict__ winf, double* __restrict__ G) {
  const int c = blockIdx.x, si = blockIdx.y;
  const long per = nper / SURR_CELLS;
  const long e0 = (long)si * nper + (long)c * per;
  const __nv_bfloat16* hi = winf + (long)slots[si] * 2 * SURR_NINF;
  const __nv_bfloat16* lo = hi + SURR_NINF;
  __shared__ float F[kTPB][kGN + 1];
  __shared__ float Ys[kTPB][2];
  // the entries of this thread: (i, j) of the triangle, or (feature, output) of the right-hand side
  short ei[kGPT], ej[kGPT];
#pragma unroll
  for (int m = 0; m < kGPT; ++m) {
    int k = threadIdx.x + m * kTPB;
    ei[m] = -1;
    ej[m] = 0;
    if (k < kGTRI) {
      int i = 0, rowlen = kGN;
      while (k >= rowlen) { k -= rowlen; ++i; --rowlen; }
      ei[m] = (short)i;
      ej[m] = (short)(i + k);
    } else if (k < kGENT) {
      k -= kGTRI;
      ei[m] = (short)(k / 2);
      ej[m] = (short)(-1 - (k % 2));       // output column, encoded negative
    }
  }
  double acc[kGPT];
#pragma unroll
  for (int m = 0; m < kGPT; ++m) acc[m] = 0.0;
  for (long j0 = 0; j0 < per; j0 += kTPB) {
    const long j = j0 + threadIdx.x;
    __syncthreads();
    if (j < per) {
      const long e = e0 + j;
      float x[3] = {X[3 * e], X[3 * e + 1], X[3 * e + 2]};
      float f[SURR_H];
      surr_features(hi, lo, x, f);
      for (int i = 0; i < SURR_H; ++i) F[threadIdx.x][i] = f[i];
      F[threadIdx.x][SURR_H] = 1.0f;
      Ys[threadIdx.x][0] = Y[2 * e];
      Ys[threadIdx.x][1] = Y[2 * e + 1];
    } else {
      for (int i = 0; i <= SURR_H; ++i) F[threadIdx.x][i] = 0.0f;
      Ys[threadIdx.x][0] = Ys[threadIdx.x][1] = 0.0f;
    }
    __syncthreads();
    const int ns = (int)min((long)kTPB, per - j0);
#pragma unroll
    for (int m = 0; m < kGPT; ++m) {
      const int i = ei[m], jj = ej[m];
      if (i < 0) continue;
      double a = acc[m];
      if (jj >= 0) {
        for (int s = 0; s < ns; ++s) a = fma((double)F[s][i], (double)F[s][jj], a);
      } else {
        const int col = -1 - jj;
        for (int s = 0; s < ns; ++s) a = fma((double)F[s][i], (double)Ys[s][col], a);
      }
      acc[m] = a;
    }
  }
  double* out = G + ((long)si * SURR_CELLS + c) * kGENT;
#pragma unroll
  for (int m = 0; m < kGPT; ++m) {
    int k = threadIdx.x + m * kTPB;
    if (k < kGENT) out[k] = acc[m];
  }
}

// Held-out errors: acc[(si * 64 + cell) * 3 + {0,1,2}] += |err|^2, |y|^2, 1
__global__ void k_surr_heldout(long n, long nper, const int* __restrict__ slots, const float* __restrict__ X,
                               const float* __restrict__ Y, const __nv_bfloat16* __restrict__ winf,
                               double* __restrict__ acc) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int si = (int)(e / nper);
  float x[3] = {X[3 * e], X[3 * e + 1], X[3 * e + 2]};
  int c[3];
  for (int i = 0; i < 3; ++i) c[i] = min(SURR_GRID - 1, max(0, (int)((x[i] + 1.0f) * (0.5f * SURR_GRID))));
  int cell = (c[0] * SURR_GRID + c[1]) * SURR_GRID + c[2];
  float2 o = surr_forward(winf + (long)slots[si] * 2 * SURR_NINF, x, cell);
  float y0 = Y[2 * e], y1 = Y[2 * e + 1];
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

// BF16 hi/lo parts of x (x ~ hi + lo with a 16-bit significand)
static void split_hilo(float x, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  *hi = __float2bfloat16_rn(x);
  *lo = __float2bfloat16_rn(x - __bfloat162float(*hi));
}

// Solve (A + lam tr(A)/n I) w = b for the two right-hand sides of one cell's
// normal equations (upper triangle of A in row order, then b as [i][2]) by
// Cholesky in FP64.  Returns false if the matrix is not positive definite.
static bool solve_head(const double* g, double lam, double w[2][SURR_HEAD_N]) {
  const int n = SURR_HEAD_N;
  std::vector<double> A((size_t)n * n), b((size_t)n * 2);
  int k = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j, ++k) A[(size_t)i * n + j] = A[(size_t)j * n + i] = g[k];
  for (int i = 0; i < n; ++i) { b[2 * i] = g[k + 2 * i]; b[2 * i + 1] = g[k + 2 * i + 1]; }
  double tr = 0;
  for (int i = 0; i < n; ++i) tr += A[(size_t)i * n + i];
  if (!(tr > 0)) return false;
  for (int i = 0; i < n; ++i) A[(size_t)i * n + i] += lam * tr / n;
  for (int j = 0; j < n; ++j) {                    // A = L L^T, L in the lower triangle
    double d = A[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) d -= A[(size_t)j * n + p] * A[(size_t)j * n + p];
    if (!(d > 0)) return false;
    d = std::sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) v -= A[(size_t)i * n + p] * A[(size_t)j * n + p];
      A[(size_t)i * n + j] = v / d;
    }
  }
  for (int c = 0; c < 2; ++c) {
    std::vector<double> y(n);
    for (int i = 0; i < n; ++i) {
      double v = b[2 * i + c];
      for (int p = 0; p < i; ++p) v -= A[(size_t)i * n + p] * y[p];
      y[i] = v / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = y[i];
      for (int p = i + 1; p < n; ++p) v -= A[(size_t)p * n + i] * w[c][p];
      w[c][i] = v / A[(size_t)i * n + i];
    }
  }
  return true;
}

static void surr_train_impl(fmm_layered* h, double rho_max, double z_min, double z_max, long nper_in, int steps,
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
  // samples stratified by cell: a multiple of 64 per component
  const long nper = (nper_in + SURR_CELLS - 1) / SURR_CELLS * SURR_CELLS;
  const long nh = std::max<long>((nper / 8 + SURR_CELLS - 1) / SURR_CELLS * SURR_CELLS, 16 * SURR_CELLS);
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
  S.X.ensure(sizeof(float) * 3 * (size_t)ns * nper);
  S.Y.ensure(sizeof(float) * 2 * (size_t)ns * nper);
  S.Xh.ensure(sizeof(float) * 3 * (size_t)ns * nh);
  S.Yh.ensure(sizeof(float) * 2 * (size_t)ns * nh);
  launch_surr_samples((long)ns * nper, nper, S.slots.as<int>(), L1, box, R, seed, S.X.as<float>(), S.Y.as<float>(), st);
  launch_surr_samples((long)ns * nh, nh, S.slots.as<int>(), L1, box, R, seed ^ 0x5DEECE66DULL, S.Xh.as<float>(),
                      S.Yh.as<float>(), st);
  FMM_CHECK(cudaGetLastError());
  // 1. standardization of the outputs per component
  std::vector<float> hy((size_t)2 * ns * nper);
  FMM_CHECK(cudaMemcpyAsync(hy.data(), S.Y.ptr, sizeof(float) * hy.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  std::vector<double> musd((size_t)4 * ns);
  for (int si = 0; si < ns; ++si)
    for (int k = 0; k < 2; ++k) {
      double s1 = 0, s2 = 0;
      for (long e = 0; e < nper; ++e) s1 += hy[2 * ((size_t)si * nper + e) + k];
      const double mu = s1 / nper;
      for (long e = 0; e < nper; ++e) {
        double d = hy[2 * ((size_t)si * nper + e) + k] - mu;
        s2 += d * d;
      }
      double sd = std::sqrt(s2 / nper);
      if (!(sd > 1e-30)) sd = 1.0;
      musd[4 * si + k] = mu;
      musd[4 * si + 2 + k] = sd;
    }
  S.musd.ensure(sizeof(double) * musd.size());
  FMM_CHECK(cudaMemcpyAsync(S.musd.ptr, musd.data(), sizeof(double) * musd.size(), cudaMemcpyHostToDevice, st));
  LAUNCH(k_surr_standardize<<<(unsigned)(((long)ns * nper + 255) / 256), 256, 0, st>>>((long)ns * nper, nper,
                                                                                         S.musd.as<double>(),
                                                                                         S.Y.as<float>()));
  // 2. Adam: Glorot-uniform initial weights, zero biases
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
  S.gpart.ensure(sizeof(float) * (size_t)ns * kNCH * kNP);
  FMM_CHECK(cudaMemcpyAsync(S.wf.ptr, w0.data(), sizeof(float) * npt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemsetAsync(S.m.ptr, 0, sizeof(float) * npt, st));
  FMM_CHECK(cudaMemsetAsync(S.v.ptr, 0, sizeof(float) * npt, st));
  const size_t smem = sizeof(float) * (kNP + kSB * 5 + 8 * kSB * SURR_H);
  FMM_CHECK(cudaFuncSetAttribute(k_surr_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  float c1 = 1.0f, c2 = 1.0f;
  for (int t = 0; t < steps; ++t) {
    LAUNCH(k_surr_train<<<dim3(kNCH, ns), kTPB, smem, st>>>(S.X.as<float>(), S.Y.as<float>(), nper, S.wf.as<float>(),
                                                             S.gpart.as<float>(), seed, t, 0));
    c1 *= 0.9f;
    c2 *= 0.999f;
    const float lr = (float)(2e-3 * 0.5 * (1.0 + std::cos(M_PI * t / steps)) + 1e-6);
    LAUNCH(k_surr_adam<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(npt, S.gpart.as<float>(), S.wf.as<float>(),
                                                                      S.m.as<float>(), S.v.as<float>(), lr, 1.0f - c1,
                                                                      1.0f - c2));
  }
  FMM_CHECK(cudaGetLastError());
  // inference copies of the hidden layers (BF16 hi/lo)
  std::vector<float> wf((size_t)npt);
  FMM_CHECK(cudaMemcpyAsync(wf.data(), S.wf.ptr, sizeof(float) * npt, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  std::vector<__nv_bfloat16> winf((size_t)nslot_all * 2 * SURR_NINF, __float2bfloat16_rn(0.0f));
  for (int si = 0; si < ns; ++si) {
    __nv_bfloat16* hi = winf.data() + (size_t)slots[si] * 2 * SURR_NINF;
    for (int i = 0; i < SURR_NTRUNK; ++i) split_hilo(wf[(size_t)si * kNP + i], hi + i, hi + SURR_NINF + i);
  }
  S.winf.ensure(sizeof(__nv_bfloat16) * winf.size());
  FMM_CHECK(cudaMemcpyAsync(S.winf.ptr, winf.data(), sizeof(__nv_bfloat16) * winf.size(), cudaMemcpyHostToDevice, st));
  // 3. output layer of every cell by least squares
  S.gram.ensure(sizeof(double) * (size_t)ns * SURR_CELLS * kGENT);
  LAUNCH(k_surr_gram<<<dim3(SURR_CELLS, ns), kTPB, 0, st>>>(nper, S.slots.as<int>(), S.X.as<float>(), S.Y.as<float>(),
                                                            S.winf.as<__nv_bfloat16>(), S.gram.as<double>()));
  FMM_CHECK(cudaGetLastError());
  std::vector<double> gram((size_t)ns * SURR_CELLS * kGENT);
  FMM_CHECK(cudaMemcpyAsync(gram.data(), S.gram.ptr, sizeof(double) * gram.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  std::vector<unsigned char> solved((size_t)nslot_all * SURR_CELLS, 0);
  for (int si = 0; si < ns; ++si) {
    __nv_bfloat16* hi = winf.data() + (size_t)slots[si] * 2 * SURR_NINF;
    for (int c = 0; c < SURR_CELLS; ++c) {
      double w[2][SURR_HEAD_N];
      if (!solve_head(&gram[((size_t)si * SURR_CELLS + c) * kGENT], 1e-10, w)) continue;
      solved[(size_t)slots[si] * SURR_CELLS + c] = 1;
      for (int k = 0; k < 2; ++k) {
        const double mu = musd[4 * si + k], sd = musd[4 * si + 2 + k];
        const int r = SURR_NTRUNK + (c * 2 + k) * SURR_HEAD_N;
        for (int i = 0; i < SURR_H; ++i) split_hilo((float)(sd * w[k][i]), hi + r + i, hi + SURR_NINF + r + i);
        split_hilo((float)(sd * w[k][SURR_H] + mu), hi + r + SURR_H, hi + SURR_NINF + r + SURR_H);
      }
    }
  }
  FMM_CHECK(cudaMemcpyAsync(S.winf.ptr, winf.data(), sizeof(__nv_bfloat16) * winf.size(), cudaMemcpyHostToDevice, st));
  // held-out check per cell
  S.acc.ensure(sizeof(double) * (size_t)ns * SURR_CELLS * 3);
  FMM_CHECK(cudaMemsetAsync(S.acc.ptr, 0, sizeof(double) * (size_t)ns * SURR_CELLS * 3, st));
  LAUNCH(k_surr_heldout<<<(unsigned)(((long)ns * nh + 127) / 128), 128, 0, st>>>(
      (long)ns * nh, nh, S.slots.as<int>(), S.Xh.as<float>(), S.Yh.as<float>(), S.winf.as<__nv_bfloat16>(),
      S.acc.as<double>()));
  std::vector<double> acc((size_t)ns * SURR_CELLS * 3);
  FMM_CHECK(cudaMemcpyAsync(acc.data(), S.acc.ptr, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  S.cell_err.assign((size_t)nslot_all * SURR_CELLS, -1.0);
  S.cell_ok.assign((size_t)nslot_all * SURR_CELLS, 0);
  for (int si = 0; si < ns; ++si)
    for (int c = 0; c < SURR_CELLS; ++c) {
      const double* a = &acc[((size_t)si * SURR_CELLS + c) * 3];
      size_t k = (size_t)slots[si] * SURR_CELLS + c;
      if (!solved[k] || a[2] < 8 || a[1] <= 0.0) continue;     // no output layer, or too few held-out points
      double err = std::sqrt(a[0] / a[1]);
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
  v.w = (const __nv_bfloat16*)S.winf.ptr;
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

extern "C" int fmm_layered_surrogate_grad(const float* params, const float* x, const float* y, float* grad) {
  if (!params || !x || !y || !grad) return FMM_ERR_ARG;
  const long n = (long)kSB * kNCH;
  DevBuf bw, bx, by, bg, bp;
  int rc = FMM_OK;
  try {
    float* dw = (float*)(bw.ensure(sizeof(float) * kNP), bw.ptr);
    float* dx = (float*)(bx.ensure(sizeof(float) * 3 * n), bx.ptr);
    float* dy = (float*)(by.ensure(sizeof(float) * 2 * n), by.ptr);
    float* dg = (float*)(bg.ensure(sizeof(float) * kNP), bg.ptr);
    float* dp = (float*)(bp.ensure(sizeof(float) * kNCH * kNP), bp.ptr);
    FMM_CHECK(cudaMemcpy(dw, params, sizeof(float) * kNP, cudaMemcpyHostToDevice));
    FMM_CHECK(cudaMemcpy(dx, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice));
    FMM_CHECK(cudaMemcpy(dy, y, sizeof(float) * 2 * n, cudaMemcpyHostToDevice));
    const size_t smem = sizeof(float) * (kNP + kSB * 5 + 8 * kSB * SURR_H);
    FMM_CHECK(cudaFuncSetAttribute(k_surr_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LAUNCH(k_surr_train<<<dim3(kNCH, 1), kTPB, smem>>>(dx, dy, n, dw, dp, 0ULL, 0, 1));
    LAUNCH(k_surr_gsum<<<(kNP + 255) / 256, 256>>>(kNP, dp, dg));
    FMM_CHECK(cudaGetLastError());
    FMM_CHECK(cudaMemcpy(grad, dg, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
  } catch (FmmError& e) {
    rc = e.code;
  }
  DevBuf* all[] = {&bw, &bx, &by, &bg, &bp};
  for (DevBuf* b : all) b->release();
  return rc;
}

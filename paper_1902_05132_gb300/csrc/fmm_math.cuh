// Device math for the layered-media Helmholtz FMM (FP64).
//
// Complex numbers are double2 (x = real, y = imaginary).  Coefficient layout:
// degree n = 0..p, order m = -n..n, flat index n*n + n + m.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define FMM_PI 3.14159265358979323846
#define FMM_MAXP 20            // largest supported expansion order
#define FMM_MAXL 8             // largest supported number of layers

typedef double2 cplx;

__host__ __device__ inline cplx C(double re, double im = 0.0) { return make_double2(re, im); }
__host__ __device__ inline cplx cadd(cplx a, cplx b) { return C(a.x + b.x, a.y + b.y); }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return C(a.x - b.x, a.y - b.y); }
__host__ __device__ inline cplx cmul(cplx a, cplx b) { return C(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline cplx cscale(cplx a, double s) { return C(a.x * s, a.y * s); }
__host__ __device__ inline cplx cconj(cplx a) { return C(a.x, -a.y); }
__host__ __device__ inline cplx cneg(cplx a) { return C(-a.x, -a.y); }
__host__ __device__ inline double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline cplx cdiv(cplx a, cplx b) {
  double s = fabs(b.x) + fabs(b.y);
  double bx = b.x / s, by = b.y / s;
  double d = bx * bx + by * by;
  return C((a.x * bx + a.y * by) / (d * s), (a.y * bx - a.x * by) / (d * s));
}
// acc += a * b as four fused multiply-adds (no separate multiply or add)
__host__ __device__ inline void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// i^e for integer e
__host__ __device__ inline cplx ipow(int e) {
  switch (((e % 4) + 4) % 4) {
    case 0: return C(1, 0);
    case 1: return C(0, 1);
    case 2: return C(-1, 0);
    default: return C(0, -1);
  }
}
__host__ __device__ inline double sgn_pow(int e) { return (e & 1) ? -1.0 : 1.0; }

__device__ inline cplx cexp_(cplx z) {
  double s, c;
  sincos(z.y, &s, &c);
  double e = exp(z.x);
  return C(e * c, e * s);
}
__device__ inline cplx csqrt_(cplx z) {
  // principal square root, branch cut on the negative real axis
  double r = hypot(z.x, z.y);
  if (r == 0.0) return C(0, 0);
  double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0) return C(t, 0.5 * z.y / t);
  return C(0.5 * fabs(z.y) / t, copysign(t, z.y));
}

// k_z = sqrt(k^2 - k_rho^2) with Re >= 0, Im >= 0 (outgoing/decaying branch).
// On the real axis beyond k this is +i sqrt(k_rho^2 - k^2).
__device__ inline cplx kz_of(double k, cplx kr) {
  if (kr.y == 0.0 && kr.x > k) return C(0.0, sqrt((kr.x - k) * (kr.x + k)));
  cplx a = C(k * k - (kr.x * kr.x - kr.y * kr.y), -2.0 * kr.x * kr.y);
  cplx s = csqrt_(a);
  if (s.y < 0) s = cneg(s);
  return s;
}

// ---------------------------------------------------------------- Bessel
// Spherical Bessel j_n(x), n = 0..p, real x >= 0.  Upward recurrence where it
// is stable (x > p), Miller's backward recurrence normalized by j_0 otherwise.
__device__ inline void sph_jn(int p, double x, double* j) {
  if (x == 0.0) {
    j[0] = 1.0;
    for (int n = 1; n <= p; ++n) j[n] = 0.0;
    return;
  }
  double s, c;
  sincos(x, &s, &c);
  double j0 = (x < 1e-4) ? 1.0 - x * x / 6.0 : s / x;
  if (x > (double)p) {
    j[0] = j0;
    if (p >= 1) j[1] = s / (x * x) - c / x;
    for (int n = 1; n < p; ++n) j[n + 1] = (2 * n + 1) / x * j[n] - j[n - 1];
    return;
  }
  int N = p + 20 + (int)x;
  double f1 = 0.0, f0 = 1e-250;     // f_{n+1}, f_n
  for (int n = N; n >= 1; --n) {
    double fm = (2 * n + 1) / x * f0 - f1;    // f_{n-1}
    f1 = f0;
    f0 = fm;
    if (n - 1 <= p) j[n - 1] = f0;
    if (fabs(f0) > 1e200) {                    // rescale
      f0 *= 1e-200; f1 *= 1e-200;
      for (int m = n - 1; m <= p; ++m) j[m] *= 1e-200;
    }
  }
  double sc = j0 / j[0];
  for (int n = 0; n <= p; ++n) j[n] *= sc;
}

// Spherical Hankel h_n^(1)(x) = j_n + i y_n, n = 0..p, real x > 0.
__device__ inline void sph_hn(int p, double x, cplx* h) {
  double j[2 * FMM_MAXP + 2];
  sph_jn(p, x, j);
  double s, c;
  sincos(x, &s, &c);
  double y0 = -c / x, y1 = -c / (x * x) - s / x;
  h[0] = C(j[0], y0);
  if (p >= 1) h[1] = C(j[1], y1);
  for (int n = 1; n < p; ++n) {
    double y2 = (2 * n + 1) / x * y1 - y0;
    y0 = y1;
    y1 = y2;
    h[n + 1] = C(j[n + 1], y1);
  }
}

// J_0(z) for complex z by its power series (accurate for |z| <~ 12).
__device__ inline cplx j0_series(cplx z) {
  cplx u = cscale(cmul(z, z), -0.25);
  cplx term = C(1, 0), acc = C(1, 0);
  for (int k = 1; k < 40; ++k) {
    term = cscale(cmul(term, u), 1.0 / (double)(k * k));
    acc = cadd(acc, term);
    if (cabs2(term) < 1e-36 * cabs2(acc)) break;
  }
  return acc;
}

// J_d(z), d = 0..dmax, complex z with small imaginary part, by Miller's
// backward recurrence normalized with J_0 + 2 sum J_{2k} = 1.
__device__ inline void besselJ_all(int dmax, cplx z, cplx* J) {
  double az = sqrt(cabs2(z));
  if (az == 0.0) {
    J[0] = C(1, 0);
    for (int d = 1; d <= dmax; ++d) J[d] = C(0, 0);
    return;
  }
  int N = dmax + 30 + (int)(1.2 * az);
  N += (N & 1);
  cplx f1 = C(0, 0), f0 = C(1e-250, 0), norm = C(0, 0);
  cplx inv = cdiv(C(1, 0), z);
  for (int n = N; n >= 1; --n) {
    // f_{n-1} = (2n/z) f_n - f_{n+1}
    cplx fm = csub(cscale(cmul(inv, f0), 2.0 * n), f1);
    f1 = f0;
    f0 = fm;
    int m = n - 1;
    if (m <= dmax) J[m] = f0;
    if (m > 0 && (m & 1) == 0) norm = cadd(norm, cscale(f0, 2.0));
    if (cabs2(f0) > 1e300) {
      f0 = cscale(f0, 1e-200); f1 = cscale(f1, 1e-200); norm = cscale(norm, 1e-200);
      for (int q = m; q <= dmax; ++q) J[q] = cscale(J[q], 1e-200);
    }
  }
  norm = cadd(norm, f0);
  cplx s = cdiv(C(1, 0), norm);
  for (int d = 0; d <= dmax; ++d) J[d] = cmul(J[d], s);
}

// ---------------------------------------------------------------- Legendre
__host__ __device__ inline double rec_a(int n, int m) {
  return sqrt((double)((2 * n - 1) * (2 * n + 1)) / (double)((n - m) * (n + m)));
}
__host__ __device__ inline double rec_b(int n, int m) {
  if (n - m - 1 <= 0) return 0.0;
  return sqrt((double)((2 * n + 1) * (n - m - 1) * (n + m - 1)) / (double)((2 * n - 3) * (n + m) * (n - m)));
}

// Normalized associated Legendre P^_n^m(x), m >= 0 only, real x with
// s = sqrt(1 - x^2) >= 0; out[n*(n+1)/2 + m].
__device__ inline void phat_real(int p, double x, double s, double* out) {
  double diag = 0.28209479177387814;   // 1/sqrt(4 pi)
  for (int m = 0; m <= p; ++m) {
    if (m > 0) diag *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
    out[m * (m + 1) / 2 + m] = diag;
    double p2 = 0.0, p1 = diag;
    for (int n = m + 1; n <= p; ++n) {
      double cur = rec_a(n, m) * x * p1 - rec_b(n, m) * p2;
      out[n * (n + 1) / 2 + m] = cur;
      p2 = p1;
      p1 = cur;
    }
  }
}

// Complex continuation with s = sqrt(1 - z^2) on the branch of the paper
// (passed in: s = k_rho / k on the Sommerfeld contours).
__device__ inline void phat_complex(int p, cplx z, cplx s, cplx* out) {
  cplx diag = C(0.28209479177387814, 0);
  for (int m = 0; m <= p; ++m) {
    if (m > 0) diag = cscale(cmul(diag, s), sqrt((2.0 * m + 1.0) / (2.0 * m)));
    out[m * (m + 1) / 2 + m] = diag;
    cplx p2 = C(0, 0), p1 = diag;
    for (int n = m + 1; n <= p; ++n) {
      cplx cur = csub(cscale(cmul(z, p1), rec_a(n, m)), cscale(p2, rec_b(n, m)));
      out[n * (n + 1) / 2 + m] = cur;
      p2 = p1;
      p1 = cur;
    }
  }
}

// Spherical coordinates of v; theta = phi = 0 at the origin.
__device__ inline void to_sph(double x, double y, double z, double& r, double& ct, double& st, double& phi) {
  r = sqrt(x * x + y * y + z * z);
  if (r > 0) {
    ct = z / r;
    double rho = sqrt(x * x + y * y);
    st = rho / r;
  } else {
    ct = 1.0;
    st = 0.0;
  }
  phi = atan2(y, x);
}

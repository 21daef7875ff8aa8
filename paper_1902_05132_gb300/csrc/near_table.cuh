// Near-field reaction kernel from a table (FMM_TABLES; the tabulation of
// Sec. 3.5 applied to the kernel of eq. generalcomponentsimag).
//
// The reaction near field needs u~^{ab}_{ll'}(rho, zt, zs) = (i/4pi) S_{0,0,0,0}
// at arbitrary target-image pairs.  Per reaction component the table holds
// R u~ (which tends to a constant as R -> 0) on a 3-D grid in
//   u = log2(k_max R), R = sqrt(rho^2 + H^2), H = zt + zs,
//   theta = atan2(rho, H) in [0, atan 6],  f = zt / H in [0, 1],
// with 10 x 16 x 8 Chebyshev points of the first kind per panel (whole
// octaves of u from -7 to 1, half octaves from 1 to 3).  A pair is evaluated
// by the barycentric formula in each coordinate; pairs outside the table
// (R out of range, rho > 6 H) go to the quadrature.
#pragma once
#include <cuda_runtime.h>

#include "fmm_math.cuh"

#define NT_NU 10
#define NT_NTH 16
#define NT_NF 8
#define NT_PANELS 12
#define NT_PER_PANEL (NT_NU * NT_NTH * NT_NF)

// Chebyshev points x_j and barycentric weights (-1)^j sin((2j+1) pi / 2n) of
// the three coordinates, packed: x(NU), lam(NU), x(NTH), lam(NTH), x(NF), lam(NF).
#define NT_CHEB_LEN (2 * (NT_NU + NT_NTH + NT_NF))

struct NearTabView {
  const cplx* vals;        // [slot][panel][NU][NTH][NF]; nullptr: no table
  const int* slot_of;      // [(l L1 + l') 4 + 2a + b] -> slot (-1: none)
  const double* cheb;      // NT_CHEB_LEN
  double kmax;
};

__host__ __device__ inline double nt_theta_max() { return 1.4056476493802699; }   // atan(6)
__host__ __device__ inline double nt_edge(int k) { return (k <= 8) ? -7.0 + k : 1.0 + 0.5 * (k - 8); }

// barycentric weights of coordinate t in [-1, 1], normalized to sum 1
__device__ inline void nt_weights(int n, const double* x, const double* lam, double t, double* c) {
  int hit = -1;
  double s = 0.0;
  for (int j = 0; j < n; ++j) {
    const double d = t - x[j];
    if (d == 0.0) hit = j;
    c[j] = lam[j] / d;
    s += c[j];
  }
  if (hit >= 0) {
    for (int j = 0; j < n; ++j) c[j] = (j == hit) ? 1.0 : 0.0;
    return;
  }
  const double r = 1.0 / s;
  for (int j = 0; j < n; ++j) c[j] *= r;
}

// u~ of one pair of component `row` (= (l L1 + l') 4 + 2a + b) from the
// table; false when the pair lies outside it.
__device__ inline bool near_table_eval(const NearTabView& V, int row, double rho, double zt, double zs, cplx* out) {
  const int slot = V.slot_of[row];
  if (slot < 0) return false;
  const double H = zt + zs;
  const double R = sqrt(rho * rho + H * H);
  const double u = log2(V.kmax * R);
  const double th = atan2(rho, H);
  if (!(u >= nt_edge(0) && u <= nt_edge(NT_PANELS)) || th > nt_theta_max()) return false;
  int k = (u < 1.0) ? (int)floor(u + 7.0) : 8 + (int)floor(2.0 * (u - 1.0));
  k = min(max(k, 0), NT_PANELS - 1);
  const double lo = nt_edge(k), hi = nt_edge(k + 1);
  double cu[NT_NU], ct[NT_NTH], cf[NT_NF];
  const double* X = V.cheb;
  nt_weights(NT_NU, X, X + NT_NU, 2.0 * (u - lo) / (hi - lo) - 1.0, cu);
  X += 2 * NT_NU;
  nt_weights(NT_NTH, X, X + NT_NTH, 2.0 * th / nt_theta_max() - 1.0, ct);
  X += 2 * NT_NTH;
  nt_weights(NT_NF, X, X + NT_NF, 2.0 * zt / H - 1.0, cf);
  const cplx* P = V.vals + ((long)slot * NT_PANELS + k) * NT_PER_PANEL;
  double ar = 0.0, ai = 0.0;
  for (int i = 0; i < NT_NU; ++i) {
    double br = 0.0, bi = 0.0;
    for (int j = 0; j < NT_NTH; ++j) {
      const cplx* q = P + (i * NT_NTH + j) * NT_NF;
      double cr = 0.0, ci = 0.0;
#pragma unroll
      for (int m = 0; m < NT_NF; ++m) {
        const cplx v = q[m];
        cr = fma(cf[m], v.x, cr);
        ci = fma(cf[m], v.y, ci);
      }
      br = fma(ct[j], cr, br);
      bi = fma(ct[j], ci, bi);
    }
    ar = fma(cu[i], br, ar);
    ai = fma(cu[i], bi, ai);
  }
  const double r = 1.0 / R;
  *out = C(ar * r, ai * r);
  return true;
}

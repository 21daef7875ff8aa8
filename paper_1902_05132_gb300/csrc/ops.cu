// Expansions and translation operators (Secs. 2.1, 3.3, 3.5; Algorithm 1).
//
// Coefficient layout: flat index n*n + n + m (n = 0..p, m = -n..n).
//   P2M  M_nm = sum_j q_j 4 pi j_n(k r_j) conj(Y_n^m(theta_j, phi_j))  (eq. melecoeffree;
//        reaction: image positions and the source-layer k, eq. melayerupgoingimage)
//   M2M  M~_nm = sum conj(S^_{n nu}^{m mu}(c_child - c_parent)) M_{nu mu}        (eq. metome)
//   L2L  L~_nm = sum S^_{nu n}^{mu m}(c_child - c_parent) L_{nu mu}            (eq. metome)
//   M2L  free space: L_nm = (ik/4pi) sum S_{nu n}^{mu m}(c_t - c_s) M_{nu mu}  (Thm. 2.3;
//        the index order is the one the derivation of eq. metole gives)
//        reaction: L = T M with
//        T = i^{n+n'+1} i^{m'-m} e^{i(m'-m)phi_ts} s_t s_s
//            int k_rho J_{m'-m}(k_rho rho_ts) Z~^a(z_t, z_s) sigma^{ab}/k_lz
//                P^_n^m(k_lz/k_l) P^_{n'}^{m'}(k_l'z/k_l') dk_rho
//        (eqs. metoleimage1-2, me2lesimplified), s_t = 1, s_s = (-1)^{n'} for
//        a = up and s_t = (-1)^{n+m}, s_s = (-1)^{m'} for a = down (the source
//        plane wave of Z~^down is e^{ik_l'z(z_s - d_{l-1})}; its Funk-Hecke
//        expansion about the image centre carries (-1)^{m'}).
//   L2P  Phi = sum L_nm j_n(k r) Y_n^m(theta, phi)                           (eq. lelayerimage)
//   Separation matrices from the Gaunt formulas (eqs. spmhat3d, singularseparation):
//     S_{n nu}^{m mu}(b) = 4 pi (-1)^m i^{nu-n} sum_q i^q z_q(kb) conj(Y_q^{mu-m}(b^)) G(n,m;nu,-mu;q)
//   with z = h^(1) for S and z = j for S^; the Gaunt coefficients
//   G(n,m;nu,mu;q) = int Y_n^m Y_nu^mu conj(Y_q^{m+mu}) dOmega are computed here by
//   Gauss-Legendre quadrature in cos(theta) (exact for these polynomials).
#include <algorithm>
#include <cmath>
#include <vector>

#include "fmm_internal.h"

__host__ __device__ inline int NM(int n, int m) { return n * n + n + m; }
__host__ __device__ inline int PH(int n, int m) { return n * (n + 1) / 2 + m; }   // m >= 0

// ---------------------------------------------------------------- Gaunt table
// G[(n,m)][(nu,mu)][q] = G(n,m; nu,-mu; q), q = 0..2p
__global__ void k_gaunt(int p, int ng, const double* __restrict__ xg, const double* __restrict__ wg,
                        double* __restrict__ G) {
  int P = (p + 1) * (p + 1);
  long total = (long)P * P * (2 * p + 1);
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= total) return;
  int q = e % (2 * p + 1);
  long ij = e / (2 * p + 1);
  int j = ij % P, i = ij / P;
  int n = (int)floor(sqrt((double)i)), m = i - n * n - n;
  int nu = (int)floor(sqrt((double)j)), mu = j - nu * nu - nu;
  // G(n,m; nu,-mu; q) = 2 pi int P^_n^m P^_nu^{-mu} P^_q^{m-mu} dx
  int M3 = m - mu;
  double val = 0.0;
  if (!((n + nu + q) & 1) && q >= abs(n - nu) && q <= n + nu && abs(M3) <= q) {
    double Pa[(2 * FMM_MAXP + 1) * (2 * FMM_MAXP + 2) / 2];
    for (int g = 0; g < ng; ++g) {
      double x = xg[g], s = sqrt(fmax(0.0, 1.0 - x * x));
      phat_real(2 * p, x, s, Pa);
      double a = Pa[PH(n, abs(m))] * ((m < 0 && (m & 1)) ? -1.0 : 1.0);
      double b = Pa[PH(nu, abs(mu))] * ((-mu < 0 && (mu & 1)) ? -1.0 : 1.0);
      double c = Pa[PH(q, abs(M3))] * ((M3 < 0 && (M3 & 1)) ? -1.0 : 1.0);
      val += wg[g] * a * b * c;
    }
    val *= 2.0 * FMM_PI;
  }
  G[e] = val;
}

// ---------------------------------------------------------------- separation matrices
// One CTA per operator.  kind 0: free-space M2L (ik/4pi) S^T; 1: M2M conj(S^); 2: L2L S^^T.
// Output layout OpT[in][out] (out contiguous).


__global__ void k_sep_ops(int p, const SepJob* __restrict__ jobs, const double* __restrict__ G,
                          cplx* __restrict__ ops) {
  const SepJob jb = jobs[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  const int Q2 = 2 * p;
  __shared__ cplx zq[2 * FMM_MAXP + 1];
  __shared__ cplx Yc[(2 * FMM_MAXP + 1) * (2 * FMM_MAXP + 1)];   // conj(Y_q^M), flat (q, M)
  double r, ct, st, ph;
  to_sph(jb.b[0], jb.b[1], jb.b[2], r, ct, st, ph);
  if (threadIdx.x == 0) {
    if (jb.kind == 0) {
      cplx hq[2 * FMM_MAXP + 1];
      sph_hn(Q2, jb.k * r, hq);
      for (int q = 0; q <= Q2; ++q) zq[q] = hq[q];
    } else {
      double jq[2 * FMM_MAXP + 2];
      sph_jn(Q2, jb.k * r, jq);
      for (int q = 0; q <= Q2; ++q) zq[q] = C(jq[q], 0.0);
    }
  }
  if (threadIdx.x == 32 || (blockDim.x <= 32 && threadIdx.x == 0)) {
    double Pa[(2 * FMM_MAXP + 1) * (2 * FMM_MAXP + 2) / 2];
    phat_real(Q2, ct, st, Pa);
    for (int q = 0; q <= Q2; ++q)
      for (int M = -q; M <= q; ++M) {
        double pv = Pa[PH(q, abs(M))] * ((M < 0 && (M & 1)) ? -1.0 : 1.0);
        double s, c;
        sincos(M * ph, &s, &c);
        Yc[NM(q, M)] = C(pv * c, -pv * s);
      }
  }
  __syncthreads();
  const int NQ = 2 * p + 1;
  for (long e = threadIdx.x; e < (long)P * P; e += blockDim.x) {
    int in = e / P, out = e % P;
    // matrix element S_{row, col} with (row, col) = (in, out) for M2L / L2L
    // (transposed use) and (out, in) for M2M
    int row = (jb.kind == 1) ? out : in;
    int col = (jb.kind == 1) ? in : out;
    int n = (int)floor(sqrt((double)row)), m = row - n * n - n;
    int nu = (int)floor(sqrt((double)col)), mu = col - nu * nu - nu;
    const double* g = G + ((long)row * P + col) * NQ;
    cplx acc = C(0, 0);
    int qlo = abs(n - nu), qhi = n + nu;
    for (int q = qlo; q <= qhi; q += 2) {
      if (abs(mu - m) > q) continue;
      double gv = g[q];
      if (gv == 0.0) continue;
      cplx t = cmul(ipow(q), zq[q]);
      cfma(acc, cscale(t, gv), Yc[NM(q, mu - m)]);
    }
    cplx S = cscale(cmul(ipow(nu - n), acc), 4.0 * FMM_PI * sgn_pow(m));
    cplx v;
    if (jb.kind == 0) v = cmul(C(0.0, jb.k / (4.0 * FMM_PI)), S);
    else if (jb.kind == 1) v = cconj(S);
    else v = S;
    ops[jb.out_off + e] = v;
  }
}

// ---------------------------------------------------------------- reaction T
// For one group (component, level, jt, js) and its nodes q:
//   near nodes (complex): Ac[q][i] = i^n s_t P^_n^m(k_lz/k_l) c_q e^{i k_lz zt},
//                         Bc[q][j] = i^{n'} s_s P^_{n'}^{m'}(k_l'z/k_l') e^{i k_l'z zs},
//   with c_q = w k_rho sigma / k_lz;  T_ij += i^{1+m'-m} Ac J_{m'-m} Bc.
//   tail nodes (real k_rho = t, k_z = i kappa): P^_n^m(i y) = i^{n-m} R_n^m(y)
//   with R real (R_n = a y R_{n-1} + b R_{n-2}; R_n^{-m} = R_n^m), c_q = -i w t sigma / kappa_l,
//   and every factor of i cancels:  T_ij += Ar J_{m'-m} Br with
//   Ar[q][i] = (-1)^{n+m} s_t R_n^m |c_q| e^{-kappa_l zt}, Br = (-1)^{n'} s_s R_{n'}^{m'} e^{-kappa_l' zs}.


__device__ inline double st_sign(int a, int n, int m) { return (a == AR_UP) ? 1.0 : sgn_pow(n + m); }
__device__ inline double ss_sign(int a, int n, int m) { return (a == AR_UP) ? sgn_pow(n) : sgn_pow(m); }

// one thread per node: A and B rows
__global__ void k_reac_nodes(int p, ReacGroup g, int n_near, const cplx* __restrict__ kr, const cplx* __restrict__ w,
                             const cplx* __restrict__ kz, int Qall, const cplx* __restrict__ sigma,
                             cplx* __restrict__ Ac, cplx* __restrict__ Bc, double* __restrict__ Ar,
                             double* __restrict__ Br) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.Q) return;
  const int P = (p + 1) * (p + 1);
  cplx kzl = kz[(long)g.l * Qall + q], kzp = kz[(long)g.lp * Qall + q];
  cplx sg = sigma[g.sig_off + q];
  if (q < n_near) {
    cplx k_r = kr[q];
    cplx c = cdiv(cmul(cmul(w[q], k_r), sg), kzl);
    cplx et = cexp_(cmul(C(0, g.zt), kzl)), es = cexp_(cmul(C(0, g.zs), kzp));
    c = cmul(c, et);
    cplx ph[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
    phat_complex(p, cscale(kzl, 1.0 / g.kl), cscale(k_r, 1.0 / g.kl), ph);
    for (int i = 0; i < P; ++i) {
      int n = (int)floor(sqrt((double)i)), m = i - n * n - n, am = abs(m);
      cplx v = ph[n * (n + 1) / 2 + am];
      if (m < 0 && (am & 1)) v = cneg(v);
      Ac[(long)q * P + i] = cscale(cmul(cmul(ipow(n), v), c), st_sign(g.a, n, m));
    }
    phat_complex(p, cscale(kzp, 1.0 / g.klp), cscale(k_r, 1.0 / g.klp), ph);
    for (int j = 0; j < P; ++j) {
      int n = (int)floor(sqrt((double)j)), m = j - n * n - n, am = abs(m);
      cplx v = ph[n * (n + 1) / 2 + am];
      if (m < 0 && (am & 1)) v = cneg(v);
      Bc[(long)q * P + j] = cscale(cmul(cmul(ipow(n), v), es), ss_sign(g.a, n, m));
    }
  } else {
    long qt = q - n_near;
    double t = kr[q].x, kapl = kzl.y, kapp = kzp.y;
    double cR = w[q].x * t * sg.x / kapl;                 // c = -i cR
    double et = exp(-kapl * g.zt), es = exp(-kapp * g.zs);
    double R[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
    for (int side = 0; side < 2; ++side) {
      double k = side ? g.klp : g.kl, y = (side ? kapp : kapl) / k, s = t / k;
      double diag = 0.28209479177387814;
      for (int m = 0; m <= p; ++m) {
        if (m > 0) diag *= sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
        R[m * (m + 1) / 2 + m] = diag;
        double r2 = 0.0, r1 = diag;
        for (int n = m + 1; n <= p; ++n) {
          double cur = rec_a(n, m) * y * r1 + rec_b(n, m) * r2;
          R[n * (n + 1) / 2 + m] = cur;
          r2 = r1;
          r1 = cur;
        }
      }
      for (int i = 0; i < P; ++i) {
        // P^_n^m(i y) = i^{n-m} R_n^{|m|}(y) for either sign of m (the factor
        // (-1)^m of P^_n^{-m} is contained in i^{n-m})
        int n = (int)floor(sqrt((double)i)), m = i - n * n - n, am = abs(m);
        double v = R[n * (n + 1) / 2 + am];
        if (side == 0) Ar[qt * P + i] = sgn_pow(n + m) * st_sign(g.a, n, m) * v * cR * et;
        else Br[qt * P + i] = sgn_pow(n) * ss_sign(g.a, n, m) * v * es;
      }
    }
  }
}

// J_d(k_rho rho_r), d = 0..2p, for every node and radial class r
__global__ void k_reac_bessel(int p, int Q, int n_near, int nr, const double* __restrict__ rho,
                              const cplx* __restrict__ kr, cplx* __restrict__ Jc, double* __restrict__ Jr) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)Q * nr) return;
  int q = e % Q, r = e / Q;
  const int D = 2 * p + 1;
  if (q < n_near) {
    cplx J[2 * (2 * FMM_MAXP) + 1];
    besselJ_all(2 * p, cscale(kr[q], rho[r]), J);
    for (int d = 0; d < D; ++d) Jc[((long)r * n_near + q) * D + d] = J[d];
  } else {
    double x = kr[q].x * rho[r];
    long base = ((long)r * (Q - n_near) + (q - n_near)) * D;
    if (x > 2.0 * p + 2.0) {
      // upward recurrence is stable for d < x
      double j0v = j0(x), j1v = j1(x);
      Jr[base] = j0v;
      if (D > 1) Jr[base + 1] = j1v;
      for (int d = 1; d + 1 < D; ++d) {
        double j2 = 2.0 * d / x * j1v - j0v;
        j0v = j1v;
        j1v = j2;
        Jr[base + d + 1] = j2;
      }
    } else {
      cplx J[2 * (2 * FMM_MAXP) + 1];
      besselJ_all(2 * p, C(x, 0.0), J);
      for (int d = 0; d < D; ++d) Jr[base + d] = J[d].x;
    }
  }
}

// T_rad[r] (OpT layout [j][i]) for one group: CTA per (radial class, m block).
#define TQR 32
__global__ void k_reac_contract(int p, int Q, int n_near, const cplx* __restrict__ Ac, const cplx* __restrict__ Bc,
                                const double* __restrict__ Ar, const double* __restrict__ Br,
                                const cplx* __restrict__ Jc, const double* __restrict__ Jr,
                                const long* __restrict__ out_off, cplx* __restrict__ ops) {
  const int r = blockIdx.x;
  const int m = (int)blockIdx.y - p;
  const int P = (p + 1) * (p + 1);
  const int D = 2 * p + 1;
  const int am = abs(m), nrow = p + 1 - am;
  const int nout = nrow * P;
  // outputs of this CTA: obase .. obase + 8 * blockDim.x (blockIdx.z splits large orders)
  const int obase = blockIdx.z * 8 * blockDim.x;
  if (obase >= nout) return;        // uniform over the CTA
  extern __shared__ double smr[];
  // tail tiles: A[TQR][nrow], B[TQR][P], J[TQR][D]; near tiles reuse the space as complex
  double* sA = smr;
  double* sB = sA + 2 * TQR * (FMM_MAXP + 1);
  double* sJ = sB + 2 * TQR * P;
  const int per = (nout - obase + blockDim.x - 1) / blockDim.x;
  double accr[8], acci[8];
  int oi[8], oj[8], od[8];
  for (int k = 0; k < 8; ++k) {
    accr[k] = acci[k] = 0.0;
    int o = obase + threadIdx.x + k * blockDim.x;
    oi[k] = o / P;
    oj[k] = o % P;
    int n2 = (int)floor(sqrt((double)oj[k])), mm = oj[k] - n2 * n2 - n2;
    od[k] = mm - m;     // may be negative
  }
  // near nodes (complex)
  cplx* cA = (cplx*)sA;
  cplx* cB = (cplx*)sB;
  cplx* cJ = (cplx*)sJ;
  for (int q0 = 0; q0 < n_near; q0 += TQR / 2) {
    int nq = min(TQR / 2, n_near - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < nq * nrow; e += blockDim.x) {
      int t = e / nrow, rr = e % nrow;
      int n = am + rr;
      cA[t * nrow + rr] = Ac[(long)(q0 + t) * P + n * n + n + m];
    }
    for (int e = threadIdx.x; e < nq * P; e += blockDim.x) cB[e] = Bc[(long)q0 * P + e];
    for (int e = threadIdx.x; e < nq * D; e += blockDim.x) cJ[e] = Jc[((long)r * n_near + q0) * D + e];
    __syncthreads();
    for (int k = 0; k < per && k < 8; ++k) {
      int o = obase + threadIdx.x + k * blockDim.x;
      if (o >= nout) break;
      int d = od[k], ad = abs(d);
      double sgnd = (d < 0 && (ad & 1)) ? -1.0 : 1.0;
      cplx a = C(accr[k], acci[k]);
      for (int t = 0; t < nq; ++t) {
        cplx jv = cscale(cJ[t * D + ad], sgnd);
        cfma(a, cmul(cA[t * nrow + oi[k]], jv), cB[t * P + oj[k]]);
      }
      accr[k] = a.x;
      acci[k] = a.y;
    }
  }
  // multiply the near part by i^{1+d}
  for (int k = 0; k < per && k < 8; ++k) {
    cplx v = cmul(ipow(1 + od[k]), C(accr[k], acci[k]));
    accr[k] = v.x;
    acci[k] = v.y;
  }
  // tail nodes (real)
  const int Qt = Q - n_near;
  for (int q0 = 0; q0 < Qt; q0 += TQR) {
    int nq = min(TQR, Qt - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < nq * nrow; e += blockDim.x) {
      int t = e / nrow, rr = e % nrow;
      int n = am + rr;
      sA[t * nrow + rr] = Ar[(long)(q0 + t) * P + n * n + n + m];
    }
    for (int e = threadIdx.x; e < nq * P; e += blockDim.x) sB[e] = Br[(long)q0 * P + e];
    for (int e = threadIdx.x; e < nq * D; e += blockDim.x) sJ[e] = Jr[((long)r * Qt + q0) * D + e];
    __syncthreads();
    for (int k = 0; k < per && k < 8; ++k) {
      int o = obase + threadIdx.x + k * blockDim.x;
      if (o >= nout) break;
      int d = od[k], ad = abs(d);
      double sgnd = (d < 0 && (ad & 1)) ? -1.0 : 1.0;
      double a = 0.0;
      for (int t = 0; t < nq; ++t) a += sA[t * nrow + oi[k]] * sJ[t * D + ad] * sB[t * P + oj[k]];
      accr[k] += sgnd * a;
    }
  }
  for (int k = 0; k < per && k < 8; ++k) {
    int o = obase + threadIdx.x + k * blockDim.x;
    if (o >= nout) break;
    int n = am + oi[k];
    int i = n * n + n + m;
    ops[out_off[r] + (long)oj[k] * P + i] = C(accr[k], acci[k]);
  }
}

// Symmetric split of a radial reaction operator.  With the signed reflection
// (R x)_{n,m} = (-1)^m x_{n,-m}, the radial integral satisfies
// I(n,-m; n',-m') = (-1)^{m+m'} I(n,m; n',m'), so I commutes with R and is block
// diagonal in the orthonormal basis
//   plus:  e_{n,0};  (e_{n,m} + (-1)^m e_{n,-m}) / sqrt2   (m > 0), index n(n+1)/2 + m
//   minus: (e_{n,m} - (-1)^m e_{n,-m}) / sqrt2              (m > 0), index n(n-1)/2 + m - 1
// Output: Ip [b][a] (np x np) followed by Im [b][a] (nm x nm), input-major.
__device__ inline int basis_terms(int p, int a, bool plus, int* idx, double* val) {
  // basis vector -> up to two (flat index, coefficient) terms
  int n, m;
  if (plus) {
    n = (int)floor((sqrt(8.0 * a + 1.0) - 1.0) * 0.5);
    while ((n + 1) * (n + 2) / 2 <= a) ++n;
    while (n * (n + 1) / 2 > a) --n;
    m = a - n * (n + 1) / 2;
  } else {
    n = 1;
    while (n * (n + 1) / 2 <= a) ++n;
    m = a - n * (n - 1) / 2 + 1;
  }
  if (m == 0) {
    idx[0] = n * n + n;
    val[0] = 1.0;
    return 1;
  }
  const double r = 0.70710678118654752440;
  double s = (m & 1) ? -1.0 : 1.0;
  idx[0] = n * n + n + m;
  val[0] = r;
  idx[1] = n * n + n - m;
  val[1] = plus ? s * r : -s * r;
  return 2;
}

__global__ void k_reac_split(int p, const cplx* __restrict__ full, cplx* __restrict__ out) {
  const int P = (p + 1) * (p + 1);
  const int np = (p + 1) * (p + 2) / 2, nm = p * (p + 1) / 2;
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long total = (long)np * np + (long)nm * nm;
  if (e >= total) return;
  bool plus = e < (long)np * np;
  int nb = plus ? np : nm;
  long le = plus ? e : e - (long)np * np;
  int b = le / nb, a = le % nb;       // out[b][a] = v_a^T I v_b
  int ia[2], ib[2];
  double va[2], vb[2];
  int na = basis_terms(p, a, plus, ia, va), nbt = basis_terms(p, b, plus, ib, vb);
  cplx acc = C(0, 0);
  for (int x = 0; x < na; ++x)
    for (int y = 0; y < nbt; ++y)
      acc = cadd(acc, cscale(full[(long)ib[y] * P + ia[x]], va[x] * vb[y]));    // I[i][j] at full[j*P + i]
  out[e] = acc;
}

// The same split for a batch of radial operators: operator y of the batch is
// read at full + y * stride and written at out + offs[y].
__global__ void k_reac_split_batch(int p, const cplx* __restrict__ full, long stride, const long* __restrict__ offs,
                                   cplx* __restrict__ out) {
  const int y = blockIdx.y;
  const int P = (p + 1) * (p + 1);
  const int np = (p + 1) * (p + 2) / 2, nm = p * (p + 1) / 2;
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long total = (long)np * np + (long)nm * nm;
  if (e >= total) return;
  const cplx* F = full + (long)y * stride;
  bool plus = e < (long)np * np;
  int nb = plus ? np : nm;
  long le = plus ? e : e - (long)np * np;
  int b = le / nb, a = le % nb;
  int ia[2], ib[2];
  double va[2], vb[2];
  int na = basis_terms(p, a, plus, ia, va), nbt = basis_terms(p, b, plus, ib, vb);
  cplx acc = C(0, 0);
  for (int x = 0; x < na; ++x)
    for (int z = 0; z < nbt; ++z) acc = cadd(acc, cscale(F[(long)ib[z] * P + ia[x]], va[x] * vb[z]));
  out[offs[y] + e] = acc;
}

// ---------------------------------------------------------------- P2M



__device__ inline void box_center(const CompGeom& cg, int level, const int* coord, double* c) {
  double w = cg.h2 / (double)(1 << level);
  for (int a = 0; a < 3; ++a) c[a] = cg.lo[a] + (coord[a] + 0.5) * w;
}

// Recurrence coefficients of the normalized Legendre functions (the same
// a_nm, b_nm as phat_real) and the diagonal factors
// P^_m^m = c_diag[m] s^m, tabulated once so that the per-particle passes do
// no FP64 square roots or divisions.  Index n(n+1)/2 + m, n <= FMM_MAXP.
__constant__ double c_reca[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
__constant__ double c_recb[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
__constant__ double c_diag[FMM_MAXP + 1];

void init_legendre_tables() {
  const int NT = (FMM_MAXP + 1) * (FMM_MAXP + 2) / 2;
  std::vector<double> a(NT, 0.0), b(NT, 0.0), dg(FMM_MAXP + 1);
  for (int n = 0; n <= FMM_MAXP; ++n)
    for (int m = 0; m < n; ++m) {
      a[n * (n + 1) / 2 + m] = rec_a(n, m);
      b[n * (n + 1) / 2 + m] = rec_b(n, m);
    }
  dg[0] = 0.28209479177387814;
  for (int m = 1; m <= FMM_MAXP; ++m) dg[m] = dg[m - 1] * sqrt((2.0 * m + 1.0) / (2.0 * m));
  FMM_CHECK(cudaMemcpyToSymbol(c_reca, a.data(), sizeof(double) * NT));
  FMM_CHECK(cudaMemcpyToSymbol(c_recb, b.data(), sizeof(double) * NT));
  FMM_CHECK(cudaMemcpyToSymbol(c_diag, dg.data(), sizeof(double) * (FMM_MAXP + 1)));
}

// j_n(x), n = 0..p, as sph_jn but multiplying by 1/x instead of dividing.
__device__ inline void sph_jn_fast(int p, double x, double* j) {
  if (x == 0.0) {
    j[0] = 1.0;
    for (int n = 1; n <= p; ++n) j[n] = 0.0;
    return;
  }
  double s, c;
  sincos(x, &s, &c);
  const double ix = 1.0 / x;
  double j0 = (x < 1e-4) ? 1.0 - x * x / 6.0 : s * ix;
  if (x > (double)p) {
    j[0] = j0;
    if (p >= 1) j[1] = (s * ix - c) * ix;
    for (int n = 1; n < p; ++n) j[n + 1] = (2 * n + 1) * ix * j[n] - j[n - 1];
    return;
  }
  int N = p + 20 + (int)x;
  double f1 = 0.0, f0 = 1e-250;
  for (int n = N; n >= 1; --n) {
    double fm = (2 * n + 1) * ix * f0 - f1;
    f1 = f0;
    f0 = fm;
    if (n - 1 <= p) j[n - 1] = f0;
    if (fabs(f0) > 1e200) {
      f0 *= 1e-200; f1 *= 1e-200;
      for (int m = n - 1; m <= p; ++m) j[m] *= 1e-200;
    }
  }
  double sc = j0 / j[0];
  for (int n = 0; n <= p; ++n) j[n] *= sc;
}

// One CTA per source leaf.  For a chunk of sources: one thread per source
// forms r, angles and j_n(k r); then one thread per (source, order m) runs
// the Legendre recurrence of column m and writes the 4 pi q j_n conj(Y_n^{+-m})
// values; then each thread sums its coefficients over the chunk.
__global__ void __launch_bounds__(128) k_p2m(int p, int chunk, const int* __restrict__ leaves, BoxGeom B,
                                             const CompGeom* __restrict__ cgs, const double* __restrict__ spos,
                                             const cplx* __restrict__ sq, cplx* __restrict__ M) {
  int b = leaves[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  const CompGeom cg = cgs[B.comp[b]];
  double c[3];
  box_center(cg, B.lev[b], B.coord + 3 * b, c);
  extern __shared__ cplx vals[];     // [chunk][P], then [chunk][p+1] j_n and [chunk][4] geometry
  double* jn = (double*)(vals + (size_t)chunk * P);
  double* geo = jn + (size_t)chunk * (p + 1);
  cplx acc[4] = {C(0, 0), C(0, 0), C(0, 0), C(0, 0)};
  for (int s0 = B.sb[b]; s0 < B.se[b]; s0 += chunk) {
    int ns = min(chunk, B.se[b] - s0);
    __syncthreads();
    for (int t = threadIdx.x; t < ns; t += blockDim.x) {
      int s = s0 + t;
      double r, ct, st, ph;
      to_sph(spos[3 * s] - c[0], spos[3 * s + 1] - c[1], spos[3 * s + 2] - c[2], r, ct, st, ph);
      sph_jn_fast(p, cg.ks * r, jn + t * (p + 1));
      geo[4 * t] = ct;
      geo[4 * t + 1] = st;
      geo[4 * t + 2] = ph;
    }
    __syncthreads();
    for (int item = threadIdx.x; item < ns * (p + 1); item += blockDim.x) {
      const int t = item / (p + 1), m = item % (p + 1);
      const double ct = geo[4 * t], st = geo[4 * t + 1], ph = geo[4 * t + 2];
      const double* j = jn + t * (p + 1);
      cplx qv = sq[s0 + t];
      double sn, cs;
      sincos(m * ph, &sn, &cs);
      sn = -sn;                                    // conj(Y)
      cplx e = cscale(cmul(C(cs, sn), qv), 4.0 * FMM_PI);
      cplx e2 = cscale(cmul(C(cs, -sn), qv), 4.0 * FMM_PI * ((m & 1) ? -1.0 : 1.0));
      double sm = 1.0;
      for (int i = 0; i < m; ++i) sm *= st;
      double p2 = 0.0, p1 = c_diag[m] * sm;
      cplx* out = vals + t * P;
      for (int n = m; n <= p; ++n) {
        double pv;
        if (n == m) pv = p1;
        else {
          pv = c_reca[n * (n + 1) / 2 + m] * ct * p1 - c_recb[n * (n + 1) / 2 + m] * p2;
          p2 = p1;
          p1 = pv;
        }
        double v = j[n] * pv;
        out[n * n + n + m] = cscale(e, v);
        if (m) out[n * n + n - m] = cscale(e2, v);
      }
    }
    __syncthreads();
    for (int k = 0; k < 4; ++k) {
      int i = threadIdx.x + k * blockDim.x;
      if (i >= P) break;
      for (int t = 0; t < ns; ++t) acc[k] = cadd(acc[k], vals[t * P + i]);
    }
  }
  for (int k = 0; k < 4; ++k) {
    int i = threadIdx.x + k * blockDim.x;
    if (i >= P) break;
    M[(long)b * P + i] = acc[k];
  }
}

// ---------------------------------------------------------------- M2M (one level)
// M_b = sum over children c with sources of OpM2M[comp][level(c)][octant(c)] M_c.
// op_base[comp * 23 + level]: element offset of the 8 operators of that level.
__global__ void k_m2m(int p, const int* __restrict__ boxes, BoxGeom B, const long* __restrict__ op_base,
                      const cplx* __restrict__ ops, cplx* __restrict__ M) {
  int b = boxes[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  extern __shared__ cplx Ms[];
  cplx acc[4] = {C(0, 0), C(0, 0), C(0, 0), C(0, 0)};
  int comp = B.comp[b];
  for (int k = 0; k < B.nchild[b]; ++k) {
    int c = B.child0[b] + k;
    if (B.se[c] == B.sb[c]) continue;
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x) Ms[i] = M[(long)c * P + i];
    __syncthreads();
    int oct = (B.coord[3 * c] & 1) | ((B.coord[3 * c + 1] & 1) << 1) | ((B.coord[3 * c + 2] & 1) << 2);
    const cplx* op = ops + op_base[comp * 23 + B.lev[c]] + (long)oct * P * P;
    for (int kk = 0; kk < 4; ++kk) {
      int i = threadIdx.x + kk * blockDim.x;
      if (i >= P) break;
      cplx a = acc[kk];
      for (int j = 0; j < P; ++j) cfma(a, op[(long)j * P + i], Ms[j]);
      acc[kk] = a;
    }
  }
  for (int kk = 0; kk < 4; ++kk) {
    int i = threadIdx.x + kk * blockDim.x;
    if (i >= P) break;
    M[(long)b * P + i] = acc[kk];
  }
}

// ---------------------------------------------------------------- M2L + L2L (one level)
// L_T = OpL2L[comp][level(T)][octant(T)] L_parent (if the parent carries a local
// expansion) + sum_{S in V(T)} OpM2L(T, S) M_S.


// Mark the reaction M2L classes used by the V lists:
// used[(comp * 23 + level) * 40 + (jt * 2 + js) * 10 + r] = 1.
__global__ void k_mark_reac(int nb, BoxGeom B, const CompGeom* __restrict__ cgs, const int* __restrict__ voff,
                            const int* __restrict__ vidx, unsigned char* __restrict__ used, int* __restrict__ err) {
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= nb) return;
  int comp = B.comp[T];
  if (cgs[comp].kind != CK_REAC) return;
  int lev = B.lev[T];
  const int* ct = B.coord + 3 * T;
  const int tab[10] = {0, 1, 2, 4, 5, 8, 9, 10, 13, 18};
  for (int e = voff[T]; e < voff[T + 1]; ++e) {
    const int* cs = B.coord + 3 * vidx[e];
    int dx = ct[0] - cs[0], dy = ct[1] - cs[1];
    int half = 1 << (lev - 1);
    int jt, js;
    if (cgs[comp].a == AR_UP) { jt = ct[2] - half; js = half - 1 - cs[2]; }
    else { jt = half - 1 - ct[2]; js = cs[2] - half; }
    int r = -1;
    for (int k = 0; k < 10; ++k) if (tab[k] == dx * dx + dy * dy) r = k;
    if (jt < 0 || jt > 1 || js < 0 || js > 1 || r < 0) { atomicOr(err, 8); continue; }
    used[((long)comp * 23 + lev) * 40 + (jt * 2 + js) * 10 + r] = 1;
  }
}

// ---------------------------------------------------------------- L2P
__global__ void k_l2p(int p, const int* __restrict__ leaves, BoxGeom B, const CompGeom* __restrict__ cgs,
                      const double* __restrict__ tpos, const cplx* __restrict__ L, cplx* __restrict__ phi) {
  int b = leaves[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  const CompGeom cg = cgs[B.comp[b]];
  double c[3];
  box_center(cg, B.lev[b], B.coord + 3 * b, c);
  extern __shared__ cplx Ls[];
  for (int i = threadIdx.x; i < P; i += blockDim.x) Ls[i] = L[(long)b * P + i];
  __syncthreads();
  for (int t = B.tb[b] + threadIdx.x; t < B.te[b]; t += blockDim.x) {
    double r, ct, st, ph;
    to_sph(tpos[3 * t] - c[0], tpos[3 * t + 1] - c[1], tpos[3 * t + 2] - c[2], r, ct, st, ph);
    double jn[FMM_MAXP + 1];
    sph_jn_fast(p, cg.kt * r, jn);
    cplx acc = C(0, 0);
    double sm = 1.0;                  // st^m
    for (int m = 0; m <= p; ++m) {
      double s, cc;
      sincos(m * ph, &s, &cc);
      const double sg = (m & 1) ? -1.0 : 1.0;
      // column m of the Legendre table by its recurrence (tabulated coefficients)
      double p2 = 0.0, p1 = c_diag[m] * sm;
      for (int n = m; n <= p; ++n) {
        double pv;
        if (n == m) pv = p1;
        else {
          pv = c_reca[n * (n + 1) / 2 + m] * ct * p1 - c_recb[n * (n + 1) / 2 + m] * p2;
          p2 = p1;
          p1 = pv;
        }
        double v = jn[n] * pv;
        cfma(acc, C(v * cc, v * s), Ls[NM(n, m)]);
        if (m) cfma(acc, C(sg * v * cc, -sg * v * s), Ls[NM(n, -m)]);
      }
      sm *= st;
    }
    phi[t] = acc;
  }
}

// ---------------------------------------------------------------- host launchers
void launch_gaunt(int p, const std::vector<double>& xg, const std::vector<double>& wg, double* G,
                  double* dx, double* dw, cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  long total = (long)P * P * (2 * p + 1);
  cudaMemcpyAsync(dx, xg.data(), 8 * xg.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dw, wg.data(), 8 * wg.size(), cudaMemcpyHostToDevice, st);
  LAUNCH(k_gaunt<<<(total + 127) / 128, 128, 0, st>>>(p, (int)xg.size(), dx, dw, G));
}

void launch_sep_ops(int p, const SepJob* jobs, int njobs, const double* G, cplx* ops, cudaStream_t st) {
  if (njobs) LAUNCH(k_sep_ops<<<njobs, 256, 0, st>>>(p, jobs, G, ops));
}

// Radial reaction M2L matrices of one group for nr radial classes.
// scratch bytes of launch_reac_group for a group of Q nodes (n_near complex)
// and nr radial classes
size_t reac_group_scratch(int p, int Q, int n_near, int nr) {
  const int P = (p + 1) * (p + 1), D = 2 * p + 1;
  const int nn = std::min(n_near, Q), Qt = Q - nn;
  return sizeof(cplx) * 2 * (size_t)nn * P + sizeof(double) * 2 * (size_t)Qt * P +
         sizeof(cplx) * (size_t)nr * nn * D + sizeof(double) * (size_t)nr * Qt * D + 1024;
}

void launch_reac_group(int p, const ReacGroup& g, const RuleNodes& R, int nr, const double* d_rho,
                       const long* d_out_off, cplx* ops, DevBuf& scratch, cudaStream_t st) {
  const int P = (p + 1) * (p + 1);
  const int D = 2 * p + 1;
  const int nn = std::min(R.n_near, g.Q), Qt = g.Q - nn;
  scratch.ensure(reac_group_scratch(p, g.Q, R.n_near, nr));
  char* base = (char*)scratch.ptr;
  cplx* Ac = (cplx*)base;
  cplx* Bc = Ac + (size_t)nn * P;
  double* Ar = (double*)(Bc + (size_t)nn * P);
  double* Br = Ar + (size_t)Qt * P;
  cplx* Jc = (cplx*)(Br + (size_t)Qt * P);
  double* Jr = (double*)(Jc + (size_t)nr * nn * D);
  LAUNCH(k_reac_nodes<<<(g.Q + 127) / 128, 128, 0, st>>>(p, g, nn, R.kr, R.w, R.kz, R.Q, R.sigma, Ac, Bc, Ar, Br));
  long ne = (long)g.Q * nr;
  LAUNCH(k_reac_bessel<<<(ne + 127) / 128, 128, 0, st>>>(p, g.Q, nn, nr, d_rho, R.kr, Jc, Jr));
  size_t smem = sizeof(double) * (2 * TQR * (FMM_MAXP + 1) + 2 * TQR * P + 2 * TQR * D);
  FMM_CHECK(cudaFuncSetAttribute(k_reac_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int threads = 256;
  dim3 grid(nr, 2 * p + 1, ((p + 1) * P + 8 * threads - 1) / (8 * threads));
  LAUNCH(k_reac_contract<<<grid, threads, smem, st>>>(p, g.Q, nn, Ac, Bc, Ar, Br, Jc, Jr, d_out_off, ops));
}

void launch_p2m(int p, const int* leaves, int n, BoxGeom B, const CompGeom* cgs, const double* spos,
                const cplx* sq, cplx* M, cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  const size_t per = sizeof(cplx) * P + sizeof(double) * (p + 1 + 4);
  int chunk = std::min(16, (int)((200 * 1024) / per));
  size_t smem = per * chunk;
  FMM_CHECK(cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (n) LAUNCH(k_p2m<<<n, 128, smem, st>>>(p, chunk, leaves, B, cgs, spos, sq, M));
}

void launch_l2p(int p, const int* leaves, int n, BoxGeom B, const CompGeom* cgs, const double* tpos,
                const cplx* L, cplx* phi, cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  if (n) LAUNCH(k_l2p<<<n, 64, sizeof(cplx) * P, st>>>(p, leaves, B, cgs, tpos, L, phi));
}

void launch_m2m(int p, const int* boxes, int n, BoxGeom B, const long* op_base, const cplx* ops, cplx* M,
                cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  if (n) LAUNCH(k_m2m<<<n, 128, sizeof(cplx) * P, st>>>(p, boxes, B, op_base, ops, M));
}

void launch_reac_split(int p, const cplx* full, cplx* out, cudaStream_t st) {
  long np = (long)(p + 1) * (p + 2) / 2, nm = (long)p * (p + 1) / 2;
  long total = np * np + nm * nm;
  LAUNCH(k_reac_split<<<(total + 255) / 256, 256, 0, st>>>(p, full, out));
}

void launch_reac_split_batch(int p, const cplx* full, long stride, const long* offs, int n, cplx* out,
                             cudaStream_t st) {
  long np = (long)(p + 1) * (p + 2) / 2, nm = (long)p * (p + 1) / 2;
  long total = np * np + nm * nm;
  if (n) LAUNCH(k_reac_split_batch<<<dim3((unsigned)((total + 255) / 256), n), 256, 0, st>>>(p, full, stride, offs, out));
}

void launch_mark_reac(int nb, BoxGeom B, const CompGeom* cgs, const int* voff, const int* vidx, unsigned char* used,
                      int* err, cudaStream_t st) {
  if (nb) LAUNCH(k_mark_reac<<<(nb + 127) / 128, 128, 0, st>>>(nb, B, cgs, voff, vidx, used, err));
}


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
// Per-node factors of the reaction M2L integrand for one component and level:
//   A[q][i] = i^n s_t P^_n^m(k_lz/k_l) * w k_rho sigma / k_lz
//   B[q][j] = i^{n'} s_s P^_{n'}^{m'}(k_l'z/k_l')
// with the vertical exponentials applied per class.


// One CTA per (job, row block m): computes the rows with order m of T for all
// columns.  Shared tiles over the quadrature nodes.
#define TQ 16
__global__ void k_reac_T(int p, const ReacJob* __restrict__ jobs, const cplx* __restrict__ kr,
                         const cplx* __restrict__ w, const cplx* __restrict__ kz, int Qall,
                         const cplx* __restrict__ sigma, cplx* __restrict__ ops) {
  const ReacJob jb = jobs[blockIdx.x];
  const int m = (int)blockIdx.y - p;
  const int P = (p + 1) * (p + 1);
  const int nrow = p + 1 - abs(m);
  const int DM = 4 * p + 1;
  extern __shared__ cplx sm[];
  cplx* As = sm;                       // [TQ][nrow]
  cplx* Bs = As + TQ * (p + 1);        // [TQ][P]
  cplx* Js = Bs + TQ * P;              // [TQ][DM]  J_d, d = -2p..2p
  const int nout = nrow * P;
  const int per = (nout + blockDim.x - 1) / blockDim.x;
  cplx acc[8];
  for (int k = 0; k < 8; ++k) acc[k] = C(0, 0);
  for (int q0 = 0; q0 < jb.Q; q0 += TQ) {
    int nq = min(TQ, jb.Q - q0);
    __syncthreads();
    // fill tiles: each thread handles nodes
    for (int t = threadIdx.x; t < nq; t += blockDim.x) {
      int q = q0 + t;
      cplx k_r = kr[q];
      cplx kzl = kz[jb.l * Qall + q], kzp = kz[jb.lp * Qall + q];
      cplx ph_t[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
      // target-layer Legendre functions (rows of order m)
      phat_complex(p, cscale(kzl, 1.0 / jb.kl), cscale(k_r, 1.0 / jb.kl), ph_t);
      cplx base = cdiv(cmul(cmul(w[q], k_r), sigma[jb.sig_off + q]), kzl);
      // vertical exponentials Z~: target factor e^{i k_lz zt}, source e^{i k_l'z zs}
      cplx ez = cexp_(cadd(cmul(C(0, jb.zt), kzl), cmul(C(0, jb.zs), kzp)));
      base = cmul(base, ez);
      int am = abs(m);
      for (int r = 0; r < nrow; ++r) {
        int n = am + r;
        cplx v = ph_t[PH(n, am)];
        if (m < 0 && (am & 1)) v = cneg(v);
        double st = (jb.a == AR_UP) ? 1.0 : sgn_pow(n + m);
        v = cscale(cmul(ipow(n), v), st);
        As[t * (p + 1) + r] = cmul(v, base);
      }
      phat_complex(p, cscale(kzp, 1.0 / jb.klp), cscale(k_r, 1.0 / jb.klp), ph_t);
      for (int j = 0; j < P; ++j) {
        int n = (int)floor(sqrt((double)j)), mm = j - n * n - n, am2 = abs(mm);
        cplx v = ph_t[PH(n, am2)];
        if (mm < 0 && (am2 & 1)) v = cneg(v);
        double ss = (jb.a == AR_UP) ? sgn_pow(n) : sgn_pow(mm);
        Bs[t * P + j] = cscale(cmul(ipow(n), v), ss);
      }
      cplx Jv[2 * (2 * FMM_MAXP) + 1];
      besselJ_all(2 * p, cscale(k_r, jb.rho), Jv);
      for (int d = 0; d <= 2 * p; ++d) {
        Js[t * DM + 2 * p + d] = Jv[d];
        Js[t * DM + 2 * p - d] = cscale(Jv[d], sgn_pow(d));
      }
    }
    __syncthreads();
    for (int k = 0; k < per && k < 8; ++k) {
      int o = threadIdx.x + k * blockDim.x;
      if (o >= nout) break;
      int r = o / P, j = o % P;
      int n2 = (int)floor(sqrt((double)j)), mm = j - n2 * n2 - n2;
      int dd = mm - m + 2 * p;
      cplx a = acc[k];
      for (int t = 0; t < nq; ++t) cfma(a, cmul(As[t * (p + 1) + r], Js[t * DM + dd]), Bs[t * P + j]);
      acc[k] = a;
    }
  }
  for (int k = 0; k < per && k < 8; ++k) {
    int o = threadIdx.x + k * blockDim.x;
    if (o >= nout) break;
    int r = o / P, j = o % P;
    int n = abs(m) + r;
    int i = NM(n, m);
    int n2 = (int)floor(sqrt((double)j)), mm = j - n2 * n2 - n2;
    int d = mm - m;
    double s, c;
    sincos(d * jb.phi, &s, &c);
    cplx pref = cmul(ipow(1 + d), C(c, s));
    ops[jb.out_off + (long)j * P + i] = cmul(pref, acc[k]);
  }
}

// ---------------------------------------------------------------- P2M



__device__ inline void box_center(const CompGeom& cg, int level, const int* coord, double* c) {
  double w = cg.h2 / (double)(1 << level);
  for (int a = 0; a < 3; ++a) c[a] = cg.lo[a] + (coord[a] + 0.5) * w;
}

// point values for expansion: out[(n,m)] = 4 pi j_n(k r) conj(Y_n^m) (conj = true)
// or j_n(k r) Y_n^m (conj = false)
__device__ inline void regular_values(int p, double k, double dx, double dy, double dz, bool conj_y,
                                      double scale, cplx* out) {
  double r, ct, st, ph;
  to_sph(dx, dy, dz, r, ct, st, ph);
  double jn[FMM_MAXP + 1];
  sph_jn(p, k * r, jn);
  double Pa[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
  phat_real(p, ct, st, Pa);
  for (int m = 0; m <= p; ++m) {
    double s, c;
    sincos(m * ph, &s, &c);
    if (conj_y) s = -s;
    for (int n = m; n <= p; ++n) {
      double v = scale * jn[n] * Pa[PH(n, m)];
      out[NM(n, m)] = C(v * c, v * s);
      if (m) {
        double sg = (m & 1) ? -1.0 : 1.0;
        out[NM(n, -m)] = C(sg * v * c, -sg * v * s);
      }
    }
  }
}

#define P2M_CHUNK 16
__global__ void k_p2m(int p, const int* __restrict__ leaves, BoxGeom B, const CompGeom* __restrict__ cgs,
                      const double* __restrict__ spos, const cplx* __restrict__ sq, cplx* __restrict__ M) {
  int b = leaves[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  const CompGeom cg = cgs[B.comp[b]];
  double c[3];
  box_center(cg, B.lev[b], B.coord + 3 * b, c);
  extern __shared__ cplx vals[];     // [P2M_CHUNK][P]
  cplx acc[4] = {C(0, 0), C(0, 0), C(0, 0), C(0, 0)};
  for (int s0 = B.sb[b]; s0 < B.se[b]; s0 += P2M_CHUNK) {
    int ns = min(P2M_CHUNK, B.se[b] - s0);
    __syncthreads();
    for (int t = threadIdx.x; t < ns; t += blockDim.x) {
      int s = s0 + t;
      regular_values(p, cg.ks, spos[3 * s] - c[0], spos[3 * s + 1] - c[1], spos[3 * s + 2] - c[2], true,
                     4.0 * FMM_PI, vals + t * P);
      cplx qv = sq[s];
      for (int i = 0; i < P; ++i) vals[t * P + i] = cmul(vals[t * P + i], qv);
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


__device__ inline long m2l_slot(const CompGeom& cg, int level, const int* ct, const int* cs, int* err) {
  int dx = ct[0] - cs[0], dy = ct[1] - cs[1], dz = ct[2] - cs[2];
  if (cg.kind == CK_FREE) return ((dz + 3) * 7 + (dy + 3)) * 7 + (dx + 3);
  int half = 1 << (level - 1);
  int jt, js;
  if (cg.a == AR_UP) { jt = ct[2] - half; js = half - 1 - cs[2]; }
  else { jt = half - 1 - ct[2]; js = cs[2] - half; }
  if (jt < 0 || jt > 1 || js < 0 || js > 1) { atomicOr(err, 8); return 0; }
  return ((jt * 2 + js) * 7 + (dy + 3)) * 7 + (dx + 3);
}

__global__ void k_m2l(int p, const int* __restrict__ boxes, int with_l2l, BoxGeom B, OpIndex OI,
                      const int* __restrict__ voff, const int* __restrict__ vidx,
                      const cplx* __restrict__ m2l_ops, const cplx* __restrict__ l2l_ops,
                      const cplx* __restrict__ M, cplx* __restrict__ L, int* __restrict__ err) {
  int T = boxes[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  extern __shared__ cplx xs[];
  cplx acc[4] = {C(0, 0), C(0, 0), C(0, 0), C(0, 0)};
  int comp = B.comp[T], lev = B.lev[T];
  const CompGeom cg = OI.cgs[comp];
  if (with_l2l) {
    int pa = B.parent[T];
    for (int i = threadIdx.x; i < P; i += blockDim.x) xs[i] = L[(long)pa * P + i];
    __syncthreads();
    int oct = (B.coord[3 * T] & 1) | ((B.coord[3 * T + 1] & 1) << 1) | ((B.coord[3 * T + 2] & 1) << 2);
    const cplx* op = l2l_ops + OI.l2l_base[comp * 23 + lev] + (long)oct * P * P;
    for (int kk = 0; kk < 4; ++kk) {
      int i = threadIdx.x + kk * blockDim.x;
      if (i >= P) break;
      cplx a = acc[kk];
      for (int j = 0; j < P; ++j) cfma(a, op[(long)j * P + i], xs[j]);
      acc[kk] = a;
    }
  }
  long base = OI.m2l_base[comp * 23 + lev];
  for (int e = voff[T]; e < voff[T + 1]; ++e) {
    int S = vidx[e];
    __syncthreads();
    for (int i = threadIdx.x; i < P; i += blockDim.x) xs[i] = M[(long)S * P + i];
    __syncthreads();
    long slot = m2l_slot(cg, lev, B.coord + 3 * T, B.coord + 3 * S, err);
    const cplx* op = m2l_ops + base + slot * P * P;
    for (int kk = 0; kk < 4; ++kk) {
      int i = threadIdx.x + kk * blockDim.x;
      if (i >= P) break;
      cplx a = acc[kk];
      for (int j = 0; j < P; ++j) cfma(a, op[(long)j * P + i], xs[j]);
      acc[kk] = a;
    }
  }
  for (int kk = 0; kk < 4; ++kk) {
    int i = threadIdx.x + kk * blockDim.x;
    if (i >= P) break;
    L[(long)T * P + i] = acc[kk];
  }
}

// Expand radial reaction integrals (phi = 0) into slots with e^{i (m'-m) phi}.
__global__ void k_phase_expand(int p, const ExpandJob* __restrict__ jobs, const cplx* __restrict__ srcb,
                               cplx* __restrict__ dstb) {
  const int P = (p + 1) * (p + 1);
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)P * P) return;
  const ExpandJob jb = jobs[blockIdx.y];
  const cplx* src = srcb + jb.src;
  cplx* dst = dstb + jb.dst;
  double phi = jb.phi;
  int j = e / P, i = e % P;
  int ni = (int)floor(sqrt((double)i)), mi = i - ni * ni - ni;
  int nj = (int)floor(sqrt((double)j)), mj = j - nj * nj - nj;
  double s, c;
  sincos((mj - mi) * phi, &s, &c);
  dst[e] = cmul(src[e], C(c, s));
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
    sph_jn(p, cg.kt * r, jn);
    double Pa[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
    phat_real(p, ct, st, Pa);
    cplx acc = C(0, 0);
    for (int m = 0; m <= p; ++m) {
      double s, cc;
      sincos(m * ph, &s, &cc);
      for (int n = m; n <= p; ++n) {
        double v = jn[n] * Pa[PH(n, m)];
        cfma(acc, C(v * cc, v * s), Ls[NM(n, m)]);
        if (m) {
          double sg = (m & 1) ? -1.0 : 1.0;
          cfma(acc, C(sg * v * cc, -sg * v * s), Ls[NM(n, -m)]);
        }
      }
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

void launch_reac_T(int p, const ReacJob* jobs, int njobs, const Rule& R, cplx* ops, cudaStream_t st) {
  if (!njobs) return;
  int P = (p + 1) * (p + 1);
  size_t smem = sizeof(cplx) * (TQ * (p + 1) + TQ * P + TQ * (4 * p + 1));
  dim3 grid(njobs, 2 * p + 1);
  int threads = 256;
  while ((p + 1) * P > 8 * threads && threads < 1024) threads *= 2;
  cudaFuncSetAttribute(k_reac_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  LAUNCH(k_reac_T<<<grid, threads, smem, st>>>(p, jobs, R.kr.as<cplx>(), R.w.as<cplx>(), R.kz.as<cplx>(), R.Q(),
                                        R.sigma.as<cplx>(), ops));
}

void launch_p2m(int p, const int* leaves, int n, BoxGeom B, const CompGeom* cgs, const double* spos,
                const cplx* sq, cplx* M, cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  size_t smem = sizeof(cplx) * P2M_CHUNK * P;
  cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (n) LAUNCH(k_p2m<<<n, 128, smem, st>>>(p, leaves, B, cgs, spos, sq, M));
}

void launch_l2p(int p, const int* leaves, int n, BoxGeom B, const CompGeom* cgs, const double* tpos,
                const cplx* L, cplx* phi, cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  if (n) LAUNCH(k_l2p<<<n, 128, sizeof(cplx) * P, st>>>(p, leaves, B, cgs, tpos, L, phi));
}

void launch_m2m(int p, const int* boxes, int n, BoxGeom B, const long* op_base, const cplx* ops, cplx* M,
                cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  if (n) LAUNCH(k_m2m<<<n, 128, sizeof(cplx) * P, st>>>(p, boxes, B, op_base, ops, M));
}

void launch_m2l(int p, const int* boxes, int n, int with_l2l, BoxGeom B, OpIndex OI, const int* voff,
                const int* vidx, const cplx* m2l_ops, const cplx* l2l_ops, const cplx* M, cplx* L, int* err,
                cudaStream_t st) {
  int P = (p + 1) * (p + 1);
  if (n) LAUNCH(k_m2l<<<n, 128, sizeof(cplx) * P, st>>>(p, boxes, with_l2l, B, OI, voff, vidx, m2l_ops, l2l_ops, M, L, err));
}

void launch_phase_expand(int p, const ExpandJob* jobs, int njobs, const cplx* src, cplx* dst, cudaStream_t st) {
  long PP = (long)(p + 1) * (p + 1) * (p + 1) * (p + 1);
  for (int j0 = 0; j0 < njobs; j0 += 60000) {
    int nj = njobs - j0 < 60000 ? njobs - j0 : 60000;
    dim3 grid((unsigned)((PP + 255) / 256), nj);
    LAUNCH(k_phase_expand<<<grid, 256, 0, st>>>(p, jobs + j0, src, dst));
  }
}

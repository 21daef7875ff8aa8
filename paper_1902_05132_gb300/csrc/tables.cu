// Tabulated Sommerfeld integrals of the reaction M2L and their polynomial
// interpolation (Sec. 3.5: eqs. uniformintegral, identitypolyexp, M2Ltable,
// metoletableform; mesh and cost in Sec. 4).
//
// Every entry of a radial reaction M2L matrix (eq. me2lesimplified) is a
// Sommerfeld integral whose integrand carries P^_n^m(k_lz/k_l)
// P^_{n'}^{m'}(k_l'z/k_l').  Written in powers of k_rho (Rodrigues' formula,
// odd degrees carrying one factor k/k_z),
//   P^_n^m(k_z/k) = tau_m (k/k_z)^mu sum_s b^s_{n|m|} (k_rho/k)^{|m|+2s},
//   mu = (n+|m|) mod 2, tau_m = (-1)^m for m < 0,
// the entry becomes a short sum over integrals that do not depend on
// (n, m, n', m'):
//   S_{q,t,mu,nu}(rho, zt, zs) = int k_rho^{t+1} J_q(k_rho rho) Z~ sigma / k_lz
//                                (k_l/k_lz)^mu (k_l'/k_l'z)^nu dk_rho,
//   T_{nm,n'm'} = i^{n+n'+1+m'-m} s_t s_s sum_s A^s S_{|m'-m|, |m|+|m'|+2s, mu, nu}
// (A^s of eq. asslegendreexpcoef with the signs tau and J_{-q} = (-1)^q J_q
// folded in; s_t, s_s the arrow signs of the direct operator in ops.cu).
//
// The integrals are tabulated once per medium (at create, flag FMM_TABLES)
// over the domain the trees can ask for: a reaction V pair at box width w
// has its centres (jt + 1/2) w and (js + 1/2) w from the interface (jt, js in
// {0, 1}) and rho = w sqrt(dx^2 + dy^2) (ten values), i.e. it lies on one of
// 40 rays through the origin of (rho, zt, zs).  Along a ray the coordinate is
// u = log2(k_max w) in [-8, 1.5], cut into panels (whole octaves below -3,
// half octaves to -1, quarter octaves above); on each panel S * w^(t+2) is
// stored at 12 Chebyshev points of the first kind and interpolated by the
// barycentric formula.  The factor w^(t+2) takes out the growth of S as
// w -> 0.  A geometry then needs no quadrature for its reaction operators:
// each class is an interpolation of every S plus the sum above.
//
// Table quadrature: the contour of the handle's rule up to ta (complex
// nodes) and, per panel, a real-axis tail from ta to ta + (30 + 7p)/w0
// (w0 the panel's smallest width, jt = js = 0) in Gauss-Legendre panels whose
// length grows from 2 to 6 / max(rho, H) of the panel's widest class, so that
// the node count per table point does not grow as w shrinks.  On the tail
// every k_jz = i kappa_j and sigma are real, so the tail sums run in real
// arithmetic with the constant phase (-i)^{1+mu+nu} applied at the end.
#include <cmath>
#include <vector>

#include "fmm_internal.h"
#include "table_algebra.h"

namespace {

constexpr int kCheb = 12;                 // interpolation points per panel
constexpr int kRays = 40;                 // (jt * 2 + js) * 10 + r
constexpr int kPanels = 19;
constexpr double kEdges[kPanels + 1] = {-8.0, -7.0, -6.0, -5.0, -4.0, -3.0, -2.5, -2.0, -1.5, -1.0, -0.75,
                                        -0.5, -0.25, 0.0,  0.25, 0.5,  0.75, 1.0,  1.25, 1.5};
// device copies of the panel edges and radial classes
__constant__ double c_edges[kPanels + 1] = {-8.0, -7.0, -6.0, -5.0, -4.0, -3.0, -2.5, -2.0, -1.5, -1.0, -0.75,
                                            -0.5, -0.25, 0.0,  0.25, 0.5,  0.75, 1.0,  1.25, 1.5};
__constant__ int c_rho2[10] = {0, 1, 2, 4, 5, 8, 9, 10, 13, 18};
constexpr int kBuildThreads = 128;        // table build: threads per point, nodes per chunk
constexpr int kAccPerThread = 8;          // tables per thread (ntab <= 1024)
constexpr int kTailGL = 16;               // Gauss-Legendre nodes per tail panel

// ---------------------------------------------------------------- host algebra
// (table_algebra.h: power forms, index set, CSR of eq. metoletableform)
using tabalg::PowerForms;
using tabalg::TabIndex;

void build_terms(int p, const PowerForms& F, const TabIndex& X, double kl, double klp, int a,
                 std::vector<int>& off, std::vector<int>& tab, std::vector<cplx>& coef) {
  std::vector<double> re, im;
  tabalg::build_terms(p, F, X, kl, klp, a, off, tab, re, im);
  coef.resize(re.size());
  for (size_t i = 0; i < re.size(); ++i) coef[i] = C(re[i], im[i]);
}

// ---------------------------------------------------------------- table build
struct TabBuildArgs {
  int p, ntab, tmax, L1;
  const int4* idx;                      // (q, t, mu, nu) per table
  const int4* slot;                     // (l, l', a, b) per slot
  const double* k;                      // wave numbers [L1]
  double kmax;
  // complex contour nodes (the handle's rule, nodes [0, n_near))
  int n_near, Qh;
  const cplx *kr_n, *w_n, *kz_n, *sig_n;        // kz [L1][Qh], sigma [L1][L1][2][2][Qh]
  // real-axis tails of the panels, concatenated
  int Nt;
  const int* tail_off;                  // [kPanels + 1]
  const double *t_t, *w_t;
  const cplx *kz_t, *sig_t;             // kz [L1][Nt], sigma [L1][L1][2][2][Nt]
  cplx* vals;                           // [slot][ray][panel][kCheb][ntab]
};

__device__ inline double cheb_x(int j) { return cos((2 * j + 1) * FMM_PI / (2.0 * kCheb)); }

// One CTA per table point (slot, ray, panel, Chebyshev point).  Node data of
// a chunk of kBuildThreads nodes (one thread each) go to shared memory as
//   c[mu nu][node], J_q[node] (q = 0..2p), k_rho^t[node] (t = 0..tmax);
// then each thread sums its tables over the chunk.
__global__ void __launch_bounds__(kBuildThreads) k_tab_build(TabBuildArgs A) {
  extern __shared__ double sm[];
  const int NQ = kBuildThreads;
  const int nq_ = 2 * A.p + 1, nt_ = A.tmax + 1;
  int pt = blockIdx.x;
  const int node = pt % kCheb;
  pt /= kCheb;
  const int panel = pt % kPanels;
  pt /= kPanels;
  const int ray = pt % kRays;
  const int slot = pt / kRays;
  const int4 sl = A.slot[slot];
  const int l = sl.x, lp = sl.y;
  const int row = ((l * A.L1 + lp) * 2 + sl.z) * 2 + sl.w;
  const double kl = A.k[l], klp = A.k[lp];
  const double u = c_edges[panel] + 0.5 * (c_edges[panel + 1] - c_edges[panel]) * (cheb_x(node) + 1.0);
  const double w = exp2(u) / A.kmax;
  const int g = ray / 10, r = ray % 10;
  const double rho = sqrt((double)c_rho2[r]) * w, zt = ((g >> 1) + 0.5) * w, zs = ((g & 1) + 0.5) * w;

  // tables of this thread: threadIdx.x + k * NQ, k < nk
  const int nk = (A.ntab > (int)threadIdx.x) ? min(kAccPerThread, (A.ntab - (int)threadIdx.x + NQ - 1) / NQ) : 0;
  int4 my[kAccPerThread];
  cplx accn[kAccPerThread];
  double acct[kAccPerThread];
#pragma unroll
  for (int k = 0; k < kAccPerThread; ++k) {
    my[k] = (k < nk) ? A.idx[threadIdx.x + k * NQ] : make_int4(0, 0, 0, 0);
    accn[k] = C(0, 0);
    acct[k] = 0.0;
  }

  // ---- complex contour nodes
  {
    cplx* cc = (cplx*)sm;
    cplx* cJ = cc + 4 * NQ;
    cplx* cP = cJ + nq_ * NQ;
    for (int q0 = 0; q0 < A.n_near; q0 += NQ) {
      const int nq = min(NQ, A.n_near - q0);
      __syncthreads();
      if (threadIdx.x < nq) {
        const int q = q0 + threadIdx.x, t = threadIdx.x;
        cplx kr = A.kr_n[q];
        cplx kzl = A.kz_n[(long)l * A.Qh + q], kzp = A.kz_n[(long)lp * A.Qh + q];
        cplx sg = A.sig_n[(long)row * A.Qh + q];
        cplx e = cexp_(cadd(cmul(C(0, zt), kzl), cmul(C(0, zs), kzp)));
        cplx base = cdiv(cmul(cmul(cmul(A.w_n[q], kr), e), sg), kzl);
        cplx rl = cdiv(C(kl, 0), kzl), rlp = cdiv(C(klp, 0), kzp);
        cc[0 * NQ + t] = base;
        cc[1 * NQ + t] = cmul(base, rlp);
        cc[2 * NQ + t] = cmul(base, rl);
        cc[3 * NQ + t] = cmul(cmul(base, rl), rlp);
        cplx J[2 * FMM_MAXP + 1];
        besselJ_all(2 * A.p, cscale(kr, rho), J);
        for (int d = 0; d < nq_; ++d) cJ[d * NQ + t] = J[d];
        cplx pw = C(1, 0);
        for (int s = 0; s < nt_; ++s) { cP[s * NQ + t] = pw; pw = cmul(pw, kr); }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kAccPerThread; ++k) {
        if (k >= nk) break;
        const cplx* c0 = cc + (my[k].z * 2 + my[k].w) * NQ;
        const cplx* j0 = cJ + my[k].x * NQ;
        const cplx* p0 = cP + my[k].y * NQ;
        cplx a = accn[k];
        for (int t = 0; t < nq; ++t) a = cadd(a, cmul(c0[t], cmul(j0[t], p0[t])));
        accn[k] = a;
      }
    }
  }
  // ---- real-axis tail of this panel (k_jz = i kappa_j, sigma real)
  {
    double* rc = sm;
    double* rJ = rc + 4 * NQ;
    double* rP = rJ + nq_ * NQ;
    const int t_lo = A.tail_off[panel], t_hi = A.tail_off[panel + 1];
    for (int q0 = t_lo; q0 < t_hi; q0 += NQ) {
      const int nq = min(NQ, t_hi - q0);
      __syncthreads();
      if (threadIdx.x < nq) {
        const int q = q0 + threadIdx.x, t = threadIdx.x;
        const double tk = A.t_t[q];
        const double kapl = A.kz_t[(long)l * A.Nt + q].y, kapp = A.kz_t[(long)lp * A.Nt + q].y;
        const double sg = A.sig_t[(long)row * A.Nt + q].x;
        const double b = A.w_t[q] * tk * exp(-kapl * zt - kapp * zs) * sg / kapl;
        const double rl = kl / kapl, rlp = klp / kapp;
        rc[0 * NQ + t] = b;
        rc[1 * NQ + t] = b * rlp;
        rc[2 * NQ + t] = b * rl;
        rc[3 * NQ + t] = b * rl * rlp;
        const double x = tk * rho;
        if (x == 0.0) {
          rJ[t] = 1.0;
          for (int d = 1; d < nq_; ++d) rJ[d * NQ + t] = 0.0;
        } else if (x > 2.0 * A.p + 2.0) {
          // upward recurrence is stable for orders below the argument
          double ja = j0(x), jb = j1(x);
          rJ[t] = ja;
          if (nq_ > 1) rJ[NQ + t] = jb;
          for (int d = 1; d + 1 < nq_; ++d) {
            double jc = 2.0 * d / x * jb - ja;
            ja = jb;
            jb = jc;
            rJ[(d + 1) * NQ + t] = jc;
          }
        } else {
          cplx J[2 * FMM_MAXP + 1];
          besselJ_all(2 * A.p, C(x, 0.0), J);
          for (int d = 0; d < nq_; ++d) rJ[d * NQ + t] = J[d].x;
        }
        double pw = 1.0;
        for (int s = 0; s < nt_; ++s) { rP[s * NQ + t] = pw; pw *= tk; }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kAccPerThread; ++k) {
        if (k >= nk) break;
        const double* c0 = rc + (my[k].z * 2 + my[k].w) * NQ;
        const double* j0p = rJ + my[k].x * NQ;
        const double* p0 = rP + my[k].y * NQ;
        double a = acct[k];
        for (int t = 0; t < nq; ++t) a = fma(c0[t] * j0p[t], p0[t], a);
        acct[k] = a;
      }
    }
  }
  // tail phase (-i)^{1+mu+nu}: base = -i b, k/k_z = -i k/kappa
  const long out = (long)blockIdx.x * A.ntab;
#pragma unroll
  for (int k = 0; k < kAccPerThread; ++k) {
    if (k >= nk) break;
    const int i = threadIdx.x + k * NQ;
    const int e = 1 + my[k].z + my[k].w;
    cplx ph = ipow((4 - (e & 3)) & 3);                    // (-i)^e = i^{-e}
    cplx v = cadd(accn[k], cscale(ph, acct[k]));
    A.vals[out + i] = cscale(v, pow(w, (double)(my[k].y + 2)));
  }
}

// ---------------------------------------------------------------- interpolation
struct TabJob {
  int slot, ray, panel;
  long term0;                           // offset of the entry (0, 0) in term_off
  double x, w;                          // Chebyshev coordinate in the panel, box width
  long full_off;                        // output: full radial matrix, input-major [j][i]
};

// One CTA per class: interpolate every S at the class's width (barycentric
// formula on the panel's 12 points, then divide by w^(t+2)), then sum each
// entry of the radial matrix from its CSR terms (eq. metoletableform).
__global__ void k_tab_T(int p, int ntab, const int4* __restrict__ idx, const cplx* __restrict__ vals,
                        const TabJob* __restrict__ jobs, const int* __restrict__ term_off,
                        const int* __restrict__ term_tab, const cplx* __restrict__ term_coef,
                        cplx* __restrict__ full) {
  extern __shared__ cplx sS[];
  const TabJob J = jobs[blockIdx.x];
  const cplx* V = vals + ((((long)J.slot * kRays + J.ray) * kPanels + J.panel) * kCheb) * ntab;
  double lam[kCheb];
  int hit = -1;
  double den = 0.0;
#pragma unroll
  for (int j = 0; j < kCheb; ++j) {
    double xj = cheb_x(j), dx = J.x - xj;
    if (dx == 0.0) hit = j;
    lam[j] = ((j & 1) ? -1.0 : 1.0) * sin((2 * j + 1) * FMM_PI / (2.0 * kCheb)) / dx;
    den += lam[j];
  }
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) {
    cplx v;
    if (hit >= 0) {
      v = V[(long)hit * ntab + i];
    } else {
      v = C(0, 0);
#pragma unroll
      for (int j = 0; j < kCheb; ++j) v = cadd(v, cscale(V[(long)j * ntab + i], lam[j]));
      v = cscale(v, 1.0 / den);
    }
    sS[i] = cscale(v, pow(J.w, -(double)(idx[i].y + 2)));
  }
  __syncthreads();
  const int P = (p + 1) * (p + 1);
  const int* off = term_off + J.term0;
  for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
    cplx acc = C(0, 0);
    for (int x = off[e]; x < off[e + 1]; ++x) cfma(acc, term_coef[x], sS[term_tab[x]]);
    const int i = e / P, j = e % P;
    full[J.full_off + (long)j * P + i] = acc;
  }
}

}  // namespace

void launch_reac_split_batch(int p, const cplx* full, long stride, const long* offs, int n, cplx* out,
                             cudaStream_t st);
void launch_sigma_at(fmm_layered* h, int Q, const cplx* kr, cplx* kz, cplx* sigma, cudaStream_t st);
void gauss_legendre_pub(int n, std::vector<double>& x, std::vector<double>& w);

static int tab_slot_index(const fmm_layered* h, int l, int lp, int a, int b) {
  return ((l * h->L1 + lp) * 2 + a) * 2 + b;
}

static void near_tables_build(fmm_layered* h, const std::vector<int4>& slots, cudaStream_t st);

// Build the tables of every reaction component of the medium (create time).
void tables_build(fmm_layered* h, cudaStream_t st) {
  TabState& T = h->tabs;
  const int p = h->p, L1 = h->L1;
  if (L1 < 2) return;
  if (p > 12) throw FmmError(FMM_ERR_UNSUPPORTED, "FMM_TABLES supports p <= 12");
  cudaEvent_t e0, e1;
  FMM_CHECK(cudaEventCreate(&e0));
  FMM_CHECK(cudaEventCreate(&e1));
  FMM_CHECK(cudaEventRecord(e0, st));
  PowerForms F(p);
  TabIndex X;
  X.build(p, F);
  T.ntab = X.size();
  if (T.ntab > kAccPerThread * kBuildThreads) throw FmmError(FMM_ERR_UNSUPPORTED, "too many tables");
  int tmax = 0;
  for (int i = 0; i < T.ntab; ++i) tmax = std::max(tmax, X.key[4 * i + 1]);
  // reaction components of the medium (every layer pair and valid arrows)
  std::vector<int4> slots;
  T.slot_of.assign((size_t)L1 * L1 * 4, -1);
  T.term_base.assign((size_t)L1 * L1 * 2, -1);
  std::vector<int> off_all, tab_all;
  std::vector<cplx> coef_all;
  const int L = L1 - 1;
  for (int l = 0; l < L1; ++l)
    for (int lp = 0; lp < L1; ++lp)
      for (int a = 0; a < 2; ++a) {
        if (!((a == AR_UP) ? (l < L) : (l > 0))) continue;
        for (int b = 0; b < 2; ++b) {
          if (!((b == AR_UP) ? (lp < L) : (lp > 0))) continue;
          T.slot_of[tab_slot_index(h, l, lp, a, b)] = (int)slots.size();
          slots.push_back(make_int4(l, lp, a, b));
        }
        std::vector<int> off, tab;
        std::vector<cplx> coef;
        build_terms(p, F, X, h->k[l], h->k[lp], a, off, tab, coef);
        T.term_base[(l * L1 + lp) * 2 + a] = (long)off_all.size();
        const int base = (int)tab_all.size();
        for (int v : off) off_all.push_back(v + base);
        tab_all.insert(tab_all.end(), tab.begin(), tab.end());
        coef_all.insert(coef_all.end(), coef.begin(), coef.end());
      }
  T.nslot = (int)slots.size();
  T.kmax = 0;
  for (double v : h->k) T.kmax = std::max(T.kmax, v);
  // real-axis tails of the panels
  std::vector<double> xg, wg, tt, tw;
  gauss_legendre_pub(kTailGL, xg, wg);
  std::vector<int> tail_off(kPanels + 1, 0);
  const double ta = h->rule.ta;
  for (int k = 0; k < kPanels; ++k) {
    const double w0 = std::exp2(kEdges[k]) / T.kmax, w1 = std::exp2(kEdges[k + 1]) / T.kmax;
    const double tend = ta + (30.0 + 7.0 * p) / w0;
    const double lmax = 6.0 / (std::sqrt(18.0) * w1);
    double len = std::min(2.0, lmax), t = ta;
    while (t < tend) {
      for (int i = 0; i < kTailGL; ++i) {
        tt.push_back(t + 0.5 * len * (xg[i] + 1.0));
        tw.push_back(0.5 * len * wg[i]);
      }
      t += len;
      len = std::min(1.5 * len, std::max(len, lmax));
    }
    tail_off[k + 1] = (int)tt.size();
  }
  const int Nt = (int)tt.size();
  // device copies: tails with sigma, indices, slots, terms (temporaries freed on return)
  struct Tmp {
    DevBuf kr, tt, tw, kz, sig, toff, slot;
    ~Tmp() { kr.release(); tt.release(); tw.release(); kz.release(); sig.release(); toff.release(); slot.release(); }
  } tmp;
  DevBuf &d_kr = tmp.kr, &d_tt = tmp.tt, &d_tw = tmp.tw, &d_kz = tmp.kz, &d_sig = tmp.sig, &d_toff = tmp.toff,
         &d_slot = tmp.slot;
  std::vector<cplx> krc(Nt);
  for (int i = 0; i < Nt; ++i) krc[i] = C(tt[i], 0.0);
  d_kr.ensure(sizeof(cplx) * Nt);
  d_tt.ensure(sizeof(double) * Nt);
  d_tw.ensure(sizeof(double) * Nt);
  d_kz.ensure(sizeof(cplx) * (size_t)Nt * L1);
  d_sig.ensure(sizeof(cplx) * (size_t)Nt * L1 * L1 * 4);
  d_toff.ensure(sizeof(int) * tail_off.size());
  d_slot.ensure(sizeof(int4) * slots.size());
  FMM_CHECK(cudaMemcpyAsync(d_kr.ptr, krc.data(), sizeof(cplx) * Nt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(d_tt.ptr, tt.data(), sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(d_tw.ptr, tw.data(), sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(d_toff.ptr, tail_off.data(), sizeof(int) * tail_off.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(d_slot.ptr, slots.data(), sizeof(int4) * slots.size(), cudaMemcpyHostToDevice, st));
  launch_sigma_at(h, Nt, d_kr.as<cplx>(), d_kz.as<cplx>(), d_sig.as<cplx>(), st);
  std::vector<int4> idx(T.ntab);
  for (int i = 0; i < T.ntab; ++i) idx[i] = make_int4(X.key[4 * i], X.key[4 * i + 1], X.key[4 * i + 2], X.key[4 * i + 3]);
  T.idx.ensure(sizeof(int4) * T.ntab);
  FMM_CHECK(cudaMemcpyAsync(T.idx.ptr, idx.data(), sizeof(int4) * T.ntab, cudaMemcpyHostToDevice, st));
  T.term_off.ensure(sizeof(int) * off_all.size());
  T.term_tab.ensure(sizeof(int) * tab_all.size() + 16);
  T.term_coef.ensure(sizeof(cplx) * coef_all.size() + 16);
  FMM_CHECK(cudaMemcpyAsync(T.term_off.ptr, off_all.data(), sizeof(int) * off_all.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(T.term_tab.ptr, tab_all.data(), sizeof(int) * tab_all.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(T.term_coef.ptr, coef_all.data(), sizeof(cplx) * coef_all.size(), cudaMemcpyHostToDevice, st));
  const long npts = (long)T.nslot * kRays * kPanels * kCheb;
  T.vals.ensure(sizeof(cplx) * (size_t)npts * T.ntab);
  TabBuildArgs A{};
  A.p = p; A.ntab = T.ntab; A.tmax = tmax; A.L1 = L1;
  A.idx = T.idx.as<int4>(); A.slot = d_slot.as<int4>(); A.k = h->d_k.as<double>(); A.kmax = T.kmax;
  A.n_near = h->rule.n_near; A.Qh = h->rule.Q();
  A.kr_n = h->rule.kr.as<cplx>(); A.w_n = h->rule.w.as<cplx>();
  A.kz_n = h->rule.kz.as<cplx>(); A.sig_n = h->rule.sigma.as<cplx>();
  A.Nt = Nt; A.tail_off = d_toff.as<int>(); A.t_t = d_tt.as<double>(); A.w_t = d_tw.as<double>();
  A.kz_t = d_kz.as<cplx>(); A.sig_t = d_sig.as<cplx>();
  A.vals = T.vals.as<cplx>();
  const size_t smem = sizeof(cplx) * (size_t)kBuildThreads * (4 + 2 * p + 1 + tmax + 1);
  FMM_CHECK(cudaFuncSetAttribute(k_tab_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LAUNCH(k_tab_build<<<(unsigned)npts, kBuildThreads, smem, st>>>(A));
  FMM_CHECK(cudaGetLastError());
  T.bytes = sizeof(cplx) * (size_t)npts * T.ntab + sizeof(cplx) * coef_all.size() +
            sizeof(int) * (tab_all.size() + off_all.size());
  near_tables_build(h, slots, st);
  FMM_CHECK(cudaEventRecord(e1, st));
  FMM_CHECK(cudaStreamSynchronize(st));      // before the temporaries are freed
  float ms = 0;
  FMM_CHECK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  T.build_ms = ms;
  T.built = true;
}

bool tables_cover(const fmm_layered* h, double w) {
  if (!h->tabs.built) return false;
  const double u = std::log2(h->tabs.kmax * w);
  return u >= kEdges[0] && u <= kEdges[kPanels];
}

static TabJob make_job(const fmm_layered* h, const TabClass& c, long full_off) {
  const TabState& T = h->tabs;
  TabJob J{};
  J.slot = T.slot_of[tab_slot_index(h, c.l, c.lp, c.a, c.b)];
  J.ray = (c.jt * 2 + c.js) * 10 + c.r;
  const double u = std::log2(T.kmax * c.w);
  int k = 0;
  while (k + 1 < kPanels && u >= kEdges[k + 1]) ++k;
  J.panel = k;
  J.x = 2.0 * (u - kEdges[k]) / (kEdges[k + 1] - kEdges[k]) - 1.0;
  J.w = c.w;
  J.term0 = T.term_base[(c.l * h->L1 + c.lp) * 2 + c.a];
  J.full_off = full_off;
  if (J.slot < 0 || J.term0 < 0) throw FmmError(FMM_ERR_ARG, "no table for this reaction component");
  return J;
}

// Radial operators of the given classes from the tables, split into the
// symmetric basis at rad + cls[i].split_off (the layout k_reac_split writes).
void tables_ops(fmm_layered* h, const std::vector<TabClass>& cls, cplx* rad, cudaStream_t st) {
  if (cls.empty()) return;
  TabState& T = h->tabs;
  const int p = h->p, P = (p + 1) * (p + 1);
  const int batch = 128;
  std::vector<TabJob> jobs;
  std::vector<long> soffs;
  for (size_t i = 0; i < cls.size(); ++i) {
    jobs.push_back(make_job(h, cls[i], (long)(i % batch) * P * P));
    soffs.push_back(cls[i].split_off);
  }
  T.jobs.ensure(sizeof(TabJob) * jobs.size());
  T.split_offs.ensure(sizeof(long) * soffs.size());
  T.full.ensure(sizeof(cplx) * (size_t)batch * P * P);
  FMM_CHECK(cudaMemcpyAsync(T.jobs.ptr, jobs.data(), sizeof(TabJob) * jobs.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(T.split_offs.ptr, soffs.data(), sizeof(long) * soffs.size(), cudaMemcpyHostToDevice, st));
  for (size_t b0 = 0; b0 < cls.size(); b0 += batch) {
    const int nb = (int)std::min<size_t>(batch, cls.size() - b0);
    LAUNCH(k_tab_T<<<nb, 256, sizeof(cplx) * T.ntab, st>>>(p, T.ntab, T.idx.as<int4>(), T.vals.as<cplx>(),
                                                        T.jobs.as<TabJob>() + b0, T.term_off.as<int>(),
                                                        T.term_tab.as<int>(), T.term_coef.as<cplx>(),
                                                        T.full.as<cplx>()));
    launch_reac_split_batch(p, T.full.as<cplx>(), (long)P * P, T.split_offs.as<long>() + b0, nb, rad, st);
  }
  FMM_CHECK(cudaGetLastError());
}

// One class, full radial matrix row-major [(n,m)][(n',m')] to host memory.
void tables_operator_host(fmm_layered* h, const TabClass& c, double* out, cudaStream_t st) {
  TabState& T = h->tabs;
  if (!tables_cover(h, c.w)) throw FmmError(FMM_ERR_ARG, "box width outside the tables (or no tables)");
  if (c.jt < 0 || c.jt > 1 || c.js < 0 || c.js > 1 || c.r < 0 || c.r > 9) throw FmmError(FMM_ERR_ARG, "class out of range");
  const int P = (h->p + 1) * (h->p + 1);
  TabJob J = make_job(h, c, 0);
  T.jobs.ensure(sizeof(TabJob));
  T.full.ensure(sizeof(cplx) * (size_t)P * P);
  FMM_CHECK(cudaMemcpyAsync(T.jobs.ptr, &J, sizeof(TabJob), cudaMemcpyHostToDevice, st));
  LAUNCH(k_tab_T<<<1, 256, sizeof(cplx) * T.ntab, st>>>(h->p, T.ntab, T.idx.as<int4>(), T.vals.as<cplx>(),
                                                     T.jobs.as<TabJob>(), T.term_off.as<int>(), T.term_tab.as<int>(),
                                                     T.term_coef.as<cplx>(), T.full.as<cplx>()));
  FMM_CHECK(cudaGetLastError());
  std::vector<cplx> f((size_t)P * P);
  FMM_CHECK(cudaMemcpyAsync(f.data(), T.full.ptr, sizeof(cplx) * f.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      out[2 * ((size_t)i * P + j)] = f[(size_t)j * P + i].x;
      out[2 * ((size_t)i * P + j) + 1] = f[(size_t)j * P + i].y;
    }
}

// ---------------------------------------------------------------- near-field kernel table
namespace {

struct NtBuildArgs {
  const int4* slot;
  const double* k;
  double kmax;
  int L1;
  int n_near, Qh;
  const cplx *kr_n, *w_n, *kz_n, *sig_n;
  int Nt;
  const int* tail_off;                  // [NT_PANELS + 1]
  const double *t_t, *w_t;
  const cplx *kz_t, *sig_t;             // kz [L1][Nt], sigma [L1][L1][2][2][Nt]
  const double* cheb;                   // NT_CHEB_LEN
  cplx* vals;
};

// One CTA per grid line (slot, panel, u point, theta point): the quadrature
// of u~ at its NT_NF points f, threads splitting the contour nodes, then a
// block reduction; the table keeps R u~.
__global__ void __launch_bounds__(128) k_ntab_build(NtBuildArgs A) {
  int b = blockIdx.x;
  const int j = b % NT_NTH;
  b /= NT_NTH;
  const int i = b % NT_NU;
  b /= NT_NU;
  const int panel = b % NT_PANELS;
  const int slot = b / NT_PANELS;
  const int4 sl = A.slot[slot];
  const int l = sl.x, lp = sl.y;
  const int row = ((l * A.L1 + lp) * 2 + sl.z) * 2 + sl.w;
  const double* X = A.cheb;
  const double lo = nt_edge(panel), hi = nt_edge(panel + 1);
  const double u = lo + 0.5 * (hi - lo) * (X[i] + 1.0);
  const double R = exp2(u) / A.kmax;
  const double th = 0.5 * nt_theta_max() * (X[2 * NT_NU + j] + 1.0);
  const double H = R * cos(th), rho = R * sin(th);
  double zt[NT_NF], zs[NT_NF];
#pragma unroll
  for (int m = 0; m < NT_NF; ++m) {
    const double f = 0.5 * (X[2 * NT_NU + 2 * NT_NTH + m] + 1.0);
    zt[m] = f * H;
    zs[m] = (1.0 - f) * H;
  }
  double ar[NT_NF], ai[NT_NF], at[NT_NF];
#pragma unroll
  for (int m = 0; m < NT_NF; ++m) ar[m] = ai[m] = at[m] = 0.0;
  // complex contour: coef = (i/4pi) w k_rho sigma / k_lz
  for (int q = threadIdx.x; q < A.n_near; q += blockDim.x) {
    const cplx kr = A.kr_n[q];
    const cplx kzl = A.kz_n[(long)l * A.Qh + q], kzp = A.kz_n[(long)lp * A.Qh + q];
    const cplx sg = A.sig_n[(long)row * A.Qh + q];
    cplx c = cmul(C(0.0, 1.0 / (4.0 * FMM_PI)), cdiv(cmul(cmul(A.w_n[q], kr), sg), kzl));
    cplx J[1];
    besselJ_all(0, cscale(kr, rho), J);
    c = cmul(c, J[0]);
#pragma unroll
    for (int m = 0; m < NT_NF; ++m) {
      const cplx v = cmul(c, cexp_(cadd(cmul(C(0, zt[m]), kzl), cmul(C(0, zs[m]), kzp))));
      ar[m] += v.x;
      ai[m] += v.y;
    }
  }
  // real tail: k_jz = i kappa_j, coef = w t sigma / (4 pi kappa_l)
  for (int q = A.tail_off[panel] + threadIdx.x; q < A.tail_off[panel + 1]; q += blockDim.x) {
    const double t = A.t_t[q];
    const double kapl = A.kz_t[(long)l * A.Nt + q].y, kapp = A.kz_t[(long)lp * A.Nt + q].y;
    const double c = A.w_t[q] * t * A.sig_t[(long)row * A.Nt + q].x / (4.0 * FMM_PI * kapl) * j0(t * rho);
#pragma unroll
    for (int m = 0; m < NT_NF; ++m) at[m] += c * exp(-kapl * zt[m] - kapp * zs[m]);
  }
  // block reduction: warps by shuffles, then the four warp sums in order
  __shared__ double red[4][3 * NT_NF];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NT_NF; ++m) {
    for (int o = 16; o > 0; o >>= 1) {
      ar[m] += __shfl_xor_sync(0xffffffffu, ar[m], o);
      ai[m] += __shfl_xor_sync(0xffffffffu, ai[m], o);
      at[m] += __shfl_xor_sync(0xffffffffu, at[m], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NT_NF; ++m) {
      red[warp][m] = ar[m];
      red[warp][NT_NF + m] = ai[m];
      red[warp][2 * NT_NF + m] = at[m];
    }
  }
  __syncthreads();
  if (threadIdx.x < NT_NF) {
    const int m = threadIdx.x;
    double sr = 0.0, si = 0.0, st = 0.0;
    for (int w = 0; w < 4; ++w) {
      sr += red[w][m];
      si += red[w][NT_NF + m];
      st += red[w][2 * NT_NF + m];
    }
    A.vals[(long)blockIdx.x * NT_NF + m] = C(R * (sr + st), R * si);
  }
}

}  // namespace

// Near-field kernel table of every reaction component (create time, with the
// M2L tables).
static void near_tables_build(fmm_layered* h, const std::vector<int4>& slots, cudaStream_t st) {
  TabState& T = h->tabs;
  const int L1 = h->L1;
  // Chebyshev points and barycentric weights of the three coordinates
  std::vector<double> cheb;
  for (int n : {NT_NU, NT_NTH, NT_NF}) {
    for (int j = 0; j < n; ++j) cheb.push_back(std::cos((2 * j + 1) * FMM_PI / (2.0 * n)));
    for (int j = 0; j < n; ++j) cheb.push_back(((j & 1) ? -1.0 : 1.0) * std::sin((2 * j + 1) * FMM_PI / (2.0 * n)));
  }
  // real-axis tails per panel: to ta + FMM_NEAR_TAIL_DECAY / H_min, H_min =
  // R0 cos(theta_max), panels growing from 2 to 6 / R1
  std::vector<double> xg, wg, tt, tw;
  gauss_legendre_pub(kTailGL, xg, wg);
  std::vector<int> tail_off(NT_PANELS + 1, 0);
  const double ta = h->rule.ta;
  for (int k = 0; k < NT_PANELS; ++k) {
    const double R0 = std::exp2(nt_edge(k)) / T.kmax, R1 = std::exp2(nt_edge(k + 1)) / T.kmax;
    const double tend = ta + FMM_NEAR_TAIL_DECAY / (R0 * std::cos(nt_theta_max()));
    const double lmax = 6.0 / R1;
    double len = std::min(2.0, lmax), t = ta;
    while (t < tend) {
      for (int i = 0; i < kTailGL; ++i) {
        tt.push_back(t + 0.5 * len * (xg[i] + 1.0));
        tw.push_back(0.5 * len * wg[i]);
      }
      t += len;
      len = std::min(1.5 * len, std::max(len, lmax));
    }
    tail_off[k + 1] = (int)tt.size();
  }
  const int Nt = (int)tt.size();
  struct Tmp {
    DevBuf kr, tt, tw, kz, sig, toff, slot;
    ~Tmp() { kr.release(); tt.release(); tw.release(); kz.release(); sig.release(); toff.release(); slot.release(); }
  } tmp;
  std::vector<cplx> krc(Nt);
  for (int i = 0; i < Nt; ++i) krc[i] = C(tt[i], 0.0);
  tmp.kr.ensure(sizeof(cplx) * Nt);
  tmp.tt.ensure(sizeof(double) * Nt);
  tmp.tw.ensure(sizeof(double) * Nt);
  tmp.kz.ensure(sizeof(cplx) * (size_t)Nt * L1);
  tmp.sig.ensure(sizeof(cplx) * (size_t)Nt * L1 * L1 * 4);
  tmp.toff.ensure(sizeof(int) * tail_off.size());
  tmp.slot.ensure(sizeof(int4) * slots.size());
  FMM_CHECK(cudaMemcpyAsync(tmp.kr.ptr, krc.data(), sizeof(cplx) * Nt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(tmp.tt.ptr, tt.data(), sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(tmp.tw.ptr, tw.data(), sizeof(double) * Nt, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(tmp.toff.ptr, tail_off.data(), sizeof(int) * tail_off.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(tmp.slot.ptr, slots.data(), sizeof(int4) * slots.size(), cudaMemcpyHostToDevice, st));
  launch_sigma_at(h, Nt, tmp.kr.as<cplx>(), tmp.kz.as<cplx>(), tmp.sig.as<cplx>(), st);
  T.ncheb.ensure(sizeof(double) * cheb.size());
  FMM_CHECK(cudaMemcpyAsync(T.ncheb.ptr, cheb.data(), sizeof(double) * cheb.size(), cudaMemcpyHostToDevice, st));
  T.nslot_map.ensure(sizeof(int) * T.slot_of.size());
  FMM_CHECK(cudaMemcpyAsync(T.nslot_map.ptr, T.slot_of.data(), sizeof(int) * T.slot_of.size(), cudaMemcpyHostToDevice, st));
  const long lines = (long)slots.size() * NT_PANELS * NT_NU * NT_NTH;
  T.nvals.ensure(sizeof(cplx) * (size_t)lines * NT_NF);
  NtBuildArgs A{};
  A.slot = tmp.slot.as<int4>(); A.k = h->d_k.as<double>(); A.kmax = T.kmax; A.L1 = L1;
  A.n_near = h->rule.n_near; A.Qh = h->rule.Q();
  A.kr_n = h->rule.kr.as<cplx>(); A.w_n = h->rule.w.as<cplx>();
  A.kz_n = h->rule.kz.as<cplx>(); A.sig_n = h->rule.sigma.as<cplx>();
  A.Nt = Nt; A.tail_off = tmp.toff.as<int>(); A.t_t = tmp.tt.as<double>(); A.w_t = tmp.tw.as<double>();
  A.kz_t = tmp.kz.as<cplx>(); A.sig_t = tmp.sig.as<cplx>();
  A.cheb = T.ncheb.as<double>();
  A.vals = T.nvals.as<cplx>();
  LAUNCH(k_ntab_build<<<(unsigned)lines, 128, 0, st>>>(A));
  FMM_CHECK(cudaGetLastError());
  FMM_CHECK(cudaStreamSynchronize(st));      // before the temporaries are freed
  T.bytes += sizeof(cplx) * (size_t)lines * NT_NF;
}

NearTabView near_table_view(const fmm_layered* h) {
  NearTabView v{};
  if (!h->tabs.built || !h->tabs.nvals.ptr) return v;
  v.vals = h->tabs.nvals.as<cplx>();
  v.slot_of = h->tabs.nslot_map.as<int>();
  v.cheb = h->tabs.ncheb.as<double>();
  v.kmax = h->tabs.kmax;
  return v;
}

// Contour quadrature rule and reaction densities (Sec. 3.1, Sec. 3.5).
//
// The Sommerfeld integrals are taken along the deformed contour of Sec. 3.5,
// Gamma1 (k_rho = -i s, 0 <= s <= b) and Gamma2 (k_rho = t - i b), with
// Gamma2 brought back to the real axis at t = ta = 1.5 max k + 1 by a vertical
// segment Gamma3; beyond ta every k_jz is positive imaginary, no singularity
// lies between the two paths, and the tail is integrated on the real axis in
// panels of fixed length (Gauss-Legendre on every piece).
//
// sigma^{ab}_{l l'}(k_rho) is obtained as Sec. 3.1 describes, by solving the
// linear system of the transmission conditions [u] = 0, [eps du/dz] = 0 at the
// L interfaces for the field A_j e^{ik_jz(z-d_j)} + B_j e^{ik_jz(d_{j-1}-z)}
// of every layer, for the two unit source waves of layer l' (arriving at its
// bottom interface, "dn", and at its top interface, "up"); then
//   sigma^{ab}_{l l'} = (k_lz / k_l'z) * (A_l if a = up else B_l)
//   for excitation dn (b = up) or up (b = down).
#include <cmath>
#include <vector>

#include "fmm_internal.h"

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = cos(FMM_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        p0 = 1.0; p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = z;
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void gauss_legendre_pub(int n, std::vector<double>& x, std::vector<double>& w) { gauss_legendre(n, x, w); }

int Rule::nodes_to(double tmax) const {
  if (tmax <= ta) return n_near;
  int np = (int)ceil((tmax - ta) / panel);
  if (np > n_tail_panels) np = n_tail_panels;
  return n_near + per_panel * np;
}

// One thread per (node, source layer): reaction densities at the node.
__global__ void k_sigma(int L1, const double* __restrict__ k, const double* __restrict__ d,
                        const double* __restrict__ eps, int Q, int q0,
                        const cplx* __restrict__ kr, cplx* __restrict__ kz_out,
                        cplx* __restrict__ sigma) {
  int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
  int lp = blockIdx.y;
  if (q >= Q) return;
  const int L = L1 - 1;
  cplx kz[FMM_MAXL], e[FMM_MAXL];
  for (int j = 0; j < L1; ++j) {
    kz[j] = kz_of(k[j], kr[q]);
    if (lp == 0) kz_out[j * Q + q] = kz[j];
  }
  for (int j = 0; j < L1; ++j) {
    e[j] = C(0, 0);
    if (j >= 1 && j <= L - 1) {
      cplx arg = cmul(C(0, 1), cscale(kz[j], d[j - 1] - d[j]));
      e[j] = cexp_(arg);
    }
  }
  const int n = 2 * L;
  // unknowns: A_0..A_{L-1} (index j), B_1..B_L (index L + j - 1)
  cplx M[2 * (FMM_MAXL - 1)][2 * (FMM_MAXL - 1) + 2];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n + 2; ++c) M[r][c] = C(0, 0);
  for (int j = 0; j < L; ++j) {
    int rc = 2 * j, rf = 2 * j + 1, up = j, lo = j + 1;
    cplx ik_up = cmul(C(0, eps[up]), kz[up]);
    cplx ik_lo = cmul(C(0, eps[lo]), kz[lo]);
    M[rc][up] = cadd(M[rc][up], C(1, 0));
    M[rf][up] = cadd(M[rf][up], ik_up);
    if (up >= 1) {
      M[rc][L + up - 1] = cadd(M[rc][L + up - 1], e[up]);
      M[rf][L + up - 1] = csub(M[rf][L + up - 1], cmul(ik_up, e[up]));
    }
    if (lo <= L - 1) {
      M[rc][lo] = csub(M[rc][lo], e[lo]);
      M[rf][lo] = csub(M[rf][lo], cmul(ik_lo, e[lo]));
    }
    M[rc][L + lo - 1] = csub(M[rc][L + lo - 1], C(1, 0));
    M[rf][L + lo - 1] = cadd(M[rf][L + lo - 1], ik_lo);
  }
  // right-hand sides: column n = excitation dn, column n+1 = excitation up
  cplx iks = cmul(C(0, eps[lp]), kz[lp]);
  if (lp <= L - 1) {
    M[2 * lp][n] = C(-1, 0);
    M[2 * lp + 1][n] = iks;
  }
  if (lp >= 1) {
    M[2 * (lp - 1)][n + 1] = C(1, 0);
    M[2 * (lp - 1) + 1][n + 1] = iks;
  }
  // Gaussian elimination with partial pivoting
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = cabs2(M[c][c]);
    for (int r = c + 1; r < n; ++r) {
      double v = cabs2(M[r][c]);
      if (v > best) { best = v; piv = r; }
    }
    if (piv != c)
      for (int cc = 0; cc < n + 2; ++cc) { cplx t = M[c][cc]; M[c][cc] = M[piv][cc]; M[piv][cc] = t; }
    cplx inv = cdiv(C(1, 0), M[c][c]);
    for (int r = c + 1; r < n; ++r) {
      cplx f = cmul(M[r][c], inv);
      if (f.x == 0.0 && f.y == 0.0) continue;
      for (int cc = c; cc < n + 2; ++cc) M[r][cc] = csub(M[r][cc], cmul(f, M[c][cc]));
    }
  }
  cplx X[2][2 * (FMM_MAXL - 1)];
  for (int rhs = 0; rhs < 2; ++rhs) {
    for (int r = n - 1; r >= 0; --r) {
      cplx s = M[r][n + rhs];
      for (int cc = r + 1; cc < n; ++cc) s = csub(s, cmul(M[r][cc], X[rhs][cc]));
      X[rhs][r] = cdiv(s, M[r][r]);
    }
  }
  for (int l = 0; l < L1; ++l) {
    cplx ratio = cdiv(kz[l], kz[lp]);
    for (int a = 0; a < 2; ++a) {
      for (int bb = 0; bb < 2; ++bb) {
        cplx val = C(0, 0);
        bool ok_a = (a == AR_UP) ? (l < L) : (l > 0);
        bool ok_b = (bb == AR_UP) ? (lp < L) : (lp > 0);
        if (ok_a && ok_b) {
          int rhs = (bb == AR_UP) ? 0 : 1;
          cplx Xv = (a == AR_UP) ? X[rhs][l] : X[rhs][L + l - 1];
          val = cmul(ratio, Xv);
        }
        sigma[((((size_t)l * L1 + lp) * 2 + a) * 2 + bb) * Q + q] = val;
      }
    }
  }
}

static void upload_nodes(fmm_layered* h, const std::vector<cplx>& kr, const std::vector<cplx>& w,
                         int q_from, cudaStream_t st) {
  Rule& R = h->rule;
  int Q = (int)kr.size();
  // (re)allocate and copy everything: the layout [L1][Q] depends on Q
  R.kr.ensure(sizeof(cplx) * Q);
  R.w.ensure(sizeof(cplx) * Q);
  R.kz.ensure(sizeof(cplx) * Q * h->L1);
  R.sigma.ensure(sizeof(cplx) * (size_t)Q * h->L1 * h->L1 * 4);
  FMM_CHECK(cudaMemcpyAsync(R.kr.ptr, kr.data(), sizeof(cplx) * Q, cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(R.w.ptr, w.data(), sizeof(cplx) * Q, cudaMemcpyHostToDevice, st));
  (void)q_from;
  if (h->L1 > 1) {
    dim3 grid((Q + 127) / 128, h->L1);
    LAUNCH(k_sigma<<<grid, 128, 0, st>>>(h->L1, h->d_k.as<double>(), h->d_d.as<double>(), h->d_eps.as<double>(),
                                  Q, 0, R.kr.as<cplx>(), R.kz.as<cplx>(), R.sigma.as<cplx>()));
  } else {
    // single layer: only k_z is needed
    dim3 grid((Q + 127) / 128, 1);
    LAUNCH(k_sigma<<<grid, 128, 0, st>>>(1, h->d_k.as<double>(), h->d_d.as<double>(), h->d_eps.as<double>(),
                                  Q, 0, R.kr.as<cplx>(), R.kz.as<cplx>(), R.sigma.as<cplx>()));
  }
  FMM_CHECK(cudaGetLastError());
}

// sigma and k_z at arbitrary contour nodes (kz [L1][Q], sigma [L1][L1][2][2][Q])
void launch_sigma_at(fmm_layered* h, int Q, const cplx* kr, cplx* kz, cplx* sigma, cudaStream_t st) {
  if (Q <= 0) return;
  dim3 grid((Q + 127) / 128, h->L1);
  LAUNCH(k_sigma<<<grid, 128, 0, st>>>(h->L1, h->d_k.as<double>(), h->d_d.as<double>(), h->d_eps.as<double>(), Q, 0,
                                       kr, kz, sigma));
  FMM_CHECK(cudaGetLastError());
}

static void build_nodes(fmm_layered* h, int n_panels, std::vector<cplx>& kr, std::vector<cplx>& w) {
  Rule& R = h->rule;
  std::vector<double> x12, w12, xt, wt;
  gauss_legendre(12, x12, w12);
  gauss_legendre(R.per_panel, xt, wt);
  kr.clear();
  w.clear();
  // Gamma1: k_rho = -i s, s in [0, b], two panels
  for (int pn = 0; pn < 2; ++pn) {
    double lo = R.b * pn / 2.0, hi = R.b * (pn + 1) / 2.0;
    for (int i = 0; i < 12; ++i) {
      double s = 0.5 * (lo + hi) + 0.5 * (hi - lo) * x12[i];
      kr.push_back(C(0.0, -s));
      w.push_back(C(0.0, -0.5 * (hi - lo) * w12[i]));      // dk = -i ds
    }
  }
  // Gamma2: k_rho = t - i b, t in [0, ta], panels of length <= b
  int n2 = (int)ceil(R.ta / R.b);
  for (int pn = 0; pn < n2; ++pn) {
    double lo = R.ta * pn / n2, hi = R.ta * (pn + 1) / n2;
    for (int i = 0; i < 12; ++i) {
      double t = 0.5 * (lo + hi) + 0.5 * (hi - lo) * x12[i];
      kr.push_back(C(t, -R.b));
      w.push_back(C(0.5 * (hi - lo) * w12[i], 0.0));
    }
  }
  // Gamma3: k_rho = ta - i s, s from b down to 0
  for (int i = 0; i < 12; ++i) {
    double s = 0.5 * R.b + 0.5 * R.b * x12[i];
    kr.push_back(C(R.ta, -s));
    w.push_back(C(0.0, 0.5 * R.b * w12[i]));              // dk = -i ds, s decreasing
  }
  R.n_near = (int)kr.size();
  for (int pn = 0; pn < n_panels; ++pn) {
    double lo = R.ta + R.panel * pn, hi = lo + R.panel;
    for (int i = 0; i < R.per_panel; ++i) {
      kr.push_back(C(0.5 * (lo + hi) + 0.5 * (hi - lo) * xt[i], 0.0));
      w.push_back(C(0.5 * (hi - lo) * wt[i], 0.0));
    }
  }
  R.n_tail_panels = n_panels;
}

void rule_init(fmm_layered* h) {
  Rule& R = h->rule;
  double kmax = 0;
  for (double v : h->k) kmax = fmax(kmax, v);
  R.b = 0.75;
  R.ta = 1.5 * kmax + 1.0;
  R.panel = 2.0;
  R.per_panel = 16;
  std::vector<cplx> kr, w;
  build_nodes(h, 40, kr, w);
  upload_nodes(h, kr, w, 0, 0);
  FMM_CHECK(cudaStreamSynchronize(0));
}

void rule_extend(fmm_layered* h, double tmax, cudaStream_t st) {
  Rule& R = h->rule;
  if (R.covers(tmax)) return;
  int need = (int)ceil((tmax - R.ta) / R.panel);
  need = need + need / 4 + 4;
  std::vector<cplx> kr, w;
  build_nodes(h, need, kr, w);
  // buffers may move: wait for users of the old ones
  FMM_CHECK(cudaStreamSynchronize(st));
  R.kr.release(); R.w.release(); R.kz.release(); R.sigma.release();
  upload_nodes(h, kr, w, 0, st);
}

// ---------------------------------------------------------------- rules of reaction M2L groups
// Copy the complex contour nodes of the handle's rule into a group's node
// block (kr, w, kz, sigma with the group's stride Qg).
__global__ void k_rule_near_copy(int L1, int n_near, int Qh, const cplx* __restrict__ kr, const cplx* __restrict__ w,
                                 const cplx* __restrict__ kz, const cplx* __restrict__ sigma, int Qg,
                                 cplx* __restrict__ gkr, cplx* __restrict__ gw, cplx* __restrict__ gkz,
                                 cplx* __restrict__ gsig) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_near) return;
  gkr[q] = kr[q];
  gw[q] = w[q];
  for (int j = 0; j < L1; ++j) gkz[(long)j * Qg + q] = kz[(long)j * Qh + q];
  for (int r = 0; r < L1 * L1 * 4; ++r) gsig[(long)r * Qg + q] = sigma[(long)r * Qh + q];
}

// Nodes for the reaction M2L classes of one group (vertical centre gap H,
// largest horizontal offset rho_max): the handle's complex contour up to ta,
// then the real tail to ta + (30 + 7p)/H -- the end the handle's rule would
// need -- in Gauss-Legendre panels whose length grows from min(2, Lmax) by
// 1.5x per panel to Lmax = 4 / max(rho_max, H), i.e. at most 4 radians of the
// Bessel factor's oscillation and a factor e^4 of the decay per panel.  The
// node count then stays near 1,500 as H shrinks, where fixed panels of length
// 2 need 8 (30 + 7p)/H nodes.  group_tail appends the tail nodes and weights
// (host); the group's block then holds n_near + that many nodes.
int group_tail(const fmm_layered* h, double H, double rho_max, std::vector<cplx>& kr, std::vector<cplx>& w) {
  const Rule& R = h->rule;
  std::vector<double> xg, wg;
  gauss_legendre(R.per_panel, xg, wg);
  const double tend = R.ta + (30.0 + 7.0 * h->p) / H;
  const double lmax = 4.0 / std::max(rho_max, H);
  double len = std::min(2.0, lmax), t = R.ta;
  int n = 0;
  while (t < tend) {
    for (int i = 0; i < R.per_panel; ++i) {
      kr.push_back(C(t + 0.5 * len * (xg[i] + 1.0), 0.0));
      w.push_back(C(0.5 * len * wg[i], 0.0));
      ++n;
    }
    t += len;
    len = std::min(1.5 * len, std::max(len, lmax));
  }
  return n;
}

// Complete a group's node block whose tail kr, w are in place: copy the
// handle's complex contour nodes in front and compute k_z and sigma at the
// tail nodes (k_sigma).
void group_rule_fill(fmm_layered* h, const RuleNodes& G, cudaStream_t st) {
  Rule& R = h->rule;
  const int L1 = h->L1, nn = G.n_near;
  cplx* gkr = const_cast<cplx*>(G.kr);
  cplx* gw = const_cast<cplx*>(G.w);
  cplx* gkz = const_cast<cplx*>(G.kz);
  cplx* gsig = const_cast<cplx*>(G.sigma);
  LAUNCH(k_rule_near_copy<<<(nn + 127) / 128, 128, 0, st>>>(L1, nn, R.Q(), R.kr.as<cplx>(), R.w.as<cplx>(),
                                                             R.kz.as<cplx>(), R.sigma.as<cplx>(), G.Q, gkr, gw, gkz,
                                                             gsig));
  if (G.Q > nn) {
    dim3 grid((unsigned)((G.Q - nn + 127) / 128), L1);
    LAUNCH(k_sigma<<<grid, 128, 0, st>>>(L1, h->d_k.as<double>(), h->d_d.as<double>(), h->d_eps.as<double>(), G.Q,
                                         nn, gkr, gkz, gsig));
  }
  FMM_CHECK(cudaGetLastError());
}

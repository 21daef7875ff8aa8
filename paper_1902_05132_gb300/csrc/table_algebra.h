// Host algebra of the tabulated reaction M2L (Sec. 3.5: eqs.
// identitypolyexp, asslegendreexpcoef, metoletableform): the power forms of
// the normalized Legendre functions, the index set of the S integrals and the
// sums that turn S values into operator entries.  Plain C++ (no CUDA types),
// so that a CPU test can compare it with the oracle's expansion.
#pragma once
#include <cmath>
#include <cstdlib>
#include <map>
#include <tuple>
#include <vector>

namespace tabalg {

constexpr double kPi = 3.14159265358979323846;

inline double sgn(int e) { return (e & 1) ? -1.0 : 1.0; }

// Coefficients of the power form of P^_n^m (m >= 0):
//   P^_n^m(x) = (1/x)^mu s^m sum_j beta[j] s^{2j},  s^2 = 1 - x^2.
// Rodrigues: P^_n^m = c_nm / (2^n n!) s^m d^{n+m}/dx^{n+m} (x^2 - 1)^n.
inline void legendre_power(int n, int m, int& mu, std::vector<double>& beta) {
  // (x^2 - 1)^n = sum_k C(n,k) (-1)^{n-k} x^{2k}
  std::vector<double> poly(2 * n + 1, 0.0);
  double binom = 1.0;
  for (int k = 0; k <= n; ++k) {
    poly[2 * k] = ((n - k) & 1) ? -binom : binom;
    binom = binom * (n - k) / (k + 1);
  }
  // differentiate n + m times
  const int D = n + m;
  std::vector<double> der(n - m + 1, 0.0);
  for (int j = D; j <= 2 * n; ++j) {
    double f = poly[j];
    for (int r = 0; r < D; ++r) f *= (double)(j - r);
    der[j - D] = f;
  }
  double lf = 0.0;                         // log of (n-m)!/(n+m)!
  for (int r = n - m + 1; r <= n + m; ++r) lf -= std::log((double)r);
  double scale = std::sqrt((2.0 * n + 1.0) / (4.0 * kPi) * std::exp(lf));
  for (int r = 1; r <= n; ++r) scale /= 2.0 * r;          // 2^n n!
  mu = (n - m) & 1;
  beta.assign(n + 2, 0.0);
  for (int j = 0; j <= n - m; ++j) {
    if ((j & 1) != mu || der[j] == 0.0) continue;
    // x^{2i'} -> (1 - s^2)^{i'};  x^{2i'+1} -> (1/x)(1 - s^2)^{i'+1}
    int i = (j - mu) / 2 + mu;
    double c = der[j] * scale, bb = 1.0;
    for (int e = 0; e <= i; ++e) {
      beta[e] += ((e & 1) ? -c : c) * bb;
      bb = bb * (i - e) / (e + 1);
    }
  }
  while (beta.size() > 1 && beta.back() == 0.0) beta.pop_back();
}

struct PowerForms {
  int p;
  std::vector<int> mu;                  // [n(n+1)/2 + m]
  std::vector<std::vector<double>> beta;
  explicit PowerForms(int p_) : p(p_) {
    for (int n = 0; n <= p; ++n)
      for (int m = 0; m <= n; ++m) {
        int u;
        std::vector<double> b;
        legendre_power(n, m, u, b);
        mu.push_back(u);
        beta.push_back(b);
      }
  }
  int at(int n, int am) const { return n * (n + 1) / 2 + am; }
};

// Table index of (q, t, mu, nu): tables sorted by (q, t, mu, nu) over the
// combinations an order-p operator reaches.
struct TabIndex {
  std::vector<int> key;                 // q, t, mu, nu per table
  std::map<std::tuple<int, int, int, int>, int> pos;
  void build(int p, const PowerForms& F) {
    std::map<std::tuple<int, int, int, int>, int> seen;
    const int P = (p + 1) * (p + 1);
    for (int i = 0; i < P; ++i) {
      int n = (int)std::floor(std::sqrt((double)i)), m = i - n * n - n;
      int fi = F.at(n, std::abs(m));
      for (int j = 0; j < P; ++j) {
        int n2 = (int)std::floor(std::sqrt((double)j)), m2 = j - n2 * n2 - n2;
        int fj = F.at(n2, std::abs(m2));
        int q = std::abs(m2 - m);
        int smax = (int)F.beta[fi].size() + (int)F.beta[fj].size() - 2;
        for (int s = 0; s <= smax; ++s)
          seen[std::make_tuple(q, std::abs(m) + std::abs(m2) + 2 * s, F.mu[fi], F.mu[fj])] = 0;
      }
    }
    key.clear();
    pos.clear();
    int x = 0;
    for (auto& kv : seen) {
      pos[kv.first] = x++;
      key.push_back(std::get<0>(kv.first));
      key.push_back(std::get<1>(kv.first));
      key.push_back(std::get<2>(kv.first));
      key.push_back(std::get<3>(kv.first));
    }
  }
  int size() const { return (int)key.size() / 4; }
};

// CSR of the sum of eq. metoletableform for one (l, l', a): for every entry
// (i, j) of the radial matrix, the tables and complex coefficients (A^s with
// the tau and J_{-q} signs, the arrow signs and i^{n+n'+1+m'-m}).
inline void build_terms(int p, const PowerForms& F, const TabIndex& X, double kl, double klp, int a,
                        std::vector<int>& off, std::vector<int>& tab, std::vector<double>& cre,
                        std::vector<double>& cim) {
  const int P = (p + 1) * (p + 1);
  off.assign((size_t)P * P + 1, 0);
  tab.clear();
  cre.clear();
  cim.clear();
  std::map<int, double> acc;
  for (int i = 0; i < P; ++i) {
    int n = (int)std::floor(std::sqrt((double)i)), m = i - n * n - n, am = std::abs(m);
    int fi = F.at(n, am);
    double tau = (m < 0 && (am & 1)) ? -1.0 : 1.0;
    double st = (a == 0) ? 1.0 : sgn(n + m);
    for (int j = 0; j < P; ++j) {
      int n2 = (int)std::floor(std::sqrt((double)j)), m2 = j - n2 * n2 - n2, am2 = std::abs(m2);
      int fj = F.at(n2, am2);
      double tau2 = (m2 < 0 && (am2 & 1)) ? -1.0 : 1.0;
      double ss = (a == 0) ? sgn(n2) : sgn(m2);
      int d = m2 - m, q = std::abs(d);
      double sq = (d < 0 && (q & 1)) ? -1.0 : 1.0;
      // i^e with e = n + n' + 1 + m' - m, times the signs
      const int e = ((n + n2 + 1 + d) % 4 + 4) % 4;
      const double f = st * ss * tau * tau2 * sq;
      const double ph_re = (e == 0) ? f : (e == 2) ? -f : 0.0;
      const double ph_im = (e == 1) ? f : (e == 3) ? -f : 0.0;
      acc.clear();
      const std::vector<double>& b1 = F.beta[fi];
      const std::vector<double>& b2 = F.beta[fj];
      for (size_t s1 = 0; s1 < b1.size(); ++s1) {
        if (b1[s1] == 0.0) continue;
        for (size_t s2 = 0; s2 < b2.size(); ++s2) {
          if (b2[s2] == 0.0) continue;
          int t = am + am2 + 2 * (int)(s1 + s2);
          double c = b1[s1] * b2[s2] / (std::pow(kl, am + 2.0 * s1) * std::pow(klp, am2 + 2.0 * s2));
          acc[t] += c;
        }
      }
      for (auto& kv : acc) {
        tab.push_back(X.pos.at(std::make_tuple(q, kv.first, F.mu[fi], F.mu[fj])));
        cre.push_back(ph_re * kv.second);
        cim.push_back(ph_im * kv.second);
      }
      off[(size_t)i * P + j + 1] = (int)tab.size();
    }
  }
}


}  // namespace tabalg

// Prints the host algebra of the tabulated reaction M2L (csrc/table_algebra.h)
// for one order, wave-number pair and target arrow, so that a CPU test can
// compare it with the oracle's independent expansion (oracle/tables.py):
//   line 1: ntab, then the (q, t, mu, nu) of every table
//   then one line per operator entry (i, j) with at least one term:
//   i j k tab_1 re_1 im_1 ... tab_k re_k im_k
// Usage: check_table_algebra p k_l k_l' a
#include <cstdio>
#include <cstdlib>

#include "table_algebra.h"

int main(int argc, char** argv) {
  if (argc != 5) return 2;
  const int p = std::atoi(argv[1]);
  const double kl = std::atof(argv[2]), klp = std::atof(argv[3]);
  const int a = std::atoi(argv[4]);
  tabalg::PowerForms F(p);
  tabalg::TabIndex X;
  X.build(p, F);
  std::vector<int> off, tab;
  std::vector<double> re, im;
  tabalg::build_terms(p, F, X, kl, klp, a, off, tab, re, im);
  std::printf("%d", X.size());
  for (int v : X.key) std::printf(" %d", v);
  std::printf("\n");
  const int P = (p + 1) * (p + 1);
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) {
      const int e = i * P + j, k = off[e + 1] - off[e];
      if (!k) continue;
      std::printf("%d %d %d", i, j, k);
      for (int x = off[e]; x < off[e + 1]; ++x) std::printf(" %d %.17g %.17g", tab[x], re[x], im[x]);
      std::printf("\n");
    }
  return 0;
}

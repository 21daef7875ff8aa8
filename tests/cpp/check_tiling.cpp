// Checks the shared-memory tiling rules of the M2L and shift kernels for
// every expansion order: each CTA's blocks fit the shared memory its launch
// asks for, launches stay within the per-CTA limit, and the thread layout
// stays within 128 threads.  Prints "ok" or the first violations.
#include <cstdio>

#include "tiling.h"

using namespace tiling;

static int bad = 0;
static void fail(const char* what, int p, long a, long b) {
  if (bad++ < 20) std::printf("p=%d %s: %ld vs %ld\n", p, what, a, b);
}

int main() {
  for (int p = 1; p <= 16; ++p) {
    const int P = (p + 1) * (p + 1), np = (p + 1) * (p + 2) / 2, nm = p * (p + 1) / 2;
    // FP64 GEMM: one launch for free-space blocks (R = P), one for reaction blocks (np, nm)
    const size_t launch_free = gemm_smem_max(P);
    const size_t launch_reac = std::max(gemm_smem_max(np), nm ? gemm_smem_max(nm) : (size_t)0);
    for (int R : {P, np, nm}) {
      if (!R) continue;
      const size_t launch = (R == P) ? launch_free : launch_reac;
      if (launch > kSmemPerCta) fail("gemm launch smem", p, (long)launch, (long)kSmemPerCta);
      int RB, CB;
      gemm_tiles(R, RB, CB);
      if (CB < 1 || CB > R) fail("gemm contraction chunk", p, CB, R);
      int rows = 0;
      for (int r0 = 0; r0 < R; r0 += RB) {
        const int rb = std::min(RB, R - r0), tk = gemm_tk(rb, CB), tr = gemm_threads_per_col(rb);
        rows += rb;
        if (tk < 1 || tr * tk > 128) fail("gemm threads", p, tr * tk, 128);
        if (kRpt * tr < rb) fail("gemm rows per thread", p, kRpt * tr, rb);
        if (gemm_smem(rb, CB, tk) > launch) fail("gemm block smem", p, (long)gemm_smem(rb, CB, tk), (long)launch);
      }
      if (rows != R) fail("gemm rows covered", p, rows, R);
    }
    // tensor-core product: operator sub-blocks of <= 128 rows, N_pad = 2 x (rows rounded to 16)
    for (int R : {P, np}) {
      const int rb = std::min(R, 128), npad = 2 * ((rb + 15) / 16 * 16);
      if (npad > 256 || npad % 16) fail("tc N_pad", p, npad, 256);
      const int nst = tc_stages(npad);
      const size_t smem = tc_smem(npad);
      if (smem > kSmemPerCta) fail("tc smem", p, (long)smem, (long)kSmemPerCta);
      if (nst == 1 && 2 * (smem + 1024) > kSmemPerSm) fail("tc one stage without two CTAs", p, (long)smem, 0);
    }
    // rotation form
    if (rot_kc(p) < 1 || rot_kc(p) > 32) fail("rot column tile", p, rot_kc(p), 32);
    if (rot_smem(p) > kSmemPerCta) fail("rot smem", p, (long)rot_smem(p), (long)kSmemPerCta);
    {
      int kc[16], thr[16];
      int nc = rot_tune_candidates(p, kc, thr, 16);
      if (nc < 1) fail("rot autotune candidates", p, nc, 1);
      for (int i = 0; i < nc; ++i)
        if (rot_smem_kc(p, kc[i]) > kSmemPerCta) fail("rot candidate smem", p, (long)rot_smem_kc(p, kc[i]), (long)kSmemPerCta);
    }
    if (shift_smem(p) > kSmemPerCta) fail("shift smem", p, (long)shift_smem(p), (long)kSmemPerCta);
    long nw = 0, naz = 0;
    for (int n = 0; n <= p; ++n) nw += (2 * n + 1) * (2 * n + 1);
    for (int m = -p; m <= p; ++m) naz += (p + 1 - std::abs(m)) * (p + 1 - std::abs(m));
    if (nw != rot_nw(p) || naz != rot_naz(p)) fail("rotation block sizes", p, nw, rot_nw(p));
  }
  std::printf(bad ? "violations: %d\n" : "ok\n", bad);
  return bad ? 1 : 0;
}

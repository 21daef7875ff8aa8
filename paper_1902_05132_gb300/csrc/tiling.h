// Host-side tiling rules of the M2L and shift kernels: how much shared
// memory a CTA asks for and how the work is cut so that every block fits.
// Plain C++ (no CUDA types), so that the same rules can be checked by a CPU
// test for every expansion order.
#pragma once
#include <algorithm>
#include <cstddef>

#ifdef __CUDACC__
#define TILING_HD __host__ __device__
#else
#define TILING_HD
#endif

namespace tiling {

constexpr size_t kCplx = 16;                 // bytes of one complex double
constexpr size_t kSmemPerSm = 228 * 1024;    // shared memory of an SM (1 KB of it reserved per CTA)
constexpr size_t kSmemPerCta = 227 * 1024;   // largest dynamic allocation of one CTA

// ---- FP64 class-batched GEMM (k_zgemm_res): thread (tr, tk) owns kRpt rows
// and kKb columns; a CTA holds RB operator rows of a CB-wide contraction
// chunk plus TK * kKb input columns of that chunk.
constexpr int kRpt = 3, kKb = 4;
constexpr size_t kGemmSmemCap = 200 * 1024;

inline size_t gemm_smem(int RB, int CB, int TK) { return kCplx * ((size_t)RB * CB + (size_t)TK * kKb * CB); }
inline int gemm_threads_per_col(int RB) { return (RB + kRpt - 1) / kRpt; }
// thread columns of a block of RB rows: as many as 128 threads allow, fewer
// if the input tile would not fit beside the operator block
inline int gemm_tk(int RB, int CB) {
  int TK = 128 / gemm_threads_per_col(RB);
  while (TK > 1 && gemm_smem(RB, CB, TK) > kGemmSmemCap) --TK;
  return TK;
}
// tile of an R x R operator: the whole operator resident if it fits, else row
// blocks of it (each resident), else 96-row blocks streamed in chunks of the
// contraction; every block, the ragged last one included, fits
inline void gemm_tiles(int R, int& RB, int& CB) {
  auto full_tk = [](int rb) { return 128 / gemm_threads_per_col(rb); };
  RB = std::min(R, 3 * 128);
  CB = R;
  while (RB > 3 && gemm_smem(RB, CB, full_tk(RB)) > kGemmSmemCap) RB -= 3;
  if (gemm_smem(RB, CB, full_tk(RB)) <= kGemmSmemCap) return;
  RB = std::min(R, 96);
  CB = (int)(kGemmSmemCap / gemm_smem(RB, 1, full_tk(RB)));
}
// largest shared memory of any block of an R x R operator
inline size_t gemm_smem_max(int R) {
  int RB, CB;
  gemm_tiles(R, RB, CB);
  size_t m = 0;
  for (int r0 = 0; r0 < R; r0 += RB) {
    int rb = std::min(RB, R - r0);
    m = std::max(m, gemm_smem(rb, CB, gemm_tk(rb, CB)));
  }
  return m;
}

// ---- tensor-core M2L (k_m2l_tc): tiles of 128 pairs, 64-entry contraction
// chunks of 128-byte rows, operator blocks of N_pad rows
constexpr size_t kTcTileM = 128, kTcRowBytes = 128;
inline size_t tc_stage_bytes(int max_npad) { return 2 * kTcTileM * kTcRowBytes + 2 * (size_t)max_npad * kTcRowBytes; }
// two pipeline stages when two CTAs still fit on an SM; otherwise one stage,
// so that two CTAs share the SM
inline int tc_stages(int max_npad) {
  const size_t stage = tc_stage_bytes(max_npad);
  return (2 * (2 * stage + 2048) <= kSmemPerSm) ? 2 : ((2 * (stage + 2048) <= kSmemPerSm) ? 1 : 2);
}
inline size_t tc_smem(int max_npad) { return 1024 + tc_stages(max_npad) * tc_stage_bytes(max_npad); }

// ---- rotation form (k_zrot, k_m2m_rot, k_l2l_rot)
TILING_HD inline long rot_nw(int p) { return (long)(p + 1) * (2 * p + 1) * (2 * p + 3) / 3; }   // sum (2n+1)^2
TILING_HD inline int rot_naz(int p) { return (p + 1) * (2 * (p + 1) * (p + 1) + 1) / 3; }        // sum (p+1-|m|)^2
inline size_t rot_fixed_bytes(int p) { return kCplx * ((size_t)rot_nw(p) + rot_naz(p)); }
// column tile of k_zrot: up to 32 columns within ~110 KB (two CTAs per SM)
// when at least 8 columns fit there, else within 200 KB
inline int rot_kc(int p) {
  const size_t P = (size_t)(p + 1) * (p + 1), fixed = rot_fixed_bytes(p), col = 2 * kCplx * P;
  int KC = (int)std::min<size_t>(32, (110 * 1024 - std::min<size_t>(fixed, 110 * 1024)) / col);
  if (KC < 8) KC = (int)std::min<size_t>(32, (200 * 1024 - std::min<size_t>(fixed, 200 * 1024)) / col);
  return std::max(KC, 1);
}
inline size_t rot_smem_kc(int p, int kc) { return rot_fixed_bytes(p) + 2 * kCplx * (size_t)kc * (p + 1) * (p + 1); }
inline size_t rot_smem(int p) { return rot_smem_kc(p, rot_kc(p)); }
// candidates the autotuner of k_zrot times: column tiles that fit one CTA
// (kc in {4, 8, 16, 24, 32} and the fixed rule's rot_kc) with 128 or 256
// threads
inline int rot_tune_candidates(int p, int* kc, int* thr, int max_n) {
  int kcs[6] = {4, 8, 16, 24, 32, rot_kc(p)};
  const int nk = (kcs[5] == 4 || kcs[5] == 8 || kcs[5] == 16 || kcs[5] == 24 || kcs[5] == 32) ? 5 : 6;
  int n = 0;
  for (int a = 0; a < nk; ++a)
    for (int t = 128; t <= 256; t += 128)
      if (rot_smem_kc(p, kcs[a]) <= kSmemPerCta && n < max_n) { kc[n] = kcs[a]; thr[n] = t; ++n; }
  return n;
}
inline size_t shift_smem(int p) { return rot_fixed_bytes(p) + 3 * kCplx * (size_t)(p + 1) * (p + 1); }

}  // namespace tiling

// Mixed-precision M2L on the fifth-generation tensor cores (tcgen05).
//
// The translations of one operator class are one product Z = A Y (Sec. 3.3:
// every V-list pair of a class uses the same separation matrix; for reaction
// classes the m-reflection split blocks).  Here that product runs as a real
// FP16 x FP16 -> FP32 tensor-core GEMM:
//
//  * complex -> real: with Y = Yr + i Yi and A = Ar + i Ai,
//        [Re Z; Im Z] = [Ar -Ai; Ai Ar] [Yr; Yi];
//  * scaling: a degree-n coefficient of a box of width w is of the order of
//    s_n = (k rho)^n / (2n+1)!!, rho = (sqrt 3 / 2) w (the bound |j_n(x)| <=
//    x^n/(2n+1)!! on the expansion of eq. melecoeffree).  Inputs are divided
//    by 2^{E_in(n')}, outputs multiplied by 2^{E_out(n)} (E = floor log2 s_n),
//    so both sides are O(1) and the operator entries A 2^{E_out + E_in} are
//    bounded by the convergence of the expansion; each operator is then
//    shifted by a power of two to fill the FP16 range, and each gathered
//    column by the power of two of its largest entry;
//  * split precision: x = hi + lo with hi = fp16(x), lo = fp16(x - hi); the
//    product takes hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32
//    rounding) accumulated in FP32 in tensor memory.
// Every scale is a power of two, so undoing it is exact; the result is
// written as FP64 translated columns for the same deterministic reduction as
// the FP64 path.
//
// Layout (GEMM "TN", both operands K-major, 128-byte swizzle): the tile of
// 128 pairs (MMA M) by the contraction (MMA K) is operand A; the operator
// rows (MMA N = 2 x 16-rounded output rows) are operand B.  Global copies are
// stored already swizzled in chunks of 64 contraction entries, so one bulk
// copy per chunk lands each operand in shared memory in the form the tensor
// core reads.  Chunks go through a one- or two-stage pipeline fed by
// cp.async.bulk and mbarriers (one stage when that lets two CTAs share an SM,
// so that one CTA's epilogue overlaps the other's copies and products); every
// wait is bounded.
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <vector>

#include "async_copy.cuh"
#include "fmm_internal.h"
#include "tiling.h"

namespace {

constexpr int kTileM = 128;              // pairs per tile (MMA M)
constexpr int kChunk = 64;               // contraction entries per 128-byte row
constexpr uint32_t kRowBytes = 128;      // one swizzled row of a chunk

__device__ inline void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ inline void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D (tensor memory) = A B^T (+ D if acc), A and B from shared memory descriptors
__device__ inline void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on the mbarrier once all tcgen05 operations issued so far by this thread are done
__device__ inline void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of the calling warp's 32 lanes
__device__ inline void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// atoms of 1024 bytes stacked along M/N.
__device__ inline uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused with this swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset between 8-row atoms
  d |= (uint64_t)1 << 46;                           // descriptor version of this architecture
  d |= (uint64_t)2 << 61;                           // swizzle: 128 bytes
  return d;
}
// Instruction descriptor of kind::f16: FP16 A and B, FP32 accumulator, both K-major.
__host__ __device__ inline uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of contraction entry kk (0..63) of row `row` inside a swizzled chunk.
__host__ __device__ inline uint32_t swz_unit(int row, int unit) {
  return (uint32_t)row * kRowBytes + (uint32_t)((unit ^ (row & 7)) * 16);
}

// degree of index i of a coefficient block: 0 full (n*n + n + m), 1 plus, 2 minus basis
__device__ inline int deg_of(int basis, int i) {
  int n;
  if (basis == 0) {
    n = (int)sqrtf((float)i);
    while ((n + 1) * (n + 1) <= i) ++n;
    while (n * n > i) --n;
  } else if (basis == 1) {
    n = 0;
    while ((n + 1) * (n + 2) / 2 <= i) ++n;
  } else {
    n = 1;
    while (n * (n + 1) / 2 <= i) ++n;
  }
  return n;
}

__device__ inline void split_half(double v, __half& hi, __half& lo) {
  hi = __float2half_rn((float)v);
  lo = __float2half_rn((float)(v - (double)__half2float(hi)));
}
// Same split from an FP32 value (x - hi is exact in FP32): no FP64 arithmetic.
__device__ inline void split_half_f(float x, __half& hi, __half& lo) {
  hi = __float2half_rn(x);
  lo = __float2half_rn(x - __half2float(hi));
}
// x * 2^e rounded to FP32 (to nearest, ties to even), from the bit pattern
// with integer arithmetic only.  Results below the FP32 normal range give a
// signed 0: the callers scale each column so that its largest entry is near
// 1, and such entries are then below 2^-126 of it.
__device__ inline float d2f_scaled(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  if (ex == 0) return __uint_as_float(sign);
  if (ex == 0x7FF) return (float)x;
  int fe = ex - 1023 + e + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7F800000u);
  uint32_t m23 = (uint32_t)((u & 0xFFFFFFFFFFFFFULL) >> 29);
  const uint32_t rem = (uint32_t)(u & 0x1FFFFFFFULL);
  if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) {
    if (++m23 == 0x800000u) {
      m23 = 0;
      if (++fe >= 255) return __uint_as_float(sign | 0x7F800000u);
    }
  }
  return __uint_as_float(sign | ((uint32_t)fe << 23) | m23);
}
// unbiased binary exponent of x (x != 0, normal): x in [2^E, 2^{E+1})
__device__ inline int dexp_of(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF) - 1023;
}

// f * 2^e as a double, built from the bit pattern with integer arithmetic only
// (exact; FP32 zeros and subnormals -- below 2^-126 of the O(1) scaled
// accumulators -- give 0).
__device__ inline double f32_scaled_to_f64(float f, int e) {
  const uint32_t u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 0xFFu);
  if (ex == 0) return 0.0;
  const int dex = ex - 127 + 1023 + e;
  if (ex == 255 || dex <= 0 || dex >= 2047) return ldexp((double)f, e);
  const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)dex << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

__device__ inline double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double m = 0.0;
  for (int i = 0; i < nw; ++i) m = fmax(m, red[i]);
  return m;
}

}  // namespace

// One operator sub-block (output rows r0 .. r0 + RB of an R_full x C block).
struct TcOpJob {
  long src_off;      // FP64 operator, input-major: entry (out r, in c) at src_off + c * R_full + r
  long dst_off;      // bytes: [hi/lo][Kc][N_pad rows][128 B]
  long scale_off;    // ints: output exponent shift - E_out(n(r)), r < RB
  int R_full, C, r0, RB, R16, N_pad, Kc, basis;
  int etab_off;      // exponents E_in[n], E_out[n] of the class's (component, level)
};

// Scaled, split, swizzled FP16 copy of an operator sub-block (one CTA each).
__global__ void __launch_bounds__(256) k_tc_prep_ops(const TcOpJob* __restrict__ jobs, const cplx* __restrict__ ops,
                                                     unsigned char* __restrict__ dst, int* __restrict__ rexp,
                                                     const int* __restrict__ etab) {
  const TcOpJob jb = jobs[blockIdx.x];
  __shared__ int Eout[128];
  __shared__ int Ein[FMM_MAXP * FMM_MAXP + 2 * FMM_MAXP + 1];
  __shared__ double red[8];
  const int* Et = etab + jb.etab_off;           // [E_in(0..MAXP) | E_out(0..MAXP)]
  for (int r = threadIdx.x; r < jb.RB; r += blockDim.x) Eout[r] = Et[FMM_MAXP + 1 + deg_of(jb.basis, jb.r0 + r)];
  for (int c = threadIdx.x; c < jb.C; c += blockDim.x) Ein[c] = Et[deg_of(jb.basis, c)];
  __syncthreads();
  const cplx* A = ops + jb.src_off;
  double mx = 0.0;
  for (long e = threadIdx.x; e < (long)jb.RB * jb.C; e += blockDim.x) {
    int r = (int)(e % jb.RB), c = (int)(e / jb.RB);
    cplx a = A[(long)c * jb.R_full + jb.r0 + r];
    mx = fmax(mx, ldexp(fmax(fabs(a.x), fabs(a.y)), Eout[r] + Ein[c]));
  }
  mx = block_max(mx, red);
  int shift = 0;
  if (mx > 0.0) {
    int e;
    frexp(mx, &e);
    shift = e - 15;               // scaled entries below 2^15
  }
  const int units = jb.Kc * (kChunk / 8);
  const long half_bytes = (long)jb.Kc * jb.N_pad * kRowBytes;
  unsigned char* D = dst + jb.dst_off;
  for (long e = threadIdx.x; e < (long)jb.N_pad * units; e += blockDim.x) {
    int jo = (int)(e / units), u = (int)(e % units);
    int chunk = u / 8, uu = u % 8;
    bool re_out = jo < jb.RB, im_out = jo >= jb.R16 && jo < jb.R16 + jb.RB;
    int r = re_out ? jo : jo - jb.R16;
    __align__(16) __half hv[8], lv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      int ji = chunk * kChunk + uu * 8 + t;
      double v = 0.0;
      if ((re_out || im_out) && ji < 2 * jb.C) {
        bool re_in = ji < jb.C;
        int c = re_in ? ji : ji - jb.C;
        cplx a = A[(long)c * jb.R_full + jb.r0 + r];
        double s = re_out ? (re_in ? a.x : -a.y) : (re_in ? a.y : a.x);
        v = ldexp(s, Eout[r] + Ein[c] - shift);
      }
      split_half(v, hv[t], lv[t]);
    }
    long off = (long)chunk * jb.N_pad * kRowBytes + swz_unit(jo, uu);
    *(uint4*)(D + off) = *(const uint4*)hv;
    *(uint4*)(D + half_bytes + off) = *(const uint4*)lv;
  }
  for (int r = threadIdx.x; r < jb.RB; r += blockDim.x) rexp[jb.scale_off + r] = shift - Eout[r];
}

// One contraction part of a run (class): free operator, or the plus / minus
// block of a reaction operator.
struct TcPart {
  long a_off;        // bytes of tile 0: tiles of [hi/lo][Kc][128 rows][128 B]
  long sig_off;      // ints: column exponent e_k per tile row
  int C, in_off, Kc, basis;
};

// Column of sorted pair k, scaled and split into the A tiles of each part of
// its run.  FP64 appears only in the loads: the degree and column scales are
// applied to the exponent bits while rounding to FP32, and the rotation and
// the symmetric-basis combination (reaction) run in FP32.
__global__ void __launch_bounds__(64) k_tc_gather(long nv, int p, const int* __restrict__ perm,
                                                  const int* __restrict__ owner, const int* __restrict__ vidx,
                                                  BoxGeom B, OpIndex OI, const cplx* __restrict__ M,
                                                  const int* __restrict__ run_start, int nruns,
                                                  const int* __restrict__ run_part, const TcPart* __restrict__ parts,
                                                  const int* __restrict__ etab, const float2* __restrict__ phase_f,
                                                  unsigned char* __restrict__ Abuf, int* __restrict__ isig) {
  const int P = (p + 1) * (p + 1);
  long k = blockIdx.x;
  if (k >= nv) return;
  // run of k: run_start[r] <= k < run_start[r + 1]
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (run_start[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  const int run = lo;
  const int m = (int)(k - run_start[run]);
  const int K = run_start[run + 1] - run_start[run];
  int e = perm[k];
  int T = owner[e], S = vidx[e];
  int comp = B.comp[T], lev = B.lev[T];
  const CompGeom& cg = OI.cgs[comp];
  extern __shared__ float2 xf[];              // [2 P]: scaled column, then its rotated symmetric form
  __shared__ int red[2];
  __shared__ int Ein[FMM_MAXP + 1];
  float2* yf = xf + P;
  const cplx* Ms = M + (long)S * P;
  const int* Et = etab + ((long)comp * 23 + lev) * 2 * (FMM_MAXP + 1);
  for (int n = threadIdx.x; n <= p; n += blockDim.x) Ein[n] = Et[n];
  __syncthreads();
  // column exponent: largest binary exponent of the degree-scaled entries
  int emax = -1 << 20;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    cplx x = Ms[i];
    int en = Ein[deg_of(0, i)];
    if (x.x != 0.0) emax = max(emax, dexp_of(x.x) - en);
    if (x.y != 0.0) emax = max(emax, dexp_of(x.y) - en);
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = emax;
  __syncthreads();
  emax = max(red[0], red[1]);
  const int ek = (emax > -(1 << 19)) ? emax + 1 : 0;      // entries below 1 after the column scale
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    cplx x = Ms[i];
    int sh = -Ein[deg_of(0, i)] - ek;
    xf[i] = make_float2(d2f_scaled(x.x, sh), d2f_scaled(x.y, sh));
  }
  __syncthreads();
  const float2* src = xf;
  if (cg.kind != CK_FREE) {
    const int* ct = B.coord + 3 * T;
    const int* cs = B.coord + 3 * S;
    const float2* ph = phase_f + ((ct[1] - cs[1] + 3) * 7 + (ct[0] - cs[0] + 3)) * (2 * p + 1) + p;
    const int np = (p + 1) * (p + 2) / 2;
    const float rr = 0.70710678118654752440f;
    for (int a = threadIdx.x; a < P; a += blockDim.x) {
      bool plus = a < np;
      int n = deg_of(plus ? 1 : 2, plus ? a : a - np);
      int mm = plus ? a - n * (n + 1) / 2 : a - np - n * (n - 1) / 2 + 1;
      float2 u;
      float2 x0 = xf[n * n + n + mm], p0 = ph[mm];
      float2 r0 = make_float2(x0.x * p0.x - x0.y * p0.y, x0.x * p0.y + x0.y * p0.x);
      if (mm == 0) {
        u = r0;
      } else {
        float2 x1 = xf[n * n + n - mm], p1 = ph[-mm];
        float s = (mm & 1) ? -1.0f : 1.0f;
        float2 r1 = make_float2(s * (x1.x * p1.x - x1.y * p1.y), s * (x1.x * p1.y + x1.y * p1.x));
        u = plus ? make_float2((r0.x + r1.x) * rr, (r0.y + r1.y) * rr)
                 : make_float2((r0.x - r1.x) * rr, (r0.y - r1.y) * rr);
      }
      yf[a] = u;
    }
    __syncthreads();
    src = yf;
  }
  for (int q = 0; q < 2; ++q) {
    int pi = run_part[2 * run + q];
    if (pi < 0) continue;
    const TcPart pt = parts[pi];
    const int units = pt.Kc * (kChunk / 8);
    const long tile_bytes = 2L * pt.Kc * kTileM * kRowBytes, half_bytes = (long)pt.Kc * kTileM * kRowBytes;
    const int tile = m / kTileM, row = m % kTileM;
    unsigned char* Tb = Abuf + pt.a_off + tile * tile_bytes;
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      int chunk = u / 8, uu = u % 8;
      __align__(16) __half hv[8], lv[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        int ji = chunk * kChunk + uu * 8 + t;
        float v = 0.0f;
        if (ji < 2 * pt.C) {
          bool re = ji < pt.C;
          float2 y = src[pt.in_off + (re ? ji : ji - pt.C)];
          v = re ? y.x : y.y;
        }
        split_half_f(v, hv[t], lv[t]);
      }
      long off = (long)chunk * kTileM * kRowBytes + swz_unit(row, uu);
      *(uint4*)(Tb + off) = *(const uint4*)hv;
      *(uint4*)(Tb + half_bytes + off) = *(const uint4*)lv;
    }
    if (threadIdx.x == 0) isig[pt.sig_off + m] = ek;
    // the last pair of the run clears the unused rows of its last tile
    if (m == K - 1) {
      const int pad = kTileM - 1 - row;
      for (long f = threadIdx.x; f < (long)pad * units; f += blockDim.x) {
        int rr2 = row + 1 + (int)(f / units), u = (int)(f % units);
        long off = (long)(u / 8) * kTileM * kRowBytes + swz_unit(rr2, u % 8);
        *(uint4*)(Tb + off) = make_uint4(0, 0, 0, 0);
        *(uint4*)(Tb + half_bytes + off) = make_uint4(0, 0, 0, 0);
      }
      for (int f = threadIdx.x; f < pad; f += blockDim.x) isig[pt.sig_off + m + 1 + f] = 0;
    }
  }
}

__global__ void k_tc_phase_f32(int n, const cplx* __restrict__ ph, float2* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)ph[i].x, (float)ph[i].y);
}

// One tile of 128 pairs times one operator sub-block.
struct TcItem {
  long a_off;        // bytes: this tile's [hi/lo][Kc][128][128 B]
  long b_off;        // bytes: operator sub-block [hi/lo][Kc][N_pad][128 B]
  long scale_off;    // output exponents of the sub-block's rows
  long sig_off;      // isig of this tile's rows
  long z_row0;       // translated-column index (sorted pair) of tile row 0
  int rows;          // valid rows of the tile
  int RB, R16, N_pad, Kc;
  int z_col0;        // first coefficient written: part offset + sub-block row r0
};

// D[128 x N_pad] = A_tile (128 x 64 Kc) * B^T in tensor memory, then Z.
__global__ void __launch_bounds__(128) k_m2l_tc(const TcItem* __restrict__ items, const unsigned char* __restrict__ Abuf,
                                               const unsigned char* __restrict__ Bbuf,
                                               const int* __restrict__ rexp, const int* __restrict__ isig,
                                               cplx* __restrict__ Z, int P, int* __restrict__ err,
                                               uint32_t extra_tx, int nst) {
  const TcItem it = items[blockIdx.x];
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t bars[5];     // full[2], empty[2], done
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = kTileM * kRowBytes;
  const uint32_t b_bytes = (uint32_t)it.N_pad * kRowBytes;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(smem_u32(&bars[i]), 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(&tmem_sh), 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;

  if (threadIdx.x == 0) {
    const uint32_t idesc = idesc_f16(kTileM, it.N_pad);
    const unsigned char* Ag = Abuf + it.a_off;
    const unsigned char* Bg = Bbuf + it.b_off;
    int issued[2] = {0, 0}, landed[2] = {0, 0};
    auto issue = [&](int c, int s) {
      uint32_t base = smem_u32(sm + s * stage_bytes);
      uint32_t bar = smem_u32(&bars[s]);
      mbar_expect_tx(bar, stage_bytes + extra_tx);      // extra_tx: 0 except in the wait-expiry test
      bulk_g2s(base, Ag + (size_t)c * a_bytes, a_bytes, bar);
      bulk_g2s(base + a_bytes, Ag + (size_t)(it.Kc + c) * a_bytes, a_bytes, bar);
      bulk_g2s(base + 2 * a_bytes, Bg + (size_t)c * b_bytes, b_bytes, bar);
      bulk_g2s(base + 2 * a_bytes + b_bytes, Bg + (size_t)(it.Kc + c) * b_bytes, b_bytes, bar);
      ++issued[s];
    };
    bool ok = true;
    // nst (1 or 2) pipeline stages: chunk c goes through stage c % nst
    issue(0, 0);
    if (nst > 1 && it.Kc > 1) issue(1, 1);
    for (int c = 0; c < it.Kc; ++c) {
      const int s = c % nst;
      const uint32_t ph = (uint32_t)(c / nst) & 1u;
      if (!mbar_wait(smem_u32(&bars[s]), ph)) { ok = false; break; }
      ++landed[s];
      tc_fence_after();
      const uint32_t base = smem_u32(sm + s * stage_bytes);
#pragma unroll
      for (int t = 0; t < kChunk / 16; ++t) {      // K = 16 per MMA: 32 bytes along the swizzled row
        const uint64_t ah = sw128_desc(base + t * 32), al = sw128_desc(base + a_bytes + t * 32);
        const uint64_t bh = sw128_desc(base + 2 * a_bytes + t * 32);
        const uint64_t bl = sw128_desc(base + 2 * a_bytes + b_bytes + t * 32);
        umma_f16(tmem, ah, bh, idesc, (c > 0 || t > 0) ? 1u : 0u);
        umma_f16(tmem, ah, bl, idesc, 1u);
        umma_f16(tmem, al, bh, idesc, 1u);
      }
      umma_commit(smem_u32(&bars[2 + s]));
      if (c + nst < it.Kc) {
        if (!mbar_wait(smem_u32(&bars[2 + s]), ph)) { ok = false; break; }
        issue(c + nst, s);
      }
    }
    umma_commit(smem_u32(&bars[4]));
    if (!ok) {
      abort_sh = 1;
      atomicOr(err, 16);
      // copies still in flight land before the CTA leaves
      for (int s = 0; s < 2; ++s)
        while (landed[s] < issued[s]) {
          if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)landed[s] & 1u)) break;
          ++landed[s];
        }
    }
  }
  if (!mbar_wait(smem_u32(&bars[4]), 0)) {
    atomicOr(&abort_sh, 1);
    atomicOr(err, 16);
  }
  __syncthreads();
  tc_fence_after();
  if (!abort_sh) {
    const int m = warp * 32 + lane;               // tile row = tensor-memory lane
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const int ek = (m < it.rows) ? isig[it.sig_off + m] : 0;
    cplx* zr = Z + (it.z_row0 + m) * (long)P + it.z_col0;
    for (int r0 = 0; r0 < it.R16; r0 += 16) {
      float re[16], im[16];
      tmem_ld16(tl + (uint32_t)r0, re);
      tmem_ld16(tl + (uint32_t)(it.R16 + r0), im);
      if (m < it.rows) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          int r = r0 + j;
          if (r < it.RB) {
            const int e = rexp[it.scale_off + r] + ek;
            zr[r] = C(f32_scaled_to_f64(re[j], e), f32_scaled_to_f64(im[j], e));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// ---------------------------------------------------------------- host driver
// floor(log2 s_n), s_n = (k rho)^n / (2n+1)!!, rho = (sqrt 3 / 2) w: the
// degree scale of the coefficients of a box of width w (see the header).
static int deg_exp(double k, double w, int n) {
  double x = k * 0.86602540378443864676 * w;
  double s = 1.0;
  for (int j = 1; j <= n; ++j) s *= x / (2.0 * j + 1.0);
  int e;
  frexp(s, &e);
  return e - 1;
}

void launch_tc_run_info(int nruns, const int* rs, const int* perm, const int* owner, BoxGeom B, int* info,
                        cudaStream_t st);

// Z for the sorted V pairs: runs are (operator key, count) in sorted order.
void run_m2l_tc(fmm_layered* h, long nv, int nruns, const std::vector<unsigned long long>& hk,
                const std::vector<int>& hc, const int* perm, const int* owner, const int* vidx, BoxGeom B,
                OpIndex OI, const std::vector<CompGeom>& cgh, const cplx* free_ops, const cplx* reac_ops,
                const cplx* M, cplx* Z, int* err, cudaStream_t st, cudaEvent_t gemm0, cudaEvent_t gemm1,
                double* gemm_flops) {
  Workspace& ws = h->W();
  TcCache& tc = h->tc;
  const int p = h->p, P = (p + 1) * (p + 1);
  const int np = (p + 1) * (p + 2) / 2, nm = p * (p + 1) / 2;
  // comp and level of every run (from its first pair)
  std::vector<int> rs(nruns + 1, 0);
  for (int r = 0; r < nruns; ++r) rs[r + 1] = rs[r] + hc[r];
  // run starts [nruns + 1], (comp, level) [2 nruns], parts [2 nruns]
  int* d_rs = (int*)tc_need(ws.tc_runs, sizeof(int) * (size_t)(5 * nruns + 1) + 64);
  int* d_info = d_rs + (nruns + 1);
  int* d_part = d_info + 2 * (size_t)nruns;
  FMM_CHECK(cudaMemcpyAsync(d_rs, rs.data(), sizeof(int) * (nruns + 1), cudaMemcpyHostToDevice, st));
  launch_tc_run_info(nruns, d_rs, perm, owner, B, d_info, st);
  std::vector<int> info(2 * (size_t)nruns);
  FMM_CHECK(cudaMemcpyAsync(info.data(), d_info, sizeof(int) * 2 * (size_t)nruns, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  // degree-scale exponents of every (component, level): [E_in | E_out], shared
  // by the operator conversion and the gather so that both use the same ones
  const int nc = (int)cgh.size();
  std::vector<int> et((size_t)nc * 23 * 2 * (FMM_MAXP + 1), 0);
  for (int c = 0; c < nc; ++c)
    for (int l = 0; l < 23; ++l) {
      const double wl = cgh[c].h2 / (double)(1 << l);
      int* E = et.data() + ((size_t)c * 23 + l) * 2 * (FMM_MAXP + 1);
      for (int n = 0; n <= p; ++n) {
        E[n] = deg_exp(cgh[c].ks, wl, n);
        E[FMM_MAXP + 1 + n] = deg_exp(cgh[c].kt, wl, n);
      }
    }
  int* d_et = (int*)tc_need(ws.tc_etab, sizeof(int) * et.size() + 64);
  FMM_CHECK(cudaMemcpyAsync(d_et, et.data(), sizeof(int) * et.size(), cudaMemcpyHostToDevice, st));
  const int nph = 49 * (2 * p + 1);
  if (!tc.phase_ready) {
    tc.phase_f.ensure(sizeof(float2) * nph);
    LAUNCH(k_tc_phase_f32<<<(nph + 127) / 128, 128, 0, st>>>(nph, OI.phase, tc.phase_f.as<float2>()));
    tc.phase_ready = true;
  }

  std::vector<TcPart> parts;
  std::vector<int> run_part(2 * (size_t)nruns, -1);
  std::vector<TcOpJob> jobs;
  std::vector<TcItem> items;
  long a_bytes_total = 0, sig_total = 0;
  double macs = 0.0;
  struct PartDesc { long op_off; int R, C, in_off, basis; bool reac; };
  for (int r = 0; r < nruns; ++r) {
    const long off = (long)(hk[r] >> 1);
    const bool reac = hk[r] & 1;
    const int K = hc[r];
    const int comp = info[2 * r], lev = info[2 * r + 1];
    PartDesc pd[2];
    int npd = 0;
    if (!reac) pd[npd++] = {off, P, P, 0, 0, false};
    else {
      pd[npd++] = {off, np, np, 0, 1, true};
      if (nm) pd[npd++] = {off + (long)np * np, nm, nm, np, 2, true};
    }
    const int ntiles = (K + kTileM - 1) / kTileM;
    for (int q = 0; q < npd; ++q) {
      const PartDesc& d = pd[q];
      TcPart pt{};
      pt.C = d.C;
      pt.in_off = d.in_off;
      pt.Kc = (2 * d.C + kChunk - 1) / kChunk;
      pt.basis = d.basis;
      pt.a_off = a_bytes_total;
      pt.sig_off = sig_total;
      a_bytes_total += (long)ntiles * 2 * pt.Kc * kTileM * kRowBytes;
      sig_total += (long)ntiles * kTileM;
      run_part[2 * r + q] = (int)parts.size();
      parts.push_back(pt);
      macs += (double)K * d.R * d.C;
      // operator sub-blocks of at most 128 output rows (cached per operator)
      for (int r0 = 0; r0 < d.R; r0 += 128) {
        const int RB = std::min(128, d.R - r0);
        auto key = std::make_tuple(d.op_off, (int)d.reac, d.basis, r0);
        auto itc = tc.ops.find(key);
        TcOpRef ref;
        if (itc == tc.ops.end()) {
          ref.RB = RB;
          ref.r0 = r0;
          ref.R16 = (RB + 15) / 16 * 16;
          ref.N_pad = 2 * ref.R16;
          ref.dst_off = tc.b_used;
          ref.scale_off = tc.s_used;
          const long bbytes = 2L * pt.Kc * ref.N_pad * kRowBytes;
          tc.b_used += bbytes;
          tc.s_used += RB;
          TcOpJob jb{};
          jb.src_off = d.op_off;
          jb.dst_off = ref.dst_off;
          jb.scale_off = ref.scale_off;
          jb.R_full = d.R;
          jb.C = d.C;
          jb.r0 = r0;
          jb.RB = RB;
          jb.R16 = ref.R16;
          jb.N_pad = ref.N_pad;
          jb.Kc = pt.Kc;
          jb.basis = d.basis;
          jb.etab_off = (comp * 23 + lev) * 2 * (FMM_MAXP + 1);
          jobs.push_back(jb);
          tc.ops[key] = ref;
          tc.pending_reac.push_back(d.reac);
        } else {
          ref = itc->second;
        }
        for (int t = 0; t < ntiles; ++t) {
          TcItem ti{};
          ti.a_off = pt.a_off + (long)t * 2 * pt.Kc * kTileM * kRowBytes;
          ti.b_off = ref.dst_off;
          ti.scale_off = ref.scale_off;
          ti.sig_off = pt.sig_off + (long)t * kTileM;
          ti.z_row0 = rs[r] + (long)t * kTileM;
          ti.rows = std::min(kTileM, K - t * kTileM);
          ti.RB = ref.RB;
          ti.R16 = ref.R16;
          ti.N_pad = ref.N_pad;
          ti.Kc = pt.Kc;
          ti.z_col0 = d.in_off + r0;
          items.push_back(ti);
        }
      }
    }
  }
  *gemm_flops = 8.0 * macs;
  double tflops = 0.0;
  for (const TcItem& t : items) tflops += 3.0 * 2.0 * kTileM * t.N_pad * (double)(t.Kc * kChunk);
  h->stats.m2l_tensor_flops = tflops;
  {
    double bytes = (double)a_bytes_total;                        // gathered tiles, read once
    std::map<long, double> ops_used;                             // operator sub-blocks, read once each
    for (const TcItem& t : items) {
      ops_used[t.b_off] = 2.0 * t.Kc * t.N_pad * (double)kRowBytes;
      bytes += (double)t.rows * t.RB * sizeof(cplx);              // translated columns written
    }
    for (auto& kv : ops_used) bytes += kv.second;
    h->stats.m2l_tc_bytes = bytes;
  }
  // operator conversions (new classes only)
  if (!jobs.empty()) {
    tc.bbuf.grow_keep(std::max<size_t>((size_t)tc.b_used, 256), (size_t)(tc.b_used_done), st);
    tc.sbuf.grow_keep(sizeof(int) * std::max<size_t>((size_t)tc.s_used, 32), sizeof(int) * (size_t)tc.s_done, st);
    // free-space and reaction operators live in different FP64 buffers: two launches
    std::vector<TcOpJob> jf, jr;
    for (size_t i = 0; i < jobs.size(); ++i) (tc.pending_reac[i] ? jr : jf).push_back(jobs[i]);
    tc.pending_reac.clear();
    TcOpJob* dj = (TcOpJob*)tc_need(ws.tc_jobs, sizeof(TcOpJob) * jobs.size() + 64);
    std::vector<TcOpJob> all = jf;
    all.insert(all.end(), jr.begin(), jr.end());
    FMM_CHECK(cudaMemcpyAsync(dj, all.data(), sizeof(TcOpJob) * all.size(), cudaMemcpyHostToDevice, st));
    if (!jf.empty())
      LAUNCH(k_tc_prep_ops<<<(unsigned)jf.size(), 256, 0, st>>>(dj, free_ops, tc.bbuf.as<unsigned char>(),
                                                               tc.sbuf.as<int>(), d_et));
    if (!jr.empty())
      LAUNCH(k_tc_prep_ops<<<(unsigned)jr.size(), 256, 0, st>>>(dj + jf.size(), reac_ops,
                                                               tc.bbuf.as<unsigned char>(), tc.sbuf.as<int>(), d_et));
    FMM_CHECK(cudaGetLastError());
    tc.b_used_done = tc.b_used;
    tc.s_done = tc.s_used;
    FMM_CHECK(cudaStreamSynchronize(st));     // the job table is rewritten by the next call
  }
  // A tiles
  unsigned char* Abuf = (unsigned char*)tc_need(ws.tc_a, (size_t)a_bytes_total + 256);
  int* isig = (int*)tc_need(ws.tc_sig, sizeof(int) * (size_t)sig_total + 64);
  TcPart* dparts = (TcPart*)tc_need(ws.tc_parts, sizeof(TcPart) * parts.size() + 64);
  FMM_CHECK(cudaMemcpyAsync(dparts, parts.data(), sizeof(TcPart) * parts.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(d_part, run_part.data(), sizeof(int) * run_part.size(), cudaMemcpyHostToDevice, st));
  LAUNCH(k_tc_gather<<<(unsigned)nv, 64, sizeof(float2) * 2 * P, st>>>(nv, p, perm, owner, vidx, B, OI, M, d_rs,
                                                                       nruns, d_part, dparts, d_et,
                                                                       tc.phase_f.as<float2>(), Abuf, isig));
  // products
  TcItem* ditems = (TcItem*)tc_need(ws.tc_items, sizeof(TcItem) * items.size() + 64);
  FMM_CHECK(cudaMemcpyAsync(ditems, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice, st));
  int max_np = 16;
  for (const TcItem& t : items) max_np = std::max(max_np, t.N_pad);
  // pipeline stages and shared memory (tiling.h): two stages when two CTAs
  // still fit on an SM, otherwise one, so that two CTAs share the SM
  const int nst = tiling::tc_stages(max_np);
  const size_t smem = tiling::tc_smem(max_np);
  FMM_CHECK(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FMM_CHECK(cudaEventRecord(gemm0, st));
  if (!items.empty())
    LAUNCH(k_m2l_tc<<<(unsigned)items.size(), 128, smem, st>>>(ditems, Abuf, tc.bbuf.as<unsigned char>(),
                                                              tc.sbuf.as<int>(), isig, Z, P, err,
                                                              (h->flags & FMM_TEST_STALL_TC) ? 16u : 0u, nst));
  FMM_CHECK(cudaEventRecord(gemm1, st));
  FMM_CHECK(cudaGetLastError());
  FMM_CHECK(cudaStreamSynchronize(st));       // host tables above go out of scope
}

__global__ void k_tc_run_info(int nruns, const int* __restrict__ rs, const int* __restrict__ perm,
                              const int* __restrict__ owner, BoxGeom B, int* __restrict__ info) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  int T = owner[perm[rs[r]]];
  info[2 * r] = B.comp[T];
  info[2 * r + 1] = B.lev[T];
}

void launch_tc_run_info(int nruns, const int* rs, const int* perm, const int* owner, BoxGeom B, int* info,
                        cudaStream_t st) {
  if (nruns) LAUNCH(k_tc_run_info<<<(nruns + 127) / 128, 128, 0, st>>>(nruns, rs, perm, owner, B, info));
}

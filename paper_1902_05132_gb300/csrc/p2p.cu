// Near-field (direct) interactions and the all-pairs direct sum.
//
// Free space: e^{ik r} / (4 pi r), skipped for bitwise-identical points.
// Reaction component (l, l', a, b) between a target at height zt = |z - d| on
// its side of the reference interface d and an image at depth zs = |z* - d|:
//   u~ = (i/4pi) int k_rho J_0(k_rho rho) e^{i k_lz zt + i k_l'z zs} sigma^{ab}/k_lz dk_rho
// (eq. generalcomponentsimag after the alpha integral).  The integral is taken
// on the rule's contour up to t_max = ta + 30 / (zt + zs), where the
// integrand has decayed below e^{-30} of its scale; on the real tail every
// factor is real and the integrand is evaluated in real arithmetic.
#include <cmath>
#include <vector>

#include "async_copy.cuh"
#include "fmm_internal.h"




__device__ inline int rule_nodes(const RuleView& R, double tmax) {
  if (tmax <= R.ta) return R.n_near;
  int np = (int)ceil((tmax - R.ta) / R.panel);
  if (np > R.n_panels) np = R.n_panels;
  return R.n_near + R.per_panel * np;
}

// J_0(z), complex z: power series for |z| <= 8, Miller's recurrence beyond.
__device__ inline cplx j0c(cplx z) {
  if (cabs2(z) <= 64.0) return j0_series(z);
  cplx J[1];
  besselJ_all(0, z, J);
  return J[0];
}

// One reaction pair on the rule (coef already holds sigma for the component).
__device__ inline cplx reac_pair(const RuleView& R, const cplx* __restrict__ coef, const cplx* __restrict__ kzl,
                                 const cplx* __restrict__ kzp, double rho, double zt, double zs, int* nq_out = nullptr) {
  int nq = rule_nodes(R, R.ta + FMM_NEAR_TAIL_DECAY / (zt + zs));
  if (nq_out) *nq_out = nq;
  cplx acc = C(0, 0);
  for (int q = 0; q < R.n_near; ++q) {
    cplx e = cexp_(cadd(cmul(C(0, zt), kzl[q]), cmul(C(0, zs), kzp[q])));
    cplx J = j0c(cscale(R.kr[q], rho));
    cfma(acc, cmul(J, e), coef[q]);
  }
  double tail = 0.0;
  for (int q = R.n_near; q < nq; ++q) {
    double t = R.kr[q].x;
    // k_z = i kappa on the real axis beyond every k_j
    double e = exp(-(kzl[q].y * zt + kzp[q].y * zs));
    tail += coef[q].x * j0(t * rho) * e;
  }
  return cadd(acc, C(tail, 0.0));
}

// Reaction component `slot` of one pair: the learned surrogate where it is
// trained and its held-out check passed for the cell of (rho, zt, zs), the
// quadrature everywhere else.
__device__ inline cplx reac_value(const RuleView& R, int slot, const cplx* __restrict__ coef,
                                  const cplx* __restrict__ kzl, const cplx* __restrict__ kzp, double rho, double zt,
                                  double zs, int* nq_out = nullptr) {
  if (R.surr.w) {
    float x[3];
    int cell;
    if (surr_inputs(R.surr, rho, zt, zs, x, &cell) && R.surr.ok[slot * SURR_CELLS + cell]) {
      float2 y = surr_forward(R.surr.w + (long)slot * 2 * SURR_NINF, x, cell);
      double h = zt + zs;
      double f = 1.0 / (4.0 * FMM_PI * sqrt(rho * rho + h * h));
      if (nq_out) *nq_out = 0;
      return C((double)y.x * f, (double)y.y * f);
    }
  }
  return reac_pair(R, coef, kzl, kzp, rho, zt, zs, nq_out);
}





#define NEAR_CHUNK 128
// One CTA (128 threads) per target leaf: thread pairs (t, t + 64) share a
// target and take alternate sources; the two halves are added at the end in
// a fixed order.
// F32 (mixed-precision form, free-space pairs only): positions relative to
// the leaf's first target (one FP64 subtraction per point, exact enough that
// r keeps ~1e-7 relative accuracy at the near-field distances), the kernel
// e^{ikr}/(4 pi r) in FP32, and a compensated (Kahan) FP32 sum per target
// that is added to the FP64 accumulator once per target.
template <bool F32>
__global__ void k_near(const int* __restrict__ leaves, NearBoxes B, const NearComp* __restrict__ ncs,
                       RuleView R, const double* __restrict__ spos, const cplx* __restrict__ sq,
                       const double* __restrict__ tpos, cplx* __restrict__ phi,
                       unsigned long long* __restrict__ counters) {
  unsigned long long my_pairs = 0, my_nodes = 0, my_surr = 0;
  int T = leaves[blockIdx.x];
  const NearComp nc = ncs[B.comp[T]];
  __shared__ double sx[NEAR_CHUNK], sy[NEAR_CHUNK], sz[NEAR_CHUNK];
  __shared__ cplx sqs[NEAR_CHUNK];
  __shared__ cplx half1[64];
  __shared__ float fx[F32 ? NEAR_CHUNK : 1], fy[F32 ? NEAR_CHUNK : 1], fz[F32 ? NEAR_CHUNK : 1];
  __shared__ float2 fq[F32 ? NEAR_CHUNK : 1];
  const bool f32 = F32 && nc.kind == CK_FREE;
  double ox = 0, oy = 0, oz = 0;               // anchor of the relative positions
  if (f32) { ox = tpos[3 * B.tb[T]]; oy = tpos[3 * B.tb[T] + 1]; oz = tpos[3 * B.tb[T] + 2]; }
  const float kf = (float)nc.k;
  const float inv4pif = (float)(1.0 / (4.0 * FMM_PI));
  const cplx* coef = R.coef + nc.coef_off;
  const cplx* kzl = R.kz + (long)nc.l * R.Q;
  const cplx* kzp = R.kz + (long)nc.lp * R.Q;
  const int lane_t = threadIdx.x & 63, par = threadIdx.x >> 6;
  const double k = nc.k;
  const double inv4pi = 1.0 / (4.0 * FMM_PI);
  for (int t0 = B.tb[T]; t0 < B.te[T]; t0 += 64) {
    int t = t0 + lane_t;
    bool act = t < B.te[T];
    double x = 0, y = 0, z = 0;
    if (act) { x = tpos[3 * t]; y = tpos[3 * t + 1]; z = tpos[3 * t + 2]; }
    cplx acc = C(0, 0);
    const float xr = (float)(x - ox), yr = (float)(y - oy), zr = (float)(z - oz);
    float ar = 0.f, cr = 0.f, ai = 0.f, ci = 0.f;    // compensated FP32 sums
    // list walk: U(T), W(T), then X(A) for A = T and its ancestors
    int A = T;
    int phase = 0;   // 0: U, 1: W, 2: X of A
    int e = B.uo[T], e_end = B.uo[T + 1];
    while (true) {
      while (e >= e_end) {
        if (phase == 0) { phase = 1; e = B.wo[T]; e_end = B.wo[T + 1]; }
        else if (phase == 1) { phase = 2; A = T; e = B.xo[A]; e_end = B.xo[A + 1]; }
        else {
          A = B.parent[A];
          if (A < 0) break;
          e = B.xo[A]; e_end = B.xo[A + 1];
        }
      }
      if (phase == 2 && A < 0) break;
      int S = (phase == 0) ? B.ui[e] : (phase == 1) ? B.wi[e] : B.xi[e];
      ++e;
      for (int s0 = B.sb[S]; s0 < B.se[S]; s0 += NEAR_CHUNK) {
        int ns = min(NEAR_CHUNK, B.se[S] - s0);
        __syncthreads();
        for (int kk = threadIdx.x; kk < ns; kk += blockDim.x) {
          sx[kk] = spos[3 * (s0 + kk)]; sy[kk] = spos[3 * (s0 + kk) + 1]; sz[kk] = spos[3 * (s0 + kk) + 2];
          sqs[kk] = sq[s0 + kk];
          if (F32 && f32) {
            fx[kk] = (float)(sx[kk] - ox); fy[kk] = (float)(sy[kk] - oy); fz[kk] = (float)(sz[kk] - oz);
            fq[kk] = make_float2((float)sqs[kk].x, (float)sqs[kk].y);
          }
        }
        __syncthreads();
        if (act) {
          if (F32 && f32) {
            for (int kk = par; kk < ns; kk += 2) {
              float dx = xr - fx[kk], dy = yr - fy[kk], dz = zr - fz[kk];
              if (dx == 0.f && dy == 0.f && dz == 0.f && x == sx[kk] && y == sy[kk] && z == sz[kk]) continue;
              float r2 = dx * dx + dy * dy + dz * dz;
              float rinv = rsqrtf(r2);
              float sn, cs;
              sincosf(kf * (r2 * rinv), &sn, &cs);
              float f = rinv * inv4pif;
              float2 qv = fq[kk];
              float tr = f * (cs * qv.x - sn * qv.y), ti = f * (cs * qv.y + sn * qv.x);
              float yv = tr - cr, tt = ar + yv;
              cr = (tt - ar) - yv; ar = tt;
              yv = ti - ci; tt = ai + yv;
              ci = (tt - ai) - yv; ai = tt;
              ++my_pairs;
            }
          } else if (nc.kind == CK_FREE) {
            for (int kk = par; kk < ns; kk += 2) {
              double dx = x - sx[kk], dy = y - sy[kk], dz = z - sz[kk];
              if (dx == 0.0 && dy == 0.0 && dz == 0.0) continue;   // bitwise-identical points (j = i)
              double r2 = dx * dx + dy * dy + dz * dz;
              double rinv = rsqrt(r2);
              double r = r2 * rinv;
              double sn, cs;
              sincos(k * r, &sn, &cs);
              double f = rinv * inv4pi;
              cfma(acc, C(cs * f, sn * f), sqs[kk]);
              ++my_pairs;
            }
          } else {
            double zt = fabs(z - nc.dref);
            for (int kk = par; kk < ns; kk += 2) {
              double dx = x - sx[kk], dy = y - sy[kk];
              double rho = sqrt(dx * dx + dy * dy);
              double zs = fabs(sz[kk] - nc.dref);
              int nq;
              cfma(acc, reac_value(R, (int)(nc.coef_off / R.Q), coef, kzl, kzp, rho, zt, zs, &nq), sqs[kk]);
              ++my_pairs;
              my_nodes += nq;
              my_surr += (nq == 0);
            }
          }
        }
      }
    }
    if (F32 && f32) acc = cadd(acc, C((double)ar - (double)cr, (double)ai - (double)ci));
    __syncthreads();
    if (par == 1) half1[lane_t] = acc;
    __syncthreads();
    if (par == 0 && act) phi[t] = cadd(phi[t], cadd(acc, half1[lane_t]));
  }
  if (counters && my_pairs) {
    atomicAdd(&counters[0], my_pairs);
    atomicAdd(&counters[1], my_nodes);
    if (my_surr) atomicAdd(&counters[2], my_surr);
  }
  if (B.comp_pairs && my_pairs) atomicAdd(&B.comp_pairs[B.comp[T]], my_pairs);
}

// Free-space near field in FP64 (U, W and X lists of free-space target
// leaves; eq. totalinteraction, j != i): one CTA of 256 threads per target
// leaf.  The sources of U(T), W(T) and X(A) for A = T and its ancestors are
// gathered in chunks of up to NF_CH points: one thread issues one
// cp.async.bulk per source-box piece for its positions (the 16-byte aligned
// cover of the piece's bytes) and one for its charges, all completing on one
// mbarrier (bounded wait); the CTA then unpacks the positions into
// structure-of-arrays form (the charges land contiguous already).  Warp w
// takes targets t = tb + w, tb + w + 8, ...; its lanes split the chunk's
// sources (lane i: sources i, i + 32, ...) and the partial sums of a target
// are added by a warp-shuffle reduction, then into the target's sum in
// shared memory, chunk after chunk in a fixed order.  Targets are taken 256
// per pass.  On an expired wait the kernel sets bit 32 of *err, waits once
// more (bounded) for its copies and returns.
constexpr int NF_THREADS = 256;
constexpr int NF_CH = 1024;                 // source points per chunk
constexpr int NF_SEG = 64;                  // source-box pieces per chunk
constexpr int NF_TG = 256;                  // targets per pass
constexpr int NF_RAWP = 24 * NF_CH + 16 * NF_SEG;
// shared memory: raw positions, charges, x/y/z, target sums, 4 piece
// tables, a 16-byte header (pieces, points) and the mbarrier
constexpr size_t NF_SMEM = (size_t)NF_RAWP + 16 * NF_CH + 24 * NF_CH + 16 * NF_TG + 4 * 4 * NF_SEG + 16 + 8;

__device__ inline void warp_sum(cplx& v);

__global__ void __launch_bounds__(NF_THREADS) k_near_free(const int* __restrict__ leaves, NearBoxes B,
                                                         const NearComp* __restrict__ ncs,
                                                         const double* __restrict__ spos,
                                                         const cplx* __restrict__ sq,
                                                         const double* __restrict__ tpos, cplx* __restrict__ phi,
                                                         unsigned long long* __restrict__ counters,
                                                         int* __restrict__ err) {
  const int T = leaves[blockIdx.x];
  const double k = ncs[B.comp[T]].k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ __align__(128) unsigned char nf_sm[];
  unsigned char* raw_pos = nf_sm;                                   // [NF_RAWP] bytes
  cplx* sqv = (cplx*)(raw_pos + NF_RAWP);                           // [NF_CH] charges (copied in place)
  double* sx = (double*)(sqv + NF_CH);                              // [NF_CH] x, y, z
  double* sy = sx + NF_CH;
  double* sz = sy + NF_CH;
  cplx* acc = (cplx*)(sz + NF_CH);                                  // [NF_TG] target sums
  int* seg_src = (int*)(acc + NF_TG);                               // first source of each piece
  int* seg_n = seg_src + NF_SEG;                                    // its points
  int* seg_at = seg_n + NF_SEG;                                     // its first slot in the chunk
  int* seg_raw = seg_at + NF_SEG;                                   // byte offset of its first point in raw_pos
  int* hdr = seg_raw + NF_SEG;                                      // [0]: pieces, [1]: points
  unsigned long long* bar = (unsigned long long*)(hdr + 4);
  const uint32_t bar_a = smem_u32(bar);
  if (threadIdx.x == 0) {
    mbar_init(bar_a, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const double inv4pi = 1.0 / (4.0 * FMM_PI);
  unsigned long long my_pairs = 0;
  uint32_t parity = 0;
  for (int tg0 = B.tb[T]; tg0 < B.te[T]; tg0 += NF_TG) {
    const int ntg = min(NF_TG, B.te[T] - tg0);
    for (int i = threadIdx.x; i < ntg; i += NF_THREADS) acc[i] = C(0, 0);
    // list walk (thread 0): U(T), W(T), then X(A) for A = T and its ancestors
    int phase = 0, A = T, e = B.uo[T], e_end = B.uo[T + 1], s_cur = 0, s_end = 0;
    while (true) {
      if (threadIdx.x == 0) {
        int nseg = 0, npts = 0;
        uint32_t rawp = 0, bytes = 0;
        // the pieces of this chunk first, then the copies (the barrier must
        // expect every byte before the first copy can complete)
        while (npts < NF_CH && nseg < NF_SEG) {
          if (s_cur >= s_end) {               // next source box of the lists
            while (e >= e_end && !(phase == 2 && A < 0)) {
              if (phase == 0) { phase = 1; e = B.wo[T]; e_end = B.wo[T + 1]; }
              else if (phase == 1) { phase = 2; A = T; e = B.xo[A]; e_end = B.xo[A + 1]; }
              else {
                A = B.parent[A];
                if (A >= 0) { e = B.xo[A]; e_end = B.xo[A + 1]; }
              }
            }
            if (phase == 2 && A < 0) break;
            const int S = (phase == 0) ? B.ui[e] : (phase == 1) ? B.wi[e] : B.xi[e];
            ++e;
            s_cur = B.sb[S];
            s_end = B.se[S];
            continue;
          }
          const int n = min(s_end - s_cur, NF_CH - npts);
          const unsigned long long b0 = 24ull * (unsigned long long)s_cur;
          const unsigned long long a0 = b0 & ~15ull, a1 = (b0 + 24ull * n + 15ull) & ~15ull;
          const uint32_t lb = (uint32_t)(a1 - a0);
          seg_src[nseg] = s_cur;
          seg_n[nseg] = n;
          seg_at[nseg] = npts;
          seg_raw[nseg] = (int)(rawp + (uint32_t)(b0 - a0));
          rawp += lb;
          bytes += lb + 16u * n;
          s_cur += n;
          npts += n;
          ++nseg;
        }
        if (nseg) {
          mbar_expect_tx(bar_a, bytes);       // the one arrival of this phase
          for (int g = 0; g < nseg; ++g) {
            const int s0 = seg_src[g], n = seg_n[g];
            const unsigned long long b0 = 24ull * (unsigned long long)s0;
            const unsigned long long a0 = b0 & ~15ull, a1 = (b0 + 24ull * n + 15ull) & ~15ull;
            bulk_g2s(smem_u32(raw_pos + (seg_raw[g] - (int)(b0 - a0))), (const unsigned char*)spos + a0,
                     (uint32_t)(a1 - a0), bar_a);
            bulk_g2s(smem_u32(sqv + seg_at[g]), sq + s0, 16u * n, bar_a);
          }
        }
        hdr[0] = nseg;
        hdr[1] = npts;
      }
      __syncthreads();
      const int nseg = hdr[0], npts = hdr[1];
      if (nseg == 0) break;
      const bool ok = mbar_wait(bar_a, parity);
      parity ^= 1u;
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicOr(err, 32);
        mbar_wait(bar_a, parity ^ 1u);        // the copies of this phase, once more (bounded)
        return;
      }
      // unpack the positions
      for (int j = threadIdx.x; j < npts; j += NF_THREADS) {
        int g = 0;
        while (g + 1 < nseg && seg_at[g + 1] <= j) ++g;
        const double* p = (const double*)(raw_pos + seg_raw[g]) + 3 * (j - seg_at[g]);
        sx[j] = p[0];
        sy[j] = p[1];
        sz[j] = p[2];
      }
      __syncthreads();
      for (int ti = warp; ti < ntg; ti += NF_THREADS / 32) {
        const int t = tg0 + ti;
        const double x = tpos[3 * t], y = tpos[3 * t + 1], z = tpos[3 * t + 2];
        cplx part = C(0, 0);
        for (int j = lane; j < npts; j += 32) {
          const double dx = x - sx[j], dy = y - sy[j], dz = z - sz[j];
          if (dx == 0.0 && dy == 0.0 && dz == 0.0) continue;   // bitwise-identical points (j = i)
          const double r2 = dx * dx + dy * dy + dz * dz;
          const double rinv = rsqrt(r2);
          double sn, cs;
          sincos(k * (r2 * rinv), &sn, &cs);
          const double f = rinv * inv4pi;
          cfma(part, C(cs * f, sn * f), sqv[j]);
          ++my_pairs;
        }
        warp_sum(part);
        if (lane == 0) acc[ti] = cadd(acc[ti], part);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < ntg; i += NF_THREADS) phi[tg0 + i] = cadd(phi[tg0 + i], acc[i]);
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, o);
  if (lane == 0 && my_pairs) {
    if (counters) atomicAdd(&counters[0], my_pairs);
    if (B.comp_pairs) atomicAdd(&B.comp_pairs[B.comp[T]], my_pairs);
  }
}

// Reaction components of the near field (U, W and X lists of reaction target
// leaves; eq. generalcomponentsimag): one CTA per target leaf, one warp per
// target (targets of the leaf strided over the warps).  The warp streams the
// sources of the lists 32 at a time, one per lane.  Pairs whose cell the
// surrogate covers are evaluated by their own lane (network forward pass);
// the pairs left to the quadrature are then taken one at a time by the whole
// warp, the lanes splitting the contour nodes (lane i takes nodes i, i + 32,
// ...).  Every lane keeps a partial sum of q_s times its share; the partials
// of a target are added by one warp-shuffle reduction in a fixed order.
// box[0..2] (if given) receive max rho, min and max of zt and zs over the
// pairs, as the bit patterns of non-negative doubles (ordered like the values).
__device__ inline void warp_sum(cplx& v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
}

// Work items: (leaf, first target) pairs, up to 4 targets each (one per
// warp), so that the targets with the costliest pairs (those next to the
// interface, where the quadrature takes the most nodes) spread over many
// CTAs; only leaves with near-field entries get items.
__global__ void __launch_bounds__(128) k_near_reac(const int* __restrict__ items, NearBoxes B,
                                                   const NearComp* __restrict__ ncs, RuleView R,
                                                   const double* __restrict__ spos, const cplx* __restrict__ sq,
                                                   const double* __restrict__ tpos, cplx* __restrict__ phi,
                                                   unsigned long long* __restrict__ counters,
                                                   unsigned long long* __restrict__ box) {
  const int T = items[2 * blockIdx.x], t_first = items[2 * blockIdx.x + 1];
  const int t_end = min(B.te[T], t_first + 4);
  const NearComp nc = ncs[B.comp[T]];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = (int)(nc.coef_off / R.Q);
  // the hidden layers of the component's network, summed to FP32, in shared
  // memory (only when a surrogate is attached: the launch then gives
  // SURR_NTRUNK floats); the cell output layers stay in global memory
  extern __shared__ float s_net[];
  const __nv_bfloat16* net = R.surr.w ? R.surr.w + (long)slot * 2 * SURR_NINF : nullptr;
  if (net) {
    for (int i = threadIdx.x; i < SURR_NTRUNK; i += blockDim.x)
      s_net[i] = __bfloat162float(net[i]) + __bfloat162float(net[SURR_NINF + i]);
    __syncthreads();
  }
  const cplx* coef = R.coef + nc.coef_off;
  const cplx* kzl = R.kz + (long)nc.l * R.Q;
  const cplx* kzp = R.kz + (long)nc.lp * R.Q;
  unsigned long long my_pairs = 0, my_nodes = 0, my_surr = 0, my_tab = 0;
  double rho_hi = 0.0, z_lo = INFINITY, z_hi = 0.0;
  for (int t = t_first + warp; t < t_end; t += 4) {
    const double x = tpos[3 * t], y = tpos[3 * t + 1];
    const double zt = fabs(tpos[3 * t + 2] - nc.dref);
    cplx acc = C(0, 0);
    int A = T, phase = 0;                  // 0: U(T), 1: W(T), 2: X(A), A = T and its ancestors
    int e = B.uo[T], e_end = B.uo[T + 1];
    while (true) {
      while (e >= e_end) {
        if (phase == 0) { phase = 1; e = B.wo[T]; e_end = B.wo[T + 1]; }
        else if (phase == 1) { phase = 2; A = T; e = B.xo[A]; e_end = B.xo[A + 1]; }
        else {
          A = B.parent[A];
          if (A < 0) break;
          e = B.xo[A]; e_end = B.xo[A + 1];
        }
      }
      if (phase == 2 && A < 0) break;
      const int S = (phase == 0) ? B.ui[e] : (phase == 1) ? B.wi[e] : B.xi[e];
      ++e;
      for (int s0 = B.sb[S]; s0 < B.se[S]; s0 += 32) {
        const int s = s0 + lane;
        const bool valid = s < B.se[S];
        double rho = 0.0, zs = 1.0;
        cplx qs = C(0, 0);
        bool by_net = false;
        if (valid) {
          const double dx = x - spos[3 * s], dy = y - spos[3 * s + 1];
          rho = sqrt(dx * dx + dy * dy);
          zs = fabs(spos[3 * s + 2] - nc.dref);
          qs = sq[s];
          rho_hi = fmax(rho_hi, rho);
          z_lo = fmin(z_lo, fmin(zt, zs));
          z_hi = fmax(z_hi, fmax(zt, zs));
          ++my_pairs;
          if (R.surr.w) {
            float xin[3];
            int cell;
            if (surr_inputs(R.surr, rho, zt, zs, xin, &cell) && R.surr.ok[slot * SURR_CELLS + cell]) {
              const float2 v = surr_forward_f32(s_net, net, xin, cell);
              const double f = 1.0 / (4.0 * FMM_PI * sqrt(rho * rho + (zt + zs) * (zt + zs)));
              cfma(acc, C((double)v.x * f, (double)v.y * f), qs);
              by_net = true;
              ++my_surr;
            }
          }
          if (!by_net && R.ntab.vals) {
            // tabulated kernel (FMM_TABLES) where the pair lies inside the table
            cplx v;
            if (near_table_eval(R.ntab, slot, rho, zt, zs, &v)) {
              cfma(acc, v, qs);
              by_net = true;
              ++my_tab;
            }
          }
        }
        unsigned todo = __ballot_sync(0xffffffffu, valid && !by_net);
        while (todo) {
          const int j = __ffs(todo) - 1;
          todo &= todo - 1;
          const double rj = __shfl_sync(0xffffffffu, rho, j), zsj = __shfl_sync(0xffffffffu, zs, j);
          const cplx qj = C(__shfl_sync(0xffffffffu, qs.x, j), __shfl_sync(0xffffffffu, qs.y, j));
          const int nq = rule_nodes(R, R.ta + FMM_NEAR_TAIL_DECAY / (zt + zsj));
          cplx part = C(0, 0);
          for (int qn = lane; qn < R.n_near; qn += 32) {
            cplx ex = cexp_(cadd(cmul(C(0, zt), kzl[qn]), cmul(C(0, zsj), kzp[qn])));
            cplx J = j0c(cscale(R.kr[qn], rj));
            cfma(part, cmul(J, ex), coef[qn]);
          }
          double tail = 0.0;
          if (R.tail_f32) {
            // mixed form: the real tail (every factor real, the integrand a
            // decaying, oscillating sum) in FP32 with a compensated sum
            const float rf = (float)rj, ztf = (float)zt, zsf = (float)zsj;
            float sum = 0.0f, cmp = 0.0f;
            for (int qn = R.n_near + lane; qn < nq; qn += 32) {
              const float term = (float)coef[qn].x * j0f((float)R.kr[qn].x * rf) *
                                 expf(-((float)kzl[qn].y * ztf + (float)kzp[qn].y * zsf));
              const float y = term - cmp, tt = sum + y;
              cmp = (tt - sum) - y;
              sum = tt;
            }
            tail = (double)sum - (double)cmp;
          } else {
            for (int qn = R.n_near + lane; qn < nq; qn += 32) {
              const double tq = R.kr[qn].x;
              tail += coef[qn].x * j0(tq * rj) * exp(-(kzl[qn].y * zt + kzp[qn].y * zsj));
            }
          }
          part.x += tail;
          cfma(acc, part, qj);
          if (lane == 0) my_nodes += nq;
        }
      }
    }
    warp_sum(acc);
    if (lane == 0) phi[t] = cadd(phi[t], acc);
  }
  if (counters) {
    for (int o = 16; o > 0; o >>= 1) {
      my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, o);
      my_surr += __shfl_xor_sync(0xffffffffu, my_surr, o);
      my_tab += __shfl_xor_sync(0xffffffffu, my_tab, o);
    }
    if (lane == 0 && my_pairs) {
      atomicAdd(&counters[0], my_pairs);
      atomicAdd(&counters[1], my_nodes);
      if (my_surr) atomicAdd(&counters[2], my_surr);
      if (my_tab && B.tab_pairs) atomicAdd(B.tab_pairs, my_tab);
      if (B.comp_pairs) atomicAdd(&B.comp_pairs[B.comp[T]], my_pairs);
    }
  }
  if (box) {
    for (int o = 16; o > 0; o >>= 1) {
      rho_hi = fmax(rho_hi, __shfl_xor_sync(0xffffffffu, rho_hi, o));
      z_lo = fmin(z_lo, __shfl_xor_sync(0xffffffffu, z_lo, o));
      z_hi = fmax(z_hi, __shfl_xor_sync(0xffffffffu, z_hi, o));
    }
    if (lane == 0 && z_hi > 0.0) {
      atomicMax(&box[0], (unsigned long long)__double_as_longlong(rho_hi));
      atomicMin(&box[1], (unsigned long long)__double_as_longlong(z_lo));
      atomicMax(&box[2], (unsigned long long)__double_as_longlong(z_hi));
    }
  }
}

// All-pairs direct sum on the GPU: one thread per target, sources streamed
// through shared memory.  Reaction part: all (a, b) of the layer pair.


__global__ void k_direct(long nt, const double* __restrict__ tgt, long ns, const double* __restrict__ src,
                         const double* __restrict__ q, DirectMedium md, RuleView R,
                         const cplx* __restrict__ coef_all, double* __restrict__ out) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  __shared__ double sx[NEAR_CHUNK], sy[NEAR_CHUNK], sz[NEAR_CHUNK];
  __shared__ cplx sqs[NEAR_CHUNK];
  __shared__ int sl[NEAR_CHUNK];
  bool act = t < nt;
  double x = 0, y = 0, z = 0;
  int lt = 0;
  if (act) {
    x = tgt[3 * t]; y = tgt[3 * t + 1]; z = tgt[3 * t + 2];
    for (int j = 0; j < md.L1 - 1; ++j) if (z < md.d[j]) ++lt;
  }
  cplx acc = C(0, 0);
  for (long s0 = 0; s0 < ns; s0 += NEAR_CHUNK) {
    int nsb = (int)min((long)NEAR_CHUNK, ns - s0);
    __syncthreads();
    for (int k = threadIdx.x; k < nsb; k += blockDim.x) {
      long s = s0 + k;
      sx[k] = src[3 * s]; sy[k] = src[3 * s + 1]; sz[k] = src[3 * s + 2];
      sqs[k] = C(q[2 * s], q[2 * s + 1]);
      int l = 0;
      for (int j = 0; j < md.L1 - 1; ++j) if (sz[k] < md.d[j]) ++l;
      sl[k] = l;
    }
    __syncthreads();
    if (!act) continue;
    for (int k = 0; k < nsb; ++k) {
      int ls = sl[k];
      double dx = x - sx[k], dy = y - sy[k], dz = z - sz[k];
      if (ls == lt && !(dx == 0.0 && dy == 0.0 && dz == 0.0)) {
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double s, c;
        sincos(md.k[lt] * r, &s, &c);
        double f = 1.0 / (4.0 * FMM_PI * r);
        cfma(acc, C(c * f, s * f), sqs[k]);
      }
      if (md.L1 == 1) continue;
      double rho = sqrt(dx * dx + dy * dy);
      const cplx* kzl = R.kz + (long)lt * R.Q;
      const cplx* kzp = R.kz + (long)ls * R.Q;
      for (int a = 0; a < 2; ++a) {
        if (a == AR_UP ? !(lt < md.L1 - 1) : !(lt > 0)) continue;
        double zt = (a == AR_UP) ? (z - md.d[lt]) : (md.d[lt - 1] - z);
        for (int b = 0; b < 2; ++b) {
          if (b == AR_UP ? !(ls < md.L1 - 1) : !(ls > 0)) continue;
          double zs = (b == AR_UP) ? (sz[k] - md.d[ls]) : (md.d[ls - 1] - sz[k]);
          const int slot = ((lt * md.L1 + ls) * 2 + a) * 2 + b;
          const cplx* coef = coef_all + (long)slot * R.Q;
          cfma(acc, reac_value(R, slot, coef, kzl, kzp, rho, zt, zs), sqs[k]);
        }
      }
    }
  }
  if (act) {
    out[2 * t] = acc.x;
    out[2 * t + 1] = acc.y;
  }
}

// coef[(l,l',a,b)][q] = (i / 4 pi) w k_rho sigma^{ab}_{l l'} / k_lz
__global__ void k_coef(int L1, int Q, const cplx* __restrict__ kr, const cplx* __restrict__ w,
                       const cplx* __restrict__ kz, const cplx* __restrict__ sigma, cplx* __restrict__ coef) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long total = (long)L1 * L1 * 4 * Q;
  if (e >= total) return;
  int q = e % Q;
  long combo = e / Q;
  int l = (int)(combo / (L1 * 4));
  cplx v = cdiv(cmul(cmul(w[q], kr[q]), sigma[e]), kz[(long)l * Q + q]);
  coef[e] = cmul(C(0.0, 1.0 / (4.0 * FMM_PI)), v);
}

// out[tidx[i]] += phi[i] for one component's target segment
__global__ void k_scatter_add(long n, const int* __restrict__ tidx, const cplx* __restrict__ phi, double* __restrict__ out) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  long g = tidx[i];
  out[2 * g] += phi[i].x;
  out[2 * g + 1] += phi[i].y;
}

// paper normalization: multiply by 4 pi / (i k_l) for targets in layer l
__global__ void k_norm_paper(long n, const double* __restrict__ tgt, DirectMedium md, double* __restrict__ out) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double z = tgt[3 * i + 2];
  int l = 0;
  for (int j = 0; j < md.L1 - 1; ++j) if (z < md.d[j]) ++l;
  double f = 4.0 * FMM_PI / md.k[l];
  double re = out[2 * i], im = out[2 * i + 1];
  // (re + i im) * f / i = f * (im - i re)
  out[2 * i] = f * im;
  out[2 * i + 1] = -f * re;
}

// ---------------------------------------------------------------- launchers
void launch_coef(int L1, const Rule& R, cplx* coef, cudaStream_t st) {
  long total = (long)L1 * L1 * 4 * R.Q();
  LAUNCH(k_coef<<<(total + 255) / 256, 256, 0, st>>>(L1, R.Q(), R.kr.as<cplx>(), R.w.as<cplx>(), R.kz.as<cplx>(),
                                              R.sigma.as<cplx>(), coef));
}

RuleView make_rule_view(const Rule& R, const cplx* coef) {
  RuleView v;
  v.kr = R.kr.as<cplx>();
  v.coef = coef;
  v.kz = R.kz.as<cplx>();
  v.Q = R.Q();
  v.n_near = R.n_near;
  v.per_panel = R.per_panel;
  v.n_panels = R.n_tail_panels;
  v.ta = R.ta;
  v.panel = R.panel;
  v.surr = SurrView{};
  v.ntab = NearTabView{};
  v.tail_f32 = 0;
  return v;
}

// Training and held-out samples of the surrogate: points drawn uniformly in
// the box by a counter-based generator, stratified by cell (the samples of
// component si and cell c are e = si nper + c (nper / 64) + j, j < nper / 64,
// uniform within the cell), component values by the quadrature.
__global__ void k_surr_samples(long n, long nper, const int* __restrict__ slots, int L1, SurrView box,
                               RuleView R, unsigned long long seed, float* __restrict__ X, float* __restrict__ Y) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int slot = slots[e / nper];
  const int lp = (slot >> 2) % L1, l = (slot >> 2) / L1;      // slot = ((l L1 + l') 2 + a) 2 + b
  const int cell = (int)((e % nper) / (nper / SURR_CELLS));
  const int c0 = cell / (SURR_GRID * SURR_GRID), c1 = (cell / SURR_GRID) % SURR_GRID, c2 = cell % SURR_GRID;
  const double inv = 1.0 / SURR_GRID;
  double u0 = (c0 + surr_uniform(seed, 3 * e)) * inv, u1 = (c1 + surr_uniform(seed, 3 * e + 1)) * inv,
         u2 = (c2 + surr_uniform(seed, 3 * e + 2)) * inv;
  double rho = u0 * box.rho_max;
  double zt = box.z_min + u1 * (box.z_max - box.z_min), zs = box.z_min + u2 * (box.z_max - box.z_min);
  cplx u = reac_pair(R, R.coef + (long)slot * R.Q, R.kz + (long)l * R.Q, R.kz + (long)lp * R.Q, rho, zt, zs);
  double f = 4.0 * FMM_PI * sqrt(rho * rho + (zt + zs) * (zt + zs));
  X[3 * e] = (float)(2.0 * u0 - 1.0);
  X[3 * e + 1] = (float)(2.0 * u1 - 1.0);
  X[3 * e + 2] = (float)(2.0 * u2 - 1.0);
  Y[2 * e] = (float)(u.x * f);
  Y[2 * e + 1] = (float)(u.y * f);
}

void launch_surr_samples(long n, long nper, const int* slots, int L1, SurrView box, RuleView R,
                         unsigned long long seed, float* X, float* Y, cudaStream_t st) {
  if (n) LAUNCH(k_surr_samples<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, nper, slots, L1, box, R, seed, X, Y));
}

void launch_near_reac(const int* items, int n, NearBoxes B, const NearComp* ncs, RuleView R, const double* spos,
                      const cplx* sq, const double* tpos, cplx* phi, unsigned long long* counters,
                      unsigned long long* box, cudaStream_t st) {
  if (!n) return;
  const size_t smem = R.surr.w ? sizeof(float) * SURR_NTRUNK : 0;
  LAUNCH(k_near_reac<<<n, 128, smem, st>>>(items, B, ncs, R, spos, sq, tpos, phi, counters, box));
}

void launch_near(const int* leaves, int n, NearBoxes B, const NearComp* ncs, RuleView R, const double* spos,
                 const cplx* sq, const double* tpos, cplx* phi, unsigned long long* counters, int* err,
                 cudaStream_t st, bool f32) {
  if (!n) return;
  if (f32) {
    LAUNCH(k_near<true><<<n, 128, 0, st>>>(leaves, B, ncs, R, spos, sq, tpos, phi, counters));
  } else {
    FMM_CHECK(cudaFuncSetAttribute(k_near_free, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NF_SMEM));
    LAUNCH(k_near_free<<<n, NF_THREADS, NF_SMEM, st>>>(leaves, B, ncs, spos, sq, tpos, phi, counters, err));
  }
}

// Dependent FP64 FMA chains (8 independent chains per thread).
__global__ void k_fp64_peak(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

double measure_fp64_peak_impl() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int blocks = nsm * 8, threads = 256, iters = 20000;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    LAUNCH(k_fp64_peak<<<blocks, threads>>>(d, iters, 0.999999, 1e-7));
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  return 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e6);
}

void launch_direct(long nt, const double* tgt, long ns, const double* src, const double* q, DirectMedium md,
                   RuleView R, const cplx* coef_all, double* out, cudaStream_t st) {
  if (nt) LAUNCH(k_direct<<<(nt + 63) / 64, 64, 0, st>>>(nt, tgt, ns, src, q, md, R, coef_all, out));
}

void launch_scatter_add(long n, const int* tidx, const cplx* phi, double* out, cudaStream_t st) {
  if (n) LAUNCH(k_scatter_add<<<(n + 255) / 256, 256, 0, st>>>(n, tidx, phi, out));
}

void launch_norm_paper(long n, const double* tgt, DirectMedium md, double* out, cudaStream_t st) {
  if (n) LAUNCH(k_norm_paper<<<(n + 255) / 256, 256, 0, st>>>(n, tgt, md, out));
}

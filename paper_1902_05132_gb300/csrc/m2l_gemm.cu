// M2L as class-batched complex GEMMs.
//
// Every V-list pair (T, S) of every level is tagged with the operator it uses
// (free space: the (k, w, offset) slot; reaction: the radial class with the
// m-reflection split).  Pairs are sorted by operator, the source expansions
// are gathered as GEMM columns (rotated by e^{i m phi} and moved to the
// symmetric basis for reaction pairs), one tiled FP64 complex GEMM per
// operator produces the translated columns, and a per-target reduction adds
// them back in V-list order (deterministic), undoing the rotation.
#include "sort.h"

#include <algorithm>
#include <vector>

#include "fmm_internal.h"
#include "tiling.h"

// owner[e] = target box of V-list entry e
__global__ void k_v_owner(int nb, const int* __restrict__ voff, int* __restrict__ owner) {
  int T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= nb) return;
  for (int e = voff[T]; e < voff[T + 1]; ++e) owner[e] = T;
}

__device__ inline bool reac_class(const CompGeom& cg, int lev, const int* ct, const int* cs, const long* reac_off,
                                  int comp, long& off, int& phidx) {
  int dx = ct[0] - cs[0], dy = ct[1] - cs[1];
  int half = 1 << (lev - 1);
  int jt, js;
  if (cg.a == AR_UP) { jt = ct[2] - half; js = half - 1 - cs[2]; }
  else { jt = half - 1 - ct[2]; js = cs[2] - half; }
  const int tab[10] = {0, 1, 2, 4, 5, 8, 9, 10, 13, 18};
  int r = -1;
  for (int k = 0; k < 10; ++k) if (tab[k] == dx * dx + dy * dy) r = k;
  phidx = (dy + 3) * 7 + (dx + 3);
  if (jt < 0 || jt > 1 || js < 0 || js > 1 || r < 0) return false;
  off = reac_off[((long)comp * 23 + lev) * 40 + (jt * 2 + js) * 10 + r];
  return off >= 0;
}

// key[e] = operator offset (class), val[e] = e
__global__ void k_v_keys(long nv, const int* __restrict__ owner, const int* __restrict__ vidx, BoxGeom B,
                         OpIndex OI, int P, unsigned long long* __restrict__ key, int* __restrict__ val,
                         int* __restrict__ err) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= nv) return;
  int T = owner[e], S = vidx[e];
  int comp = B.comp[T], lev = B.lev[T];
  const CompGeom& cg = OI.cgs[comp];
  const int* ct = B.coord + 3 * T;
  const int* cs = B.coord + 3 * S;
  long off = 0;
  if (cg.kind == CK_FREE) {
    int dx = ct[0] - cs[0], dy = ct[1] - cs[1], dz = ct[2] - cs[2];
    off = OI.m2l_base[comp * 23 + lev] + (long)(((dz + 3) * 7 + (dy + 3)) * 7 + (dx + 3)) * P * P;
    key[e] = (unsigned long long)off << 1;
  } else {
    int ph;
    if (!reac_class(cg, lev, ct, cs, OI.reac_off, comp, off, ph)) {
      atomicOr(err, 8);
      off = 0;
    }
    key[e] = ((unsigned long long)off << 1) | 1ULL;
  }
  val[e] = (int)e;
}

// Y[k] = column of sorted pair k (P complex): M_S, or for reaction pairs the
// rotated expansion in the symmetric basis [plus (np) | minus (nm)].  One
// thread per output coefficient (each reads at most two coefficients of M_S).
__global__ void k_m2l_gather(long nv, int p, const int* __restrict__ perm, const int* __restrict__ owner,
                             const int* __restrict__ vidx, BoxGeom B, OpIndex OI, const cplx* __restrict__ M,
                             cplx* __restrict__ Y) {
  const int P = (p + 1) * (p + 1);
  const long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (g >= nv * P) return;
  const long k = g / P;
  const int a = (int)(g - k * P);
  const int e = perm[k];
  const int T = owner[e], S = vidx[e];
  const CompGeom& cg = OI.cgs[B.comp[T]];
  const cplx* Ms = M + (long)S * P;
  if (cg.kind == CK_FREE) {
    Y[g] = Ms[a];
    return;
  }
  const int* ct = B.coord + 3 * T;
  const int* cs = B.coord + 3 * S;
  const cplx* ph = OI.phase + ((ct[1] - cs[1] + 3) * 7 + (ct[0] - cs[0] + 3)) * (2 * p + 1) + p;
  const int np = (p + 1) * (p + 2) / 2;
  const bool plus = a < np;
  int n, m;
  if (plus) {
    n = 0;
    while ((n + 1) * (n + 2) / 2 <= a) ++n;
    m = a - n * (n + 1) / 2;
  } else {
    const int b = a - np;
    n = 1;
    while (n * (n + 1) / 2 <= b) ++n;
    m = b - n * (n - 1) / 2 + 1;
  }
  const cplx x0 = cmul(Ms[n * n + n + m], ph[m]);
  cplx u;
  if (m == 0) {
    u = x0;
  } else {
    const double s = (m & 1) ? -1.0 : 1.0;
    const cplx x1 = cscale(cmul(Ms[n * n + n - m], ph[-m]), s);
    u = cscale(plus ? cadd(x0, x1) : csub(x0, x1), 0.70710678118654752440);
  }
  Y[g] = u;
}

// Batched complex GEMM: for every batch, Z[k][r] = sum_c A[c][r] Y[k][c]
// (A input-major with leading dimension R; Y, Z with strides ldy, ldz).
struct GemmBatch {
  long a_off, y_off, z_off;
  int R, C, K, ldy, ldz;
  int r0, RB;            // rows r0 .. r0 + RB of the operator handled by this batch
  int CB;                // contraction chunk staged in shared memory (C: operator resident)
  int TK;                // thread columns; the input tile is TK * Z_KB columns of CB entries
};
// One CTA per batch: the operator (R x C, input-major) stays in shared
// memory; columns stream through in tiles of TK*KB.  Thread (tr, tk) owns rows
// tr + TR*i (i < RPT) and columns tk + TK*j (j < KB).
#define Z_RPT 3                    // tiling::kRpt
#define Z_KB 4                     // tiling::kKb
static_assert(Z_RPT == tiling::kRpt && Z_KB == tiling::kKb, "tiling constants");
__global__ void __launch_bounds__(128) k_zgemm_res(const GemmBatch* __restrict__ batches, const cplx* __restrict__ A,
                                                   const cplx* __restrict__ Y, cplx* __restrict__ Z) {
  const GemmBatch bt = batches[blockIdx.x];
  const int R = bt.RB, Cc = bt.C, K = bt.K, CB = bt.CB;   // R: rows of this block, CB: contraction chunk
  const int TR = (R + Z_RPT - 1) / Z_RPT;
  const int TK = bt.TK;                                    // TR * TK <= 128, chosen by the host
  const int KT = TK * Z_KB;
  extern __shared__ cplx sm[];
  cplx* As = sm;                      // [CB][RB]
  cplx* Ys = As + (size_t)R * CB;     // [KT][CB]
  const cplx* Ab = A + bt.a_off;
  const int tr = threadIdx.x % TR, tk = threadIdx.x / TR;
  const bool act = tk < TK;
  const cplx* Yb = Y + bt.y_off;
  cplx* Zb = Z + bt.z_off;
  int rows[Z_RPT];
#pragma unroll
  for (int i = 0; i < Z_RPT; ++i) rows[i] = min(tr + TR * i, R - 1);
  for (int k0 = 0; k0 < K; k0 += KT) {
    cplx acc[Z_RPT][Z_KB];
#pragma unroll
    for (int i = 0; i < Z_RPT; ++i)
#pragma unroll
      for (int j = 0; j < Z_KB; ++j) acc[i][j] = C(0, 0);
    for (int c0 = 0; c0 < Cc; c0 += CB) {
      const int cb = min(CB, Cc - c0);
      __syncthreads();
      if (k0 == 0 || CB < Cc)         // a resident operator is staged once
        for (int e = threadIdx.x; e < R * cb; e += blockDim.x) {
          int c = e / R, rr = e % R;
          As[e] = Ab[(long)(c0 + c) * bt.R + bt.r0 + rr];
        }
      for (int e = threadIdx.x; e < KT * cb; e += blockDim.x) {
        int kk = e / cb, c = e % cb;
        int k = k0 + kk;
        Ys[e] = (k < K) ? Yb[(long)k * bt.ldy + c0 + c] : C(0, 0);
      }
      __syncthreads();
      if (act) {
#pragma unroll 2
        for (int c = 0; c < cb; ++c) {
          cplx a[Z_RPT], y[Z_KB];
#pragma unroll
          for (int i = 0; i < Z_RPT; ++i) a[i] = As[c * R + rows[i]];
#pragma unroll
          for (int j = 0; j < Z_KB; ++j) y[j] = Ys[(tk + TK * j) * cb + c];
#pragma unroll
          for (int i = 0; i < Z_RPT; ++i)
#pragma unroll
            for (int j = 0; j < Z_KB; ++j) cfma(acc[i][j], a[i], y[j]);
        }
      }
    }
    if (act) {
#pragma unroll
      for (int i = 0; i < Z_RPT; ++i)
#pragma unroll
        for (int j = 0; j < Z_KB; ++j) {
          int r = tr + TR * i, k = k0 + tk + TK * j;
          if (r < R && k < K) Zb[(long)k * bt.ldz + bt.r0 + r] = acc[i][j];
        }
    }
  }
}

// L_T = sum over V(T) of the translated columns.  Free space: in list order.
// Reaction: the way back from the symmetric basis and the rotation by
// e^{-im phi} are linear and depend on the pair only through its horizontal
// offset (phi), so the columns are first summed per offset (offsets in
// increasing index, list order within one), and each offset's sum is
// transformed once.  One CTA per target box; deterministic.
#define REDUCE_MAXV 512
__global__ void k_m2l_reduce(int p, const int* __restrict__ boxes, BoxGeom B, OpIndex OI,
                             const int* __restrict__ voff, const int* __restrict__ vidx,
                             const int* __restrict__ inv, const cplx* __restrict__ Z, cplx* __restrict__ L) {
  const int T = boxes[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  const int comp = B.comp[T];
  const bool reac = OI.cgs[comp].kind == CK_REAC;
  const int np = (p + 1) * (p + 2) / 2;
  const double r = 0.70710678118654752440;
  const int* ct = B.coord + 3 * T;
  const int e0 = voff[T], nvl = voff[T + 1] - e0;
  __shared__ int phi_of[REDUCE_MAXV], order[REDUCE_MAXV], start[50];
  const bool grouped = reac && nvl <= REDUCE_MAXV;
  if (grouped) {
    for (int j = threadIdx.x; j < nvl; j += blockDim.x) {
      const int* cs = B.coord + 3 * vidx[e0 + j];
      phi_of[j] = (ct[1] - cs[1] + 3) * 7 + (ct[0] - cs[0] + 3);
    }
    __syncthreads();
    if (threadIdx.x == 0) {                     // stable counting sort by offset
      for (int f = 0; f < 50; ++f) start[f] = 0;
      for (int j = 0; j < nvl; ++j) ++start[phi_of[j] + 1];
      for (int f = 0; f < 49; ++f) start[f + 1] += start[f];
      int fill[49];
      for (int f = 0; f < 49; ++f) fill[f] = start[f];
      for (int j = 0; j < nvl; ++j) order[fill[phi_of[j]]++] = j;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    int n = (int)floor(sqrt((double)i));
    while ((n + 1) * (n + 1) <= i) ++n;
    while (n * n > i) --n;
    int m = i - n * n - n, am = m < 0 ? -m : m;
    int ip = n * (n + 1) / 2 + am, im = am ? np + n * (n - 1) / 2 + am - 1 : 0;
    double sg = (m < 0 && (am & 1)) ? -1.0 : 1.0;
    cplx acc = C(0, 0);
    if (!reac) {
      for (int e = e0; e < e0 + nvl; ++e) acc = cadd(acc, Z[(long)inv[e] * P + i]);
    } else if (grouped) {
      for (int f = 0; f < 49; ++f) {
        if (start[f + 1] == start[f]) continue;
        cplx zp = C(0, 0), zm = C(0, 0);
        for (int j = start[f]; j < start[f + 1]; ++j) {
          const cplx* z = Z + (long)inv[e0 + order[j]] * P;
          zp = cadd(zp, z[ip]);
          if (m != 0) zm = cadd(zm, z[im]);
        }
        cplx v;
        if (m == 0) v = zp;
        else if (m > 0) v = cscale(cadd(zp, zm), r);
        else v = cscale(csub(zp, zm), r * sg);
        const cplx* ph = OI.phase + f * (2 * p + 1) + p;
        acc = cadd(acc, cmul(v, cconj(ph[m])));
      }
    } else {
      for (int e = e0; e < e0 + nvl; ++e) {
        const cplx* z = Z + (long)inv[e] * P;
        cplx v;
        if (m == 0) v = z[ip];
        else if (m > 0) v = cscale(cadd(z[ip], z[im]), r);
        else v = cscale(csub(z[ip], z[im]), r * sg);
        const int* cs = B.coord + 3 * vidx[e];
        const cplx* ph = OI.phase + ((ct[1] - cs[1] + 3) * 7 + (ct[0] - cs[0] + 3)) * (2 * p + 1) + p;
        acc = cadd(acc, cmul(v, cconj(ph[m])));
      }
    }
    L[(long)T * P + i] = acc;
  }
}

// L_T += L2L(L_parent) for the boxes of one level (>= 3).
__global__ void k_l2l(int p, const int* __restrict__ boxes, BoxGeom B, OpIndex OI, const cplx* __restrict__ l2l_ops,
                      cplx* __restrict__ L) {
  const int T = boxes[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  extern __shared__ cplx xs[];
  const int pa = B.parent[T];
  for (int i = threadIdx.x; i < P; i += blockDim.x) xs[i] = L[(long)pa * P + i];
  __syncthreads();
  const int* ct = B.coord + 3 * T;
  int oct = (ct[0] & 1) | ((ct[1] & 1) << 1) | ((ct[2] & 1) << 2);
  const cplx* op = l2l_ops + OI.l2l_base[B.comp[T] * 23 + B.lev[T]] + (long)oct * P * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    cplx a = L[(long)T * P + i];
    for (int j = 0; j < P; ++j) cfma(a, op[(long)j * P + i], xs[j]);
    L[(long)T * P + i] = a;
  }
}

__global__ void k_inverse_perm(long n, const int* __restrict__ perm, int* __restrict__ inv) {
  long k = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (k < n) inv[perm[k]] = (int)k;
}

using tiling::gemm_smem;
using tiling::gemm_smem_max;
using tiling::gemm_tiles;
using tiling::gemm_tk;
static_assert(sizeof(cplx) == tiling::kCplx, "complex layout");

void run_m2l_tc(fmm_layered* h, long nv, int nruns, const std::vector<unsigned long long>& hk,
                const std::vector<int>& hc, const int* perm, const int* owner, const int* vidx, BoxGeom B,
                OpIndex OI, const std::vector<CompGeom>& cgh, const cplx* free_ops, const cplx* reac_ops,
                const cplx* M, cplx* Z, int* err, cudaStream_t st, cudaEvent_t gemm0, cudaEvent_t gemm1,
                double* gemm_flops);

void run_m2l_rot(fmm_layered* h, const std::vector<int>& runs, const std::vector<long>& col0,
                 const std::vector<int>& cnt, const int* d_rs, int nruns, const int* perm, const int* owner,
                 const int* vidx, BoxGeom B, const std::vector<CompGeom>& cgh, const cplx* Y, cplx* Z,
                 double* macs, cudaEvent_t ev_start, cudaStream_t st);

void launch_l2l_rot(fmm_layered* h, const int* boxes, int n, BoxGeom B, const long* az_tab, cplx* L, cudaStream_t st);

// Host driver: all V pairs of all levels.  L receives the M2L part for every
// box with targets at level >= 2; then L2L level by level.
void run_m2l_gemm(fmm_layered* h, int nb, long nv, const std::vector<std::vector<int>>& m2l_lvl,
                  const int* dsched, const std::vector<long>& o_m2l, int maxlev, BoxGeom B, OpIndex OI,
                  const int* voff, const int* vidx, const cplx* free_ops, const cplx* reac_ops,
                  const cplx* l2l_ops, const cplx* M, cplx* L, int* err, cudaStream_t st,
                  cudaEvent_t gemm0, cudaEvent_t gemm1, double* gemm_flops, const std::vector<CompGeom>& cgh,
                  const long* l2l_rot_tab) {
  Workspace& ws = h->W();
  const int p = h->p, P = (p + 1) * (p + 1);
  const int np = (p + 1) * (p + 2) / 2, nm = p * (p + 1) / 2;
  if (nv > 0) {
    ws.g_owner.ensure(4 * nv);
    ws.g_keys.ensure(8 * nv * 2);
    ws.g_vals.ensure(4 * nv * 2);
    ws.g_inv.ensure(4 * nv);
    const bool mixed = (h->flags & FMM_MIXED) != 0;
    if (!mixed) ws.g_Y.ensure(sizeof(cplx) * (size_t)nv * P);
    ws.g_Z.ensure(sizeof(cplx) * (size_t)nv * P);
    int* owner = ws.g_owner.as<int>();
    unsigned long long* keys = ws.g_keys.as<unsigned long long>();
    unsigned long long* keys2 = keys + nv;
    int* vals = ws.g_vals.as<int>();
    int* perm = vals + nv;
    int* inv = ws.g_inv.as<int>();
    LAUNCH(k_v_owner<<<(nb + 127) / 128, 128, 0, st>>>(nb, voff, owner));
    LAUNCH(k_v_keys<<<(nv + 255) / 256, 256, 0, st>>>(nv, owner, vidx, B, OI, P, keys, vals, err));
    // stable sort by operator key (keys and vals are overwritten)
    dev_sort_pairs(keys, vals, keys2, perm, nv, 0, 64, ws.sort_tmp, st);
    LAUNCH(k_inverse_perm<<<(nv + 255) / 256, 256, 0, st>>>(nv, perm, inv));
    // run-length encode the sorted keys
    ws.g_runs.ensure((8 + 4) * (size_t)nv + 64);
    unsigned long long* ukeys = ws.g_runs.as<unsigned long long>();
    int* counts = (int*)(ukeys + nv);
    int* nruns_d = (int*)(counts + nv);
    dev_run_length(keys2, nv, ukeys, counts, nruns_d, ws.sort_tmp, st);
    int nruns = 0;
    FMM_CHECK(cudaMemcpyAsync(&nruns, nruns_d, 4, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaStreamSynchronize(st));
    std::vector<unsigned long long> hk(nruns);
    std::vector<int> hc(nruns);
    FMM_CHECK(cudaMemcpyAsync(hk.data(), ukeys, 8 * (size_t)nruns, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaMemcpyAsync(hc.data(), counts, 4 * (size_t)nruns, cudaMemcpyDeviceToHost, st));
    if (mixed) {
      FMM_CHECK(cudaStreamSynchronize(st));
      run_m2l_tc(h, nv, nruns, hk, hc, perm, owner, vidx, B, OI, cgh, free_ops, reac_ops, M, ws.g_Z.as<cplx>(),
                 err, st, gemm0, gemm1, gemm_flops);
    } else {
    // gather the columns
    LAUNCH(k_m2l_gather<<<(unsigned)((nv * P + 255) / 256), 256, 0, st>>>(nv, p, perm, owner, vidx, B, OI, M,
                                                                          ws.g_Y.as<cplx>()));
    FMM_CHECK(cudaStreamSynchronize(st));
    // batches and tiles
    std::vector<GemmBatch> bfree, breac;
    long k0 = 0;
    double macs = 0.0;       // complex multiply-adds of the translations (operator entries x columns)
    // free-space classes in rotation form from p = 5 on (2.7x fewer products at p = 8)
    const bool use_rot = p >= 5;
    std::vector<int> rot_runs, rot_cnt;
    std::vector<long> rot_col0;
    for (int r = 0; r < nruns; ++r) {
      long off = (long)(hk[r] >> 1);
      bool reac = hk[r] & 1;
      int K = hc[r];
      // one batch per operator block, split into chunks of at most 128
      // columns so that large classes spread over several CTAs
      // free-space and reaction operators live in different buffers: the
      // batch offsets index the buffer of their kind (free batches launch first)
      std::vector<GemmBatch>& dst = reac ? breac : bfree;
      auto add = [&](long a_off, int R, long yz) {
        int RB, CB;
        gemm_tiles(R, RB, CB);
        for (int r0 = 0; r0 < R; r0 += RB) {
          const int rb = std::min(RB, R - r0), tk = gemm_tk(rb, CB);
          // column chunks of about 128, a whole number of column tiles (tk * Z_KB)
          const int kt = tk * Z_KB, chunk = std::max(kt, (128 / kt) * kt);
          for (int c0 = 0; c0 < K; c0 += chunk) {
            GemmBatch g{};
            g.a_off = a_off; g.R = R; g.C = R; g.K = std::min(chunk, K - c0);
            g.y_off = (k0 + c0) * P + yz; g.z_off = (k0 + c0) * P + yz; g.ldy = P; g.ldz = P;
            g.r0 = r0; g.RB = rb; g.CB = CB; g.TK = tk;
            dst.push_back(g);
          }
        }
      };
      if (!reac && use_rot) {
        rot_runs.push_back(r);
        rot_col0.push_back(k0);
        rot_cnt.push_back(K);
      } else if (!reac) {
        add(off, P, 0);
        macs += (double)K * P * P;
      } else {
        add(off, np, 0);
        if (nm) add(off + (long)np * np, nm, np);
        macs += (double)K * ((double)np * np + (double)nm * nm);
      }
      k0 += K;
    }
    ws.g_bat.ensure(sizeof(GemmBatch) * (bfree.size() + breac.size()) + 64);
    GemmBatch* dbat = ws.g_bat.as<GemmBatch>();
    std::vector<GemmBatch> ordered = bfree;
    ordered.insert(ordered.end(), breac.begin(), breac.end());
    FMM_CHECK(cudaMemcpyAsync(dbat, ordered.data(), sizeof(GemmBatch) * ordered.size(), cudaMemcpyHostToDevice, st));
    auto smem_of = [&](int R) { return gemm_smem_max(R); };
    size_t smax = std::max(smem_of(P), std::max(smem_of(np), nm ? smem_of(nm) : (size_t)0));
    FMM_CHECK(cudaFuncSetAttribute(k_zgemm_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
    if (!rot_runs.empty()) {
      std::vector<int> rs(nruns + 1, 0);
      for (int r = 0; r < nruns; ++r) rs[r + 1] = rs[r] + hc[r];
      int* d_rs = (int*)tc_need(ws.rot_rs, sizeof(int) * rs.size() + 64);
      FMM_CHECK(cudaMemcpyAsync(d_rs, rs.data(), sizeof(int) * rs.size(), cudaMemcpyHostToDevice, st));
      run_m2l_rot(h, rot_runs, rot_col0, rot_cnt, d_rs, nruns, perm, owner, vidx, B, cgh, ws.g_Y.as<cplx>(),
                  ws.g_Z.as<cplx>(), &macs, gemm0, st);
    } else {
      FMM_CHECK(cudaEventRecord(gemm0, st));
    }
    *gemm_flops = 8.0 * macs;
    if (!bfree.empty())
      LAUNCH(k_zgemm_res<<<(unsigned)bfree.size(), 128, smem_of(P), st>>>(dbat, free_ops, ws.g_Y.as<cplx>(),
                                                                          ws.g_Z.as<cplx>()));
    if (!breac.empty())
      LAUNCH(k_zgemm_res<<<(unsigned)breac.size(), 128, std::max(smem_of(np), nm ? smem_of(nm) : (size_t)0), st>>>(
          dbat + bfree.size(), reac_ops, ws.g_Y.as<cplx>(), ws.g_Z.as<cplx>()));
    FMM_CHECK(cudaEventRecord(gemm1, st));
    FMM_CHECK(cudaGetLastError());
    }
    // per-target sums (all levels)
    for (int l = 2; l <= maxlev; ++l)
      if (!m2l_lvl[l].empty())
        LAUNCH(k_m2l_reduce<<<(unsigned)m2l_lvl[l].size(), 128, 0, st>>>(p, dsched + o_m2l[l], B, OI, voff, vidx, inv,
                                                                        ws.g_Z.as<cplx>(), L));
    FMM_CHECK(cudaStreamSynchronize(st));   // host vectors above go out of scope
  } else {
    FMM_CHECK(cudaMemsetAsync(L, 0, sizeof(cplx) * (size_t)nb * P, st));
  }
  // L2L, top down
  for (int l = 3; l <= maxlev; ++l) {
    if (m2l_lvl[l].empty()) continue;
    if (l2l_rot_tab) launch_l2l_rot(h, dsched + o_m2l[l], (int)m2l_lvl[l].size(), B, l2l_rot_tab, L, st);
    else LAUNCH(k_l2l<<<(unsigned)m2l_lvl[l].size(), 128, sizeof(cplx) * P, st>>>(p, dsched + o_m2l[l], B, OI, l2l_ops, L));
  }
  FMM_CHECK(cudaGetLastError());
  (void)np;
}

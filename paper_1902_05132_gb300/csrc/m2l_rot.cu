// Free-space M2L in rotation form (O(p^3) per translation).
//
// The free-space translation L = A(b) M of Thm. 2.3 / eq. metole for a centre
// offset b factors through a rotation Q that takes b to |b| z:
//     A(b) = W^T A(|b| z) conj(W),
// where W is block diagonal in the degree n with
//     Y_n^m(Q x) = sum_m' W[(n,m),(n,m')] Y_n^m'(x)        (|x| = 1),
// and the coaxial operator A(|b| z) couples only equal orders m (the
// harmonic Y_q^{mu-m} of the Gaunt formula vanishes on the z axis unless
// mu = m).  Per translation this costs 2 sum_n (2n+1)^2 + sum_m (p+1-|m|)^2
// complex multiply-adds instead of (p+1)^4 (2,427 instead of 6,561 at p = 8).
// W is computed once per handle for the 343 offset directions of the V
// lists by a product quadrature on the sphere (Gauss-Legendre in cos theta,
// equispaced in phi), exact for these polynomials; A(|b| z) comes from the
// same Gaunt-formula kernel as the dense operators and is cached per
// (k, box width, |offset|^2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "fmm_internal.h"
#include "tiling.h"

void launch_sep_ops(int p, const SepJob* jobs, int njobs, const double* G, cplx* ops, cudaStream_t st);

namespace {

using tiling::rot_naz;
using tiling::rot_nw;
__host__ __device__ inline int rot_ob(int n) { return n * (2 * n - 1) * (2 * n + 1) / 3; }   // start of block n
// start of the order-m block of the compact coaxial operator (m = -p..p)
__host__ __device__ inline int rot_om(int p, int m) {
  int o = 0;
  for (int j = -p; j < m; ++j) o += (p + 1 - abs(j)) * (p + 1 - abs(j));
  return o;
}
__device__ inline int deg_full(int i) {
  int n = (int)sqrtf((float)i);
  while ((n + 1) * (n + 1) <= i) ++n;
  while (n * n > i) --n;
  return n;
}

// Y_n^m at the quadrature points, plain (slot -1, stored last) and rotated by
// the Q of every direction slot: Ybuf[(slot or 343)][pt][(n,m)].
__global__ void k_rot_y(int p, int npt, int nphi, const double* __restrict__ xg, cplx* __restrict__ Ybuf) {
  const int slot = blockIdx.y;                 // 0..342 directions, 343: unrotated
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npt) return;
  const int P = (p + 1) * (p + 1);
  const double ct0 = xg[pt / nphi], st0 = sqrt(fmax(0.0, 1.0 - ct0 * ct0));
  const double ph0 = 2.0 * FMM_PI * (pt % nphi) / nphi;
  double x[3] = {st0 * cos(ph0), st0 * sin(ph0), ct0};
  if (slot < 343) {
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    double r = sqrt((double)(dx * dx + dy * dy + dz * dz));
    if (r > 0) {
      // Q = R_y(-theta) R_z(-phi) maps the direction (theta, phi) to +z
      double th = acos(fmin(1.0, fmax(-1.0, dz / r))), ph = atan2((double)dy, (double)dx);
      double cp = cos(ph), sp = sin(ph), cth = cos(th), sth = sin(th);
      double a0 = cp * x[0] + sp * x[1], a1 = -sp * x[0] + cp * x[1], a2 = x[2];
      x[0] = cth * a0 - sth * a2;
      x[1] = a1;
      x[2] = sth * a0 + cth * a2;
    }
  }
  double ct = fmin(1.0, fmax(-1.0, x[2]));
  double st = sqrt(x[0] * x[0] + x[1] * x[1]);
  double phi = atan2(x[1], x[0]);
  double Pa[(FMM_MAXP + 1) * (FMM_MAXP + 2) / 2];
  phat_real(p, ct, st, Pa);
  cplx* Y = Ybuf + ((long)slot * npt + pt) * P;
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m) {
      int am = abs(m);
      double v = Pa[n * (n + 1) / 2 + am] * ((m < 0 && (am & 1)) ? -1.0 : 1.0);
      double s, c;
      sincos(m * phi, &s, &c);
      Y[n * n + n + m] = C(v * c, v * s);
    }
}

// W of every slot: W[slot][ob(n) + (m+n)(2n+1) + (m'+n)] = sum_pt w_pt Y_n^m(Q x_pt) conj(Y_n^m'(x_pt))
__global__ void k_rot_w(int p, int npt, const double* __restrict__ wpt, const cplx* __restrict__ Ybuf,
                        cplx* __restrict__ Wall) {
  const int slot = blockIdx.x;
  const int P = (p + 1) * (p + 1);
  const long NW = rot_nw(p);
  const cplx* Yq = Ybuf + (long)slot * npt * P;
  const cplx* Yx = Ybuf + (long)343 * npt * P;
  for (long e = threadIdx.x; e < NW; e += blockDim.x) {
    int n = 0;
    while (rot_ob(n + 1) <= e) ++n;
    const int loc = (int)(e - rot_ob(n)), w2 = 2 * n + 1;
    const int m = loc / w2 - n, mp = loc % w2 - n;
    cplx acc = C(0, 0);
    for (int q = 0; q < npt; ++q) cfma(acc, cscale(Yq[(long)q * P + n * n + n + m], wpt[q]), cconj(Yx[(long)q * P + n * n + n + mp]));
    Wall[(long)slot * NW + e] = acc;
  }
}

// operator slot of each run: direction index of its first pair's offset
__global__ void k_run_slot(int nruns, const int* __restrict__ rs, const int* __restrict__ perm,
                           const int* __restrict__ owner, const int* __restrict__ vidx, BoxGeom B,
                           int* __restrict__ out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nruns) return;
  int e = perm[rs[r]];
  int T = owner[e], S = vidx[e];
  const int* ct = B.coord + 3 * T;
  const int* cs = B.coord + 3 * S;
  int dx = ct[0] - cs[0], dy = ct[1] - cs[1], dz = ct[2] - cs[2];
  out[3 * r] = ((dz + 3) * 7 + (dy + 3)) * 7 + (dx + 3);
  out[3 * r + 1] = B.comp[T];
  out[3 * r + 2] = B.lev[T];
}

}  // namespace

struct RotBatch {
  long col0;         // translated-column index of the first pair
  long az_off;       // dense coaxial operator (input-major, P x P)
  int K;             // pairs in this batch (<= the kernel's column tile)
  int slot;          // direction slot (W)
};

// Z[col] = W^T A_z conj(W) Y[col] for the columns of one batch (one CTA).
__global__ void __launch_bounds__(256) k_zrot(int p, int KC, const RotBatch* __restrict__ batches,
                                              const cplx* __restrict__ Wall, const cplx* __restrict__ az_ops,
                                              const cplx* __restrict__ Y, cplx* __restrict__ Z) {
  const RotBatch bt = batches[blockIdx.x];
  const int P = (p + 1) * (p + 1);
  const int NW = (int)rot_nw(p), NAZ = rot_naz(p);
  extern __shared__ cplx sm[];
  cplx* Wc = sm;                  // [NW]
  cplx* Az = Wc + NW;             // [NAZ] compact, order-m blocks of (p+1-|m|)^2, row = output degree
  cplx* T0 = Az + NAZ;            // [KC][P]
  cplx* T1 = T0 + (size_t)KC * P; // [KC][P]
  __shared__ int om[2 * FMM_MAXP + 1];
  for (int m = threadIdx.x - p; m <= p; m += blockDim.x) om[m + p] = rot_om(p, m);
  const cplx* Wg = Wall + (long)bt.slot * NW;
  for (int e = threadIdx.x; e < NW; e += blockDim.x) Wc[e] = Wg[e];
  const cplx* A = az_ops + bt.az_off;
  __syncthreads();
  for (int m = -p; m <= p; ++m) {
    const int am = abs(m), nb = p + 1 - am, o = om[m + p];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int n = am + e / nb, np_ = am + e % nb;                 // output n, input n'
      Az[o + e] = A[(long)(np_ * np_ + np_ + m) * P + (n * n + n + m)];
    }
  }
  for (int e = threadIdx.x; e < bt.K * P; e += blockDim.x) T0[e] = Y[(bt.col0 + e / P) * (long)P + e % P];
  __syncthreads();
  // conj(W): rotate the multipole expansion into the frame of the offset
  for (int e = threadIdx.x; e < bt.K * P; e += blockDim.x) {
    const int k = e / P, i = e % P, n = deg_full(i), m = i - n * n - n, w2 = 2 * n + 1;
    const cplx* wr = Wc + rot_ob(n) + (m + n) * w2;
    const cplx* x = T0 + k * P + n * n;
    cplx acc = C(0, 0);
    for (int j = 0; j < w2; ++j) cfma(acc, cconj(wr[j]), x[j]);
    T1[e] = acc;
  }
  __syncthreads();
  // coaxial translation, order by order
  for (int e = threadIdx.x; e < bt.K * P; e += blockDim.x) {
    const int k = e / P, i = e % P, n = deg_full(i), m = i - n * n - n, am = abs(m), nb = p + 1 - am;
    const cplx* ar = Az + om[m + p] + (n - am) * nb;
    const cplx* x = T1 + k * P;
    cplx acc = C(0, 0);
    for (int j = 0; j < nb; ++j) {
      const int np_ = am + j;
      cfma(acc, ar[j], x[np_ * np_ + np_ + m]);
    }
    T0[e] = acc;
  }
  __syncthreads();
  // W^T: back to the original frame
  for (int e = threadIdx.x; e < bt.K * P; e += blockDim.x) {
    const int k = e / P, i = e % P, n = deg_full(i), m = i - n * n - n, w2 = 2 * n + 1;
    const cplx* wc = Wc + rot_ob(n) + (m + n);
    const cplx* x = T0 + k * P + n * n;
    cplx acc = C(0, 0);
    for (int j = 0; j < w2; ++j) cfma(acc, wc[j * w2], x[j]);
    Z[(bt.col0 + k) * (long)P + i] = acc;
  }
}

// W tables of the handle (once).
static void rot_tables(fmm_layered* h, cudaStream_t st) {
  RotCache& R = h->rot;
  if (R.ready) return;
  const int p = h->p, P = (p + 1) * (p + 1);
  std::vector<double> xg, wg;
  gauss_legendre_pub(p + 2, xg, wg);
  const int nphi = 2 * p + 2, npt = (p + 2) * nphi;
  std::vector<double> wpt(npt);
  for (int i = 0; i < npt; ++i) wpt[i] = wg[i / nphi] * 2.0 * FMM_PI / nphi;
  DevBuf dx, dw, ybuf;
  dx.ensure(sizeof(double) * xg.size());
  dw.ensure(sizeof(double) * npt);
  ybuf.ensure(sizeof(cplx) * (size_t)344 * npt * P);
  FMM_CHECK(cudaMemcpyAsync(dx.ptr, xg.data(), sizeof(double) * xg.size(), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(dw.ptr, wpt.data(), sizeof(double) * npt, cudaMemcpyHostToDevice, st));
  R.w.ensure(sizeof(cplx) * (size_t)343 * rot_nw(p));
  LAUNCH(k_rot_y<<<dim3((npt + 63) / 64, 344), 64, 0, st>>>(p, npt, nphi, dx.as<double>(), ybuf.as<cplx>()));
  LAUNCH(k_rot_w<<<343, 128, 0, st>>>(p, npt, dw.as<double>(), ybuf.as<cplx>(), R.w.as<cplx>()));
  FMM_CHECK(cudaGetLastError());
  FMM_CHECK(cudaStreamSynchronize(st));      // the temporary buffers are freed on return
  R.ready = true;
}

static uint64_t rbits(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}

// Free-space runs of the sorted V pairs through the rotation form: Z for
// every pair of the runs listed (run index r, its first column and count).
void run_m2l_rot(fmm_layered* h, const std::vector<int>& runs, const std::vector<long>& col0,
                 const std::vector<int>& cnt, const int* d_rs, int nruns, const int* perm, const int* owner,
                 const int* vidx, BoxGeom B, const std::vector<CompGeom>& cgh, const cplx* Y, cplx* Z,
                 double* macs, cudaEvent_t ev_start, cudaStream_t st) {
  if (runs.empty()) {
    FMM_CHECK(cudaEventRecord(ev_start, st));
    return;
  }
  Workspace& ws = h->W();
  RotCache& R = h->rot;
  const int p = h->p, P = (p + 1) * (p + 1);
  rot_tables(h, st);
  // slot, component and level of every run
  int* d_info = (int*)tc_need(ws.rot_info, sizeof(int) * 3 * (size_t)nruns + 64);
  LAUNCH(k_run_slot<<<(nruns + 127) / 128, 128, 0, st>>>(nruns, d_rs, perm, owner, vidx, B, d_info));
  std::vector<int> info(3 * (size_t)nruns);
  FMM_CHECK(cudaMemcpyAsync(info.data(), d_info, sizeof(int) * info.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  // coaxial operators (k, w, |d|^2), built on first use
  std::vector<SepJob> jobs;
  auto az_of = [&](int comp, int lev, int slot) -> long {
    const double k = cgh[comp].kt, w = cgh[comp].h2 / (double)(1 << lev);
    const int dx = slot % 7 - 3, dy = (slot / 7) % 7 - 3, dz = slot / 49 - 3;
    const int d2 = dx * dx + dy * dy + dz * dz;
    auto key = std::make_tuple(rbits(k), rbits(w), d2);
    auto it = R.az.find(key);
    if (it != R.az.end()) return it->second;
    long off = R.az_used;
    R.az_used += (long)P * P;
    R.az[key] = off;
    SepJob j{};
    j.b[0] = 0.0;
    j.b[1] = 0.0;
    j.b[2] = std::sqrt((double)d2) * w;
    j.k = k;
    j.kind = 0;
    j.out_off = off;
    jobs.push_back(j);
    return off;
  };
  const int NW = (int)rot_nw(p), NAZ = rot_naz(p);
  std::vector<long> run_az(runs.size());
  std::vector<int> run_slot(runs.size());
  for (size_t i = 0; i < runs.size(); ++i) {
    const int r = runs[i];
    run_slot[i] = info[3 * r];
    run_az[i] = az_of(info[3 * r + 1], info[3 * r + 2], run_slot[i]);
    *macs += (double)cnt[i] * (2.0 * NW + NAZ);
  }
  // batches of at most KC columns of one run
  auto make_batches = [&](int KC, std::vector<RotBatch>& bat) {
    bat.clear();
    for (size_t i = 0; i < runs.size(); ++i)
      for (int c0 = 0; c0 < cnt[i]; c0 += KC) {
        RotBatch b{};
        b.col0 = col0[i] + c0;
        b.az_off = run_az[i];
        b.K = std::min(KC, cnt[i] - c0);
        b.slot = run_slot[i];
        bat.push_back(b);
      }
  };
  std::vector<RotBatch> bat;
  if (!jobs.empty()) {
    R.az_buf.grow_keep(sizeof(cplx) * (size_t)R.az_used, sizeof(cplx) * (size_t)(R.az_used - (long)jobs.size() * P * P),
                       st);
    SepJob* dj = (SepJob*)tc_need(ws.rot_jobs, sizeof(SepJob) * jobs.size() + 64);
    FMM_CHECK(cudaMemcpyAsync(dj, jobs.data(), sizeof(SepJob) * jobs.size(), cudaMemcpyHostToDevice, st));
    launch_sep_ops(p, dj, (int)jobs.size(), h->tab.gaunt.as<double>(), R.az_buf.as<cplx>(), st);
    FMM_CHECK(cudaGetLastError());
  }
  // launch with column tile KC and `thr` threads per CTA
  auto launch = [&](int KC, int thr) {
    make_batches(KC, bat);
    RotBatch* db = (RotBatch*)tc_need(ws.rot_bat, sizeof(RotBatch) * bat.size() + 64);
    FMM_CHECK(cudaMemcpyAsync(db, bat.data(), sizeof(RotBatch) * bat.size(), cudaMemcpyHostToDevice, st));
    const size_t smem = tiling::rot_smem_kc(p, KC);
    FMM_CHECK(cudaFuncSetAttribute(k_zrot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return db;
  };
  TuneState& T = h->tune;
  if (!T.zrot_done) {
    // autotuner: time every candidate tile on this evaluation's own batches
    // (every candidate computes the same columns, so Z is final either way)
    // and keep the fastest for the handle; the choice goes to the statistics
    int kc[16], thr[16];
    const int nc = tiling::rot_tune_candidates(p, kc, thr, 16);
    cudaEvent_t a, b;
    FMM_CHECK(cudaEventCreate(&a));
    FMM_CHECK(cudaEventCreate(&b));
    float best = INFINITY;
    T.zrot_trials.clear();
    for (int i = 0; i < nc; ++i) {
      RotBatch* db = launch(kc[i], thr[i]);
      FMM_CHECK(cudaEventRecord(a, st));
      const size_t smem = tiling::rot_smem_kc(p, kc[i]);
      LAUNCH(k_zrot<<<(unsigned)bat.size(), thr[i], smem, st>>>(p, kc[i], db, R.w.as<cplx>(), R.az_buf.as<cplx>(), Y, Z));
      FMM_CHECK(cudaGetLastError());
      FMM_CHECK(cudaEventRecord(b, st));
      FMM_CHECK(cudaEventSynchronize(b));
      float ms = 0;
      FMM_CHECK(cudaEventElapsedTime(&ms, a, b));
      T.zrot_trials.push_back(ms);
      if (kc[i] == tiling::rot_kc(p) && thr[i] == 128) T.zrot_rule_ms = ms;
      if (ms < best) { best = ms; T.zrot_kc = kc[i]; T.zrot_threads = thr[i]; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    T.zrot_ms = best;
    T.zrot_done = true;
  }
  const int KC = T.zrot_kc, THR = T.zrot_threads;
  RotBatch* db = launch(KC, THR);
  FMM_CHECK(cudaEventRecord(ev_start, st));   // the translation launches start here
  LAUNCH(k_zrot<<<(unsigned)bat.size(), THR, tiling::rot_smem_kc(p, KC), st>>>(p, KC, db, R.w.as<cplx>(),
                                                                             R.az_buf.as<cplx>(), Y, Z));
  FMM_CHECK(cudaGetLastError());
}

// ---------------------------------------------------------------- M2M and L2L in rotation form
// The shifts between a box and its children factor the same way: with b the
// child-minus-parent centre offset (direction (+-1, +-1, +-1)), M2M
// conj(S^(b)) and L2L S^(b)^T equal W^T [operator at |b| z] conj(W), both
// kinds of coefficients turning by conj(W) under the rotation.

// one direction stage: out[i] = sum_j Wr(i, j) x[(n(i), j)] over the block of n(i)
__device__ inline void rot_stage(int P, const cplx* Wc, const cplx* x, cplx* out, bool conj_rows, bool accumulate) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int n = deg_full(i), m = i - n * n - n, w2 = 2 * n + 1;
    const cplx* xb = x + n * n;
    cplx acc = accumulate ? out[i] : C(0, 0);
    if (conj_rows) {
      const cplx* wr = Wc + rot_ob(n) + (m + n) * w2;       // row (n, m) of conj(W)
      for (int j = 0; j < w2; ++j) cfma(acc, cconj(wr[j]), xb[j]);
    } else {
      const cplx* wc = Wc + rot_ob(n) + (m + n);             // column (n, m) of W: W^T row
      for (int j = 0; j < w2; ++j) cfma(acc, wc[j * w2], xb[j]);
    }
    out[i] = acc;
  }
}
__device__ inline void coax_stage(int p, int P, const cplx* Az, const int* om, const cplx* x, cplx* out) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int n = deg_full(i), m = i - n * n - n, am = abs(m), nb = p + 1 - am;
    const cplx* ar = Az + om[m + p] + (n - am) * nb;
    cplx acc = C(0, 0);
    for (int j = 0; j < nb; ++j) {
      const int np_ = am + j;
      cfma(acc, ar[j], x[np_ * np_ + np_ + m]);
    }
    out[i] = acc;
  }
}
__device__ inline void load_coax(int p, int P, const cplx* A, const int* om, cplx* Az) {
  for (int m = -p; m <= p; ++m) {
    const int am = abs(m), nb = p + 1 - am, o = om[m + p];
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int n = am + e / nb, np_ = am + e % nb;
      Az[o + e] = A[(long)(np_ * np_ + np_ + m) * P + (n * n + n + m)];
    }
  }
}
__device__ inline int octant_slot(const int* coord) {
  const int dx = (coord[0] & 1) ? 1 : -1, dy = (coord[1] & 1) ? 1 : -1, dz = (coord[2] & 1) ? 1 : -1;
  return ((dz + 3) * 7 + (dy + 3)) * 7 + (dx + 3);
}

// M_b = sum over children with sources of the rotated shift of M_child (one CTA per parent box)
__global__ void __launch_bounds__(128) k_m2m_rot(int p, const int* __restrict__ boxes, BoxGeom B,
                                                 const long* __restrict__ az_tab, const cplx* __restrict__ Wall,
                                                 const cplx* __restrict__ az_ops, cplx* __restrict__ M) {
  const int b = boxes[blockIdx.x];
  const int P = (p + 1) * (p + 1), NW = (int)rot_nw(p), NAZ = rot_naz(p);
  extern __shared__ cplx sm[];
  cplx* Wc = sm;
  cplx* Az = Wc + NW;
  cplx* x = Az + NAZ;
  cplx* t = x + P;
  cplx* acc = t + P;
  __shared__ int om[2 * FMM_MAXP + 1];
  for (int m = threadIdx.x - p; m <= p; m += blockDim.x) om[m + p] = rot_om(p, m);
  for (int i = threadIdx.x; i < P; i += blockDim.x) acc[i] = C(0, 0);
  const int comp = B.comp[b];
  bool az_loaded = false;
  __syncthreads();
  for (int k = 0; k < B.nchild[b]; ++k) {
    const int c = B.child0[b] + k;
    if (B.se[c] == B.sb[c]) continue;
    if (!az_loaded) {                     // every child is one level below b
      load_coax(p, P, az_ops + az_tab[comp * 23 + B.lev[c]], om, Az);
      az_loaded = true;
    }
    const cplx* Wg = Wall + (long)octant_slot(B.coord + 3 * c) * NW;
    for (int e = threadIdx.x; e < NW; e += blockDim.x) Wc[e] = Wg[e];
    for (int i = threadIdx.x; i < P; i += blockDim.x) x[i] = M[(long)c * P + i];
    __syncthreads();
    rot_stage(P, Wc, x, t, true, false);
    __syncthreads();
    coax_stage(p, P, Az, om, t, x);
    __syncthreads();
    rot_stage(P, Wc, x, acc, false, true);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) M[(long)b * P + i] = acc[i];
}

// L_T += rotated shift of L_parent (one CTA per box of one level >= 3)
__global__ void __launch_bounds__(128) k_l2l_rot(int p, const int* __restrict__ boxes, BoxGeom B,
                                                 const long* __restrict__ az_tab, const cplx* __restrict__ Wall,
                                                 const cplx* __restrict__ az_ops, cplx* __restrict__ L) {
  const int T = boxes[blockIdx.x];
  const int P = (p + 1) * (p + 1), NW = (int)rot_nw(p), NAZ = rot_naz(p);
  extern __shared__ cplx sm[];
  cplx* Wc = sm;
  cplx* Az = Wc + NW;
  cplx* x = Az + NAZ;
  cplx* t = x + P;
  cplx* out = t + P;
  __shared__ int om[2 * FMM_MAXP + 1];
  for (int m = threadIdx.x - p; m <= p; m += blockDim.x) om[m + p] = rot_om(p, m);
  __syncthreads();
  load_coax(p, P, az_ops + az_tab[B.comp[T] * 23 + B.lev[T]], om, Az);
  const cplx* Wg = Wall + (long)octant_slot(B.coord + 3 * T) * NW;
  for (int e = threadIdx.x; e < NW; e += blockDim.x) Wc[e] = Wg[e];
  const int pa = B.parent[T];
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    x[i] = L[(long)pa * P + i];
    out[i] = L[(long)T * P + i];
  }
  __syncthreads();
  rot_stage(P, Wc, x, t, true, false);
  __syncthreads();
  coax_stage(p, P, Az, om, t, x);
  __syncthreads();
  rot_stage(P, Wc, x, out, false, true);
  __syncthreads();
  for (int i = threadIdx.x; i < P; i += blockDim.x) L[(long)T * P + i] = out[i];
}

// Coaxial shift operators for every (component, level >= 3) present: table
// of offsets into the rotation cache's operator buffer (-1 where unused).
void rot_shift_tables(fmm_layered* h, const std::vector<CompGeom>& cgh, const std::vector<std::vector<char>>& has_level,
                      int maxlev, std::vector<long>& m2m_az, std::vector<long>& l2l_az, cudaStream_t st) {
  RotCache& R = h->rot;
  const int p = h->p, P = (p + 1) * (p + 1), nc = (int)cgh.size();
  rot_tables(h, st);
  m2m_az.assign((size_t)nc * 23, -1);
  l2l_az.assign((size_t)nc * 23, -1);
  std::vector<SepJob> jobs;
  for (int c = 0; c < nc; ++c)
    for (int l = 3; l <= maxlev; ++l) {
      if (!has_level[c][l]) continue;
      const double w = cgh[c].h2 / (double)(1 << l);
      for (int kind = 1; kind <= 2; ++kind) {
        const double k = (kind == 1) ? cgh[c].ks : cgh[c].kt;
        auto key = std::make_tuple(rbits(k), rbits(w), -kind);
        auto it = R.az.find(key);
        long off;
        if (it == R.az.end()) {
          off = R.az_used;
          R.az_used += (long)P * P;
          R.az[key] = off;
          SepJob j{};
          j.b[2] = 0.86602540378443864676 * w;      // |(+-w/2, +-w/2, +-w/2)|
          j.k = k;
          j.kind = kind;
          j.out_off = off;
          jobs.push_back(j);
        } else {
          off = it->second;
        }
        (kind == 1 ? m2m_az : l2l_az)[(size_t)c * 23 + l] = off;
      }
    }
  if (!jobs.empty()) {
    R.az_buf.grow_keep(sizeof(cplx) * (size_t)R.az_used, sizeof(cplx) * (size_t)(R.az_used - (long)jobs.size() * P * P),
                       st);
    SepJob* dj = (SepJob*)tc_need(h->W().rot_jobs, sizeof(SepJob) * jobs.size() + 64);
    FMM_CHECK(cudaMemcpyAsync(dj, jobs.data(), sizeof(SepJob) * jobs.size(), cudaMemcpyHostToDevice, st));
    launch_sep_ops(p, dj, (int)jobs.size(), h->tab.gaunt.as<double>(), R.az_buf.as<cplx>(), st);
    FMM_CHECK(cudaGetLastError());
    FMM_CHECK(cudaStreamSynchronize(st));   // the job table is rewritten by the next build
  }
}


void launch_m2m_rot(fmm_layered* h, const int* boxes, int n, BoxGeom B, const long* az_tab, cplx* M, cudaStream_t st) {
  if (!n) return;
  const size_t smem = tiling::shift_smem(h->p);
  FMM_CHECK(cudaFuncSetAttribute(k_m2m_rot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LAUNCH(k_m2m_rot<<<n, 128, smem, st>>>(h->p, boxes, B, az_tab, h->rot.w.as<cplx>(), h->rot.az_buf.as<cplx>(), M));
}

void launch_l2l_rot(fmm_layered* h, const int* boxes, int n, BoxGeom B, const long* az_tab, cplx* L, cudaStream_t st) {
  if (!n) return;
  const size_t smem = tiling::shift_smem(h->p);
  FMM_CHECK(cudaFuncSetAttribute(k_l2l_rot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  LAUNCH(k_l2l_rot<<<n, 128, smem, st>>>(h->p, boxes, B, az_tab, h->rot.w.as<cplx>(), h->rot.az_buf.as<cplx>(), L));
}

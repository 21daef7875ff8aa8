// C ABI and host orchestration of one evaluation (Algorithm 1 for every
// component, summed as in eq. totalinteraction).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <atomic>
#include <map>
#include <set>
#include <thread>
#include <vector>

#include "fmm_internal.h"

// ---- launchers of the other translation units
void launch_gaunt(int p, const std::vector<double>& xg, const std::vector<double>& wg, double* G, double* dx,
                  double* dw, cudaStream_t st);
void launch_sep_ops(int p, const SepJob* jobs, int njobs, const double* G, cplx* ops, cudaStream_t st);
void launch_reac_group(int p, const ReacGroup& g, const RuleNodes& R, int nr, const double* d_rho, const long* d_out_off,
                       cplx* ops, DevBuf& scratch, cudaStream_t st);
size_t reac_group_scratch(int p, int Q, int n_near, int nr);
void launch_p2m(int p, const int* leaves, int n, BoxGeom B, const CompGeom* cgs, const double* spos,
                const cplx* sq, cplx* M, cudaStream_t st);
void launch_m2m(int p, const int* boxes, int n, BoxGeom B, const long* op_base, const cplx* ops, cplx* M,
                cudaStream_t st);
void launch_reac_split(int p, const cplx* full, cplx* out, cudaStream_t st);
void run_m2l_gemm(fmm_layered* h, int nb, long nv, const std::vector<std::vector<int>>& m2l_lvl,
                  const int* dsched, const std::vector<long>& o_m2l, int maxlev, BoxGeom B, OpIndex OI,
                  const int* voff, const int* vidx, const cplx* free_ops, const cplx* reac_ops,
                  const cplx* l2l_ops, const cplx* M, cplx* L, int* err, cudaStream_t st,
                  cudaEvent_t gemm0, cudaEvent_t gemm1, double* gemm_flops, const std::vector<CompGeom>& cgh,
                  const long* l2l_rot_tab);
void rot_shift_tables(fmm_layered* h, const std::vector<CompGeom>& cgh, const std::vector<std::vector<char>>& has_level,
                      int maxlev, std::vector<long>& m2m_az, std::vector<long>& l2l_az, cudaStream_t st);
void launch_m2m_rot(fmm_layered* h, const int* boxes, int n, BoxGeom B, const long* az_tab, cplx* M, cudaStream_t st);
void launch_mark_reac(int nb, BoxGeom B, const CompGeom* cgs, const int* voff, const int* vidx, unsigned char* used,
                      int* err, cudaStream_t st);
void launch_l2p(int p, const int* leaves, int n, BoxGeom B, const CompGeom* cgs, const double* tpos,
                const cplx* L, cplx* phi, cudaStream_t st);
void launch_coef(int L1, const Rule& R, cplx* coef, cudaStream_t st);
RuleView make_rule_view(const Rule& R, const cplx* coef);
void launch_near_reac(const int* leaves, int n, NearBoxes B, const NearComp* ncs, RuleView R, const double* spos,
                      const cplx* sq, const double* tpos, cplx* phi, unsigned long long* counters,
                      unsigned long long* box, cudaStream_t st);
void launch_near(const int* leaves, int n, NearBoxes B, const NearComp* ncs, RuleView R, const double* spos,
                 const cplx* sq, const double* tpos, cplx* phi, unsigned long long* counters, int* err,
                 cudaStream_t st, bool f32);
double measure_fp64_peak_impl();
void launch_direct(long nt, const double* tgt, long ns, const double* src, const double* q, DirectMedium md,
                   RuleView R, const cplx* coef_all, double* out, cudaStream_t st);
void launch_scatter_add(long n, const int* tidx, const cplx* phi, double* out, cudaStream_t st);
void launch_norm_paper(long n, const double* tgt, DirectMedium md, double* out, cudaStream_t st);
void build_trees(fmm_layered* h, long ns, const double* src, const double* q, long nt, const double* tgt,
                 std::vector<double>& gap_out, cudaStream_t st);
void tree_host_copy(fmm_layered* h, std::vector<int>& comp, std::vector<int>& lev,
                    std::vector<unsigned long long>& prefix, std::vector<int>& sb, std::vector<int>& se,
                    std::vector<int>& tb, std::vector<int>& te, std::vector<int>& parent);

static thread_local std::string g_create_err;
thread_local long g_fmm_launches = 0;

using Clock = std::chrono::steady_clock;
static double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

template <class T>
static T* need(DevBuf& b, size_t n) {
  b.ensure(sizeof(T) * (n ? n : 1));
  return b.as<T>();
}
template <class T>
static T* upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  T* p = need<T>(b, v.size());
  if (!v.empty()) FMM_CHECK(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return p;
}

// ---------------------------------------------------------------- create
void init_legendre_tables();
SurrView surrogate_view(const fmm_layered* h);

static void create_impl(fmm_layered* h) {
  FMM_CHECK(cudaGetDevice(&h->dev));
  init_legendre_tables();
  upload(h->d_k, h->k, 0);
  std::vector<double> dd = h->d;
  if (dd.empty()) dd.push_back(0.0);
  upload(h->d_d, dd, 0);
  upload(h->d_eps, h->eps, 0);
  rule_init(h);
  // Gaunt table
  int p = h->p, P = (p + 1) * (p + 1);
  std::vector<double> xg, wg;
  gauss_legendre_pub(2 * p + 2, xg, wg);
  double* G = need<double>(h->tab.gaunt, (size_t)P * P * (2 * p + 1));
  DevBuf tmpx, tmpw;
  double* dx = need<double>(tmpx, xg.size());
  double* dw = need<double>(tmpw, wg.size());
  launch_gaunt(p, xg, wg, G, dx, dw, 0);
  FMM_CHECK(cudaGetLastError());
  // e^{i m phi} for the 49 horizontal offsets of reaction M2L pairs
  std::vector<cplx> ph(49 * (2 * p + 1));
  for (int dy = -3; dy <= 3; ++dy)
    for (int dx = -3; dx <= 3; ++dx) {
      double phi = atan2((double)dy, (double)dx);
      for (int m = -p; m <= p; ++m)
        ph[((dy + 3) * 7 + (dx + 3)) * (2 * p + 1) + (m + p)] = C(cos(m * phi), sin(m * phi));
    }
  upload(h->tab.phase, ph, 0);
  FMM_CHECK(cudaStreamSynchronize(0));
  tmpx.release();
  tmpw.release();
  if (h->flags & FMM_TABLES) {
    tables_build(h, 0);
    h->stats.ms_tables = h->tabs.build_ms;
    h->stats.table_bytes = (double)h->tabs.bytes;
  }
}

extern "C" int fmm_layered_create(int n_layers, const double* k, const double* interfaces, const double* eps,
                                  int p, int leaf, unsigned flags, fmm_layered_t** out) {
  if (out) *out = nullptr;
  g_create_err.clear();
  if (!out || n_layers < 1 || n_layers > FMM_MAXL || !k || (n_layers > 1 && !interfaces) || p < 1 ||
      p > 16 || leaf < 1) {
    g_create_err = "invalid argument (layers in [1,8], p in [1,16], leaf >= 1, k and interfaces given)";
    return FMM_ERR_ARG;
  }
  for (int l = 0; l < n_layers; ++l) {
    if (!(k[l] > 0) || !std::isfinite(k[l]) || (eps && (!(eps[l] > 0) || !std::isfinite(eps[l])))) {
      g_create_err = "wave numbers and material coefficients must be positive and finite";
      return FMM_ERR_ARG;
    }
  }
  for (int j = 0; j + 1 < n_layers; ++j) {
    if (!std::isfinite(interfaces[j]) || (j > 0 && !(interfaces[j] < interfaces[j - 1]))) {
      g_create_err = "interfaces must be finite and strictly decreasing";
      return FMM_ERR_ARG;
    }
  }
  auto t0 = Clock::now();
  fmm_layered* h = new fmm_layered();
  h->L1 = n_layers;
  h->k.assign(k, k + n_layers);
  h->d.assign(interfaces ? interfaces : k, interfaces ? interfaces + (n_layers - 1) : k);
  if (n_layers == 1) h->d.clear();
  h->eps.assign(n_layers, 1.0);
  if (eps) h->eps.assign(eps, eps + n_layers);
  h->p = p;
  h->leaf = leaf;
  h->flags = flags;
  try {
    create_impl(h);
  } catch (FmmError& e) {
    g_create_err = e.msg;
    fmm_layered_destroy(h);
    return e.code;
  }
  h->stats.ms_setup = ms_since(t0);
  h->stats.n_quad_near = h->rule.n_near;
  h->stats.n_quad_total = h->rule.Q();
  *out = h;
  return FMM_OK;
}

static void release_workspace(Workspace& ws);

extern "C" void fmm_layered_destroy(fmm_layered_t* h) {
  if (!h) return;
  h->surr.release();
  h->tabs.release();
  if (h->bstream) cudaStreamDestroy(h->bstream);
  if (h->bdone) cudaEventDestroy(h->bdone);
  DevBuf* all[] = {&h->d_k, &h->d_d, &h->d_eps, &h->rule.kr, &h->rule.w, &h->rule.kz, &h->rule.sigma,
                   &h->tab.gaunt, &h->tab.phase};
  for (DevBuf* b : all) b->release();
  if (h->wsp.use_count() == 1) release_workspace(h->W());
  DevBuf* gb[] = {&h->tc.bbuf, &h->tc.sbuf, &h->tc.phase_f, &h->rot.w, &h->rot.az_buf};
  for (DevBuf* b : gb) b->release();
  h->cache.free_buf.release();
  h->cache.shift_buf.release();
  h->cache.rad_buf.release();
  delete h;
}

static void release_workspace(Workspace& ws) {
  DevBuf* wsb[] = {&ws.slayer, &ws.tlayer, &ws.sorder, &ws.torder, &ws.iota, &ws.ltmp, &ws.counts, &ws.bbox,
                   &ws.gap, &ws.flags, &ws.spos_u, &ws.sq_u, &ws.skey_u, &ws.sval_u, &ws.sidx_u, &ws.tpos_u,
                   &ws.tkey_u, &ws.tval_u, &ws.tidx_u, &ws.skey, &ws.sperm, &ws.spos, &ws.sq, &ws.sidx,
                   &ws.slocal, &ws.tkey, &ws.tperm, &ws.tpos, &ws.tidx, &ws.tlocal, &ws.segs, &ws.segl, &ws.segs_keys,
                   &ws.bcomp, &ws.blevel, &ws.bprefix, &ws.bsb, &ws.bse, &ws.btb, &ws.bte, &ws.bparent,
                   &ws.bchild0, &ws.bnchild, &ws.bcoord, &ws.lvlcnt, &ws.lvlscan, &ws.lvl_begin, &ws.lcnt,
                   &ws.loff, &ws.vi, &ws.ui, &ws.wi, &ws.xi, &ws.M, &ws.L, &ws.m2l_free, &ws.m2m_op,
                   &ws.l2l_op, &ws.m2l_reac, &ws.op_tab, &ws.phi, &ws.out_tmp, &ws.sort_tmp, &ws.grule,
                   &ws.gargs};
  for (DevBuf* b : wsb) b->release();
  DevBuf* gb[] = {&ws.g_owner, &ws.g_keys, &ws.g_vals, &ws.g_inv, &ws.g_Y, &ws.g_Z, &ws.g_runs, &ws.g_bat,
                  &ws.tc_runs, &ws.tc_jobs, &ws.tc_a, &ws.tc_sig, &ws.tc_parts, &ws.tc_items, &ws.tc_etab,
                  &ws.rot_info, &ws.rot_jobs, &ws.rot_bat, &ws.rot_rs, &ws.rot_tab};
  for (DevBuf* b : gb) b->release();
}

extern "C" int fmm_layered_share_workspace(fmm_layered_t* h, fmm_layered_t* owner) {
  if (!h || !owner) return FMM_ERR_ARG;
  if (h->dev != owner->dev) {
    h->err = "handles on different devices";
    return FMM_ERR_ARG;
  }
  if (h->wsp == owner->wsp) return FMM_OK;
  cudaDeviceSynchronize();           // no evaluation of h may still use its old workspace
  if (h->wsp.use_count() == 1) release_workspace(h->W());
  h->wsp = owner->wsp;
  return FMM_OK;
}

extern "C" const char* fmm_layered_last_error(const fmm_layered_t* h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

extern "C" int fmm_layered_stats(const fmm_layered_t* h, fmm_stats_t* s) {
  if (!h || !s) return FMM_ERR_ARG;
  *s = h->stats;
  return FMM_OK;
}

extern "C" int fmm_layered_table_operator(fmm_layered_t* h, int l, int lp, int a, int b, double w, int jt, int js,
                                          int r, double* out) {
  if (!h || !out) return FMM_ERR_ARG;
  if (l < 0 || lp < 0 || l >= h->L1 || lp >= h->L1 || a < 0 || a > 1 || b < 0 || b > 1 || !(w > 0)) {
    h->err = "invalid class";
    return FMM_ERR_ARG;
  }
  try {
    FMM_CHECK(cudaSetDevice(h->dev));
    tables_operator_host(h, TabClass{l, lp, a, b, jt, js, r, w, 0}, out, 0);
  } catch (FmmError& e) {
    h->err = e.msg;
    return e.code;
  }
  return FMM_OK;
}

static DirectMedium medium_of(const fmm_layered* h) {
  DirectMedium md{};
  md.L1 = h->L1;
  for (int l = 0; l < h->L1; ++l) md.k[l] = h->k[l];
  for (size_t j = 0; j < h->d.size(); ++j) md.d[j] = h->d[j];
  return md;
}

// reaction coefficients for the current rule: [(l,l',a,b)][q]
static cplx* rule_coef(fmm_layered* h, cudaStream_t st) {
  cplx* coef = need<cplx>(h->W().op_tab, (size_t)h->L1 * h->L1 * 4 * h->rule.Q());
  launch_coef(h->L1, h->rule, coef, st);
  FMM_CHECK(cudaGetLastError());
  return coef;
}

// ---------------------------------------------------------------- direct
extern "C" int fmm_layered_direct(fmm_layered_t* h, long ns, const double* src, const double* q, long nt,
                                  const double* tgt, double* out, void* stream) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (ns < 0 || nt < 0 || (ns && (!src || !q)) || (nt && (!tgt || !out))) {
    h->err = "invalid argument";
    return FMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  try {
    if (nt == 0) return FMM_OK;
    // tail long enough for the smallest vertical gap: classify on the device
    std::vector<double> gap;
    build_trees(h, ns, src, q, nt, tgt, gap, st);
    double gmin = INFINITY, smin = INFINITY;
    for (int l = 0; l < h->L1; ++l)
      for (int sd = 0; sd < 2; ++sd) {
        smin = fmin(smin, gap[(0 * h->L1 + l) * 2 + sd]);
        gmin = fmin(gmin, gap[(1 * h->L1 + l) * 2 + sd]);
      }
    if (h->L1 > 1 && std::isfinite(gmin + smin)) rule_extend(h, h->rule.near_tmax(gmin + smin), st);
    cplx* coef = rule_coef(h, st);
    RuleView rv = make_rule_view(h->rule, coef);
    rv.surr = surrogate_view(h);
    launch_direct(nt, tgt, ns, src, q, medium_of(h), rv, coef, out, st);
    if (h->flags & FMM_NORM_PAPER) launch_norm_paper(nt, tgt, medium_of(h), out, st);
    FMM_CHECK(cudaGetLastError());
    FMM_CHECK(cudaStreamSynchronize(st));
  } catch (FmmError& e) {
    h->err = e.msg;
    return e.code;
  }
  return FMM_OK;
}

// ---------------------------------------------------------------- eval
struct StageEvents {
  cudaEvent_t ev[12];
  StageEvents() { for (auto& e : ev) cudaEventCreate(&e); }
  ~StageEvents() { for (auto& e : ev) cudaEventDestroy(e); }
  void mark(int i, cudaStream_t st) { cudaEventRecord(ev[i], st); }
  double ms(int a, int b) {
    float v = 0;
    cudaEventElapsedTime(&v, ev[a], ev[b]);
    return v;
  }
};

static const int RHO2[10] = {0, 1, 2, 4, 5, 8, 9, 10, 13, 18};

static uint64_t dbits(double x) {
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}

// Append n operators of P^2 elements to a cache buffer (device contents kept).
static long cache_alloc(DevBuf& buf, long& used, long n_elems, cudaStream_t st) {
  long off = used;
  buf.grow_keep(sizeof(cplx) * (size_t)(used + n_elems), sizeof(cplx) * (size_t)used, st);
  used += n_elems;
  return off;
}

static void eval_impl(fmm_layered* h, long ns, const double* src, const double* q, long nt, const double* tgt,
                      double* out, cudaStream_t st) {
  Workspace& ws = h->W();
  OpCache& oc = h->cache;
  const int p = h->p, P = (p + 1) * (p + 1);
  const long PP = (long)P * P;
  FMM_CHECK(cudaMemsetAsync(out, 0, sizeof(double) * 2 * nt, st));
  if (nt == 0 || ns == 0) return;
  StageEvents E;
  E.mark(0, st);
  long launches0 = g_fmm_launches;
  auto t0 = Clock::now();
  std::vector<double> gap;
  build_trees(h, ns, src, q, nt, tgt, gap, st);
  const std::vector<Comp>& comps = h->comps;
  const int nc = (int)comps.size();
  h->comp_work.assign(nc, 0.0);
  if (nc == 0) {                       // no component selected: the potentials stay zero
    h->stats.n_launches = g_fmm_launches - launches0;
    return;
  }
  const int nb = h->nboxes;
  const std::vector<int>& lvl = h->lvl_begin;
  int maxlev = 0;
  while (maxlev + 1 < 22 && lvl[maxlev + 2] > lvl[maxlev + 1]) ++maxlev;
  std::vector<CompGeom> cg(nc);
  int nfree = 0, nreac = 0;
  for (int c = 0; c < nc; ++c) {
    const Comp& C_ = comps[c];
    for (int a = 0; a < 3; ++a) cg[c].lo[a] = C_.c[a] - C_.h;
    cg[c].h2 = 2.0 * C_.h;
    cg[c].ks = C_.ks;
    cg[c].kt = C_.kt;
    cg[c].kind = C_.kind;
    cg[c].a = C_.a;
    cg[c].dref = C_.dref;
    cg[c].free_idx = (C_.kind == CK_FREE) ? nfree++ : -1;
    cg[c].reac_idx = (C_.kind == CK_REAC) ? nreac++ : -1;
  }
  CompGeom* dcg = upload(ws.segl, cg, st);   // segl is free after the tree build
  BoxGeom B;
  B.comp = ws.bcomp.as<int>(); B.lev = ws.blevel.as<int>(); B.sb = ws.bsb.as<int>(); B.se = ws.bse.as<int>();
  B.tb = ws.btb.as<int>(); B.te = ws.bte.as<int>(); B.parent = ws.bparent.as<int>();
  B.child0 = ws.bchild0.as<int>(); B.nchild = ws.bnchild.as<int>(); B.coord = ws.bcoord.as<int>();
  const int* loff = ws.loff.as<int>();
  // reaction M2L classes used by the V lists
  unsigned char* dused = need<unsigned char>(ws.lvlcnt, (size_t)nc * 23 * 40);
  int* err = need<int>(ws.flags, 1);
  FMM_CHECK(cudaMemsetAsync(dused, 0, (size_t)nc * 23 * 40, st));
  FMM_CHECK(cudaMemsetAsync(err, 0, 4, st));
  launch_mark_reac(nb, B, dcg, loff, ws.vi.as<int>(), dused, err, st);
  FMM_CHECK(cudaGetLastError());
  // host copies needed for scheduling
  std::vector<int> bcomp(nb), bnchild(nb), bsb(nb), bse(nb), btb(nb), bte(nb), bpar(nb);
  std::vector<unsigned char> used((size_t)nc * 23 * 40);
  FMM_CHECK(cudaMemcpyAsync(bcomp.data(), ws.bcomp.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(bnchild.data(), ws.bnchild.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(bsb.data(), ws.bsb.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(bse.data(), ws.bse.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(btb.data(), ws.btb.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(bte.data(), ws.bte.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(bpar.data(), ws.bparent.ptr, 4 * nb, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(used.data(), dused, used.size(), cudaMemcpyDeviceToHost, st));
  std::vector<int> lo_all(4 * (size_t)(nb + 1));
  FMM_CHECK(cudaMemcpyAsync(lo_all.data(), ws.loff.ptr, 4 * lo_all.size(), cudaMemcpyDeviceToHost, st));
  int herr0 = 0;
  FMM_CHECK(cudaMemcpyAsync(&herr0, err, 4, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  if (herr0) throw FmmError(FMM_ERR_UNSUPPORTED, "reaction M2L pair outside the interface band");
  const int* uo = lo_all.data() + (nb + 1);
  h->stats.n_u_pairs = uo[nb];
  {
    long vr = 0;
    for (int b = 0; b < nb; ++b)
      if (comps[bcomp[b]].kind == CK_REAC) vr += lo_all[b + 1] - lo_all[b];
    h->stats.n_v_pairs_reac = vr;
  }
  // does any reaction component need near-field (direct) interactions?
  bool reac_near = false;
  for (int b = 0; b < nb && !reac_near; ++b) {
    if (comps[bcomp[b]].kind != CK_REAC) continue;
    for (int k = 1; k < 4; ++k) {
      const int* o = lo_all.data() + (size_t)k * (nb + 1);
      if (o[b + 1] > o[b]) { reac_near = true; break; }
    }
  }
  std::vector<std::vector<char>> has_level(nc, std::vector<char>(23, 0));
  for (int l = 0; l <= maxlev; ++l)
    for (int b = lvl[l]; b < lvl[l + 1]; ++b) has_level[bcomp[b]][l] = 1;
  h->stats.ms_tree = ms_since(t0);
  E.mark(1, st);
  // ---- operators (cached across evaluations)
  auto t1 = Clock::now();
  {
    size_t bytes = sizeof(cplx) * (size_t)(oc.free_used + oc.shift_used + oc.rad_used);
    if (bytes > (size_t)8 << 30) oc.clear();        // keep the cache bounded
  }
  std::vector<long> m2m_base(nc * 23, -1), l2l_base(nc * 23, -1), m2l_base(nc * 23, -1);
  std::vector<long> reac_off((size_t)nc * 23 * 40, -1);
  std::vector<SepJob> sep_shift, sep_free;
  // dense free-space M2L operators: read by the tensor-core form and by the
  // dense FP64 form (p < 5); the FP64 form runs p >= 5 in rotation form
  const bool dense_free = (h->flags & FMM_MIXED) || p < 5;
  for (int c = 0; c < nc; ++c) {
    for (int l = 2; l <= maxlev; ++l) {
      if (!has_level[c][l]) continue;
      double w = cg[c].h2 / (double)(1 << l);
      if (l >= 3) {
        for (int kind = 1; kind <= 2; ++kind) {
          double k = (kind == 1) ? cg[c].ks : cg[c].kt;
          auto key = std::make_tuple(dbits(k), dbits(w), kind);
          auto it = oc.shift.find(key);
          long off;
          if (it == oc.shift.end()) {
            off = cache_alloc(oc.shift_buf, oc.shift_used, 8 * PP, st);
            oc.shift[key] = off;
            for (int o = 0; o < 8; ++o) {
              SepJob j{};
              for (int a = 0; a < 3; ++a) j.b[a] = (((o >> a) & 1) ? 0.5 : -0.5) * w;
              j.k = k;
              j.kind = kind;
              j.out_off = off + (long)o * PP;
              sep_shift.push_back(j);
            }
          } else {
            off = it->second;
          }
          (kind == 1 ? m2m_base : l2l_base)[c * 23 + l] = off;
        }
      }
      if (comps[c].kind == CK_FREE) {
        auto key = std::make_pair(dbits(cg[c].kt), dbits(w));
        auto it = oc.free_m2l.find(key);
        long off;
        if (it == oc.free_m2l.end() && !dense_free) {
          // FP64 path with p >= 5: the free-space translations run in
          // rotation form (coaxial operators only), so the 343 dense
          // operators are not built; the offset only names the class
          off = oc.free_virtual;
          oc.free_virtual += 343 * PP;
          oc.free_m2l[key] = off;
        } else if (it == oc.free_m2l.end()) {
          off = cache_alloc(oc.free_buf, oc.free_used, 343 * PP, st);
          oc.free_m2l[key] = off;
          for (int dz = -3; dz <= 3; ++dz)
            for (int dy = -3; dy <= 3; ++dy)
              for (int dx = -3; dx <= 3; ++dx) {
                if (std::max(abs(dx), std::max(abs(dy), abs(dz))) < 2) continue;
                SepJob j{};
                j.b[0] = dx * w; j.b[1] = dy * w; j.b[2] = dz * w;
                j.k = cg[c].kt;
                j.kind = 0;
                j.out_off = off + (((dz + 3) * 7 + (dy + 3)) * 7 + (dx + 3)) * PP;
                sep_free.push_back(j);
              }
        } else {
          off = it->second;
        }
        m2l_base[c * 23 + l] = off;
      }
    }
  }
  // reaction radial operators: only classes present, computed once per geometry
  struct Pending { int c, l, jt, js; std::vector<int> rs; std::vector<long> offs; };
  std::vector<Pending> pend;
  std::vector<TabClass> tab_cls;
  double tmax = h->rule.ta;
  for (int c = 0; c < nc; ++c) {
    if (comps[c].kind != CK_REAC) continue;
    for (int l = 2; l <= maxlev; ++l) {
      double w = cg[c].h2 / (double)(1 << l);
      for (int g = 0; g < 4; ++g) {
        Pending pd{c, l, g / 2, g % 2, {}, {}};
        const bool by_table = tables_cover(h, w);
        for (int r = 0; r < 10; ++r) {
          if (!used[((size_t)c * 23 + l) * 40 + g * 10 + r]) continue;
          const Comp& C_ = comps[c];
          auto key = std::make_tuple(C_.l, C_.lp, C_.a, C_.b, dbits(w), pd.jt, pd.js, r);
          auto it = oc.rad.find(key);
          if (it != oc.rad.end()) {
            reac_off[((size_t)c * 23 + l) * 40 + g * 10 + r] = it->second;
          } else if (by_table) {
            // interpolated from the tabulated integrals (FMM_TABLES)
            const long npp = (long)(p + 1) * (p + 2) / 2, nmm = (long)p * (p + 1) / 2;
            long off = cache_alloc(oc.rad_buf, oc.rad_used, npp * npp + nmm * nmm, st);
            oc.rad[key] = off;
            reac_off[((size_t)c * 23 + l) * 40 + g * 10 + r] = off;
            tab_cls.push_back(TabClass{C_.l, C_.lp, C_.a, C_.b, pd.jt, pd.js, r, w, off});
          } else {
            pd.rs.push_back(r);
          }
        }
        if (!pd.rs.empty()) pend.push_back(pd);     // each group integrates on its own rule (group_rule)
      }
    }
  }
  // the near field needs the rule up to ta + 30 / (smallest vertical gap)
  double gmin = INFINITY, smin = INFINITY;
  for (int l = 0; l < h->L1; ++l)
    for (int sd = 0; sd < 2; ++sd) {
      smin = fmin(smin, gap[(0 * h->L1 + l) * 2 + sd]);
      gmin = fmin(gmin, gap[(1 * h->L1 + l) * 2 + sd]);
    }
  if (h->L1 > 1 && std::isfinite(gmin + smin) && reac_near)
    tmax = std::max(tmax, h->rule.near_tmax(gmin + smin));
  if ((tmax - h->rule.ta) / h->rule.panel > 4.0e6)
    throw FmmError(FMM_ERR_UNSUPPORTED, "points too close to an interface: the quadrature tail would exceed 4e6 panels");
  rule_extend(h, tmax, st);
  const int Q = h->rule.Q();
  h->stats.n_quad_total = Q;
  long n_classes = 0, t_nodes = 0;
  if (!sep_shift.empty() || !sep_free.empty()) {
    std::vector<SepJob> all = sep_shift;
    all.insert(all.end(), sep_free.begin(), sep_free.end());
    SepJob* dj = (SepJob*)need<char>(ws.op_tab, sizeof(SepJob) * all.size());
    FMM_CHECK(cudaMemcpyAsync(dj, all.data(), sizeof(SepJob) * all.size(), cudaMemcpyHostToDevice, st));
    launch_sep_ops(p, dj, (int)sep_shift.size(), h->tab.gaunt.as<double>(), oc.shift_buf.as<cplx>(), st);
    launch_sep_ops(p, dj + sep_shift.size(), (int)sep_free.size(), h->tab.gaunt.as<double>(), oc.free_buf.as<cplx>(), st);
    FMM_CHECK(cudaGetLastError());
  }
  // reaction groups by quadrature: plan every group on the host (its own
  // scale-adapted rule, cache slots of its classes), upload the nodes and the
  // small argument arrays of all groups at once, then launch the groups one
  // after the other without synchronizing in between
  struct GroupPlan {
    ReacGroup g;
    std::vector<double> rho;
    std::vector<long> split;
    long node0;              // first node of the group in the concatenated node arrays
  };
  std::vector<GroupPlan> plans;
  std::vector<cplx> hkr, hw;
  {
    const long npp = (long)(p + 1) * (p + 2) / 2, nmm = (long)p * (p + 1) / 2;
    const long split_elems = npp * npp + nmm * nmm;
    const int nn = h->rule.n_near;
    for (Pending& pd : pend) {
      const Comp& C_ = comps[pd.c];
      const double w = cg[pd.c].h2 / (double)(1 << pd.l);
      GroupPlan gp;
      ReacGroup& g = gp.g;
      g = ReacGroup{};
      g.l = C_.l; g.lp = C_.lp; g.a = C_.a; g.b = C_.b;
      g.kl = h->k[C_.l]; g.klp = h->k[C_.lp];
      g.zt = (pd.jt + 0.5) * w;
      g.zs = (pd.js + 0.5) * w;
      double rho_max = 0.0;
      for (int r : pd.rs) rho_max = std::max(rho_max, sqrt((double)RHO2[r]) * w);
      gp.node0 = (long)hkr.size();
      hkr.resize(hkr.size() + nn, C(0, 0));          // complex contour: filled on the device
      hw.resize(hw.size() + nn, C(0, 0));
      g.Q = nn + group_tail(h, g.zt + g.zs, rho_max, hkr, hw);
      g.sig_off = ((((long)C_.l * h->L1 + C_.lp) * 2 + C_.a) * 2 + C_.b) * g.Q;
      for (int r : pd.rs) {
        gp.rho.push_back(sqrt((double)RHO2[r]) * w);
        long off = cache_alloc(oc.rad_buf, oc.rad_used, split_elems, st);
        gp.split.push_back(off);
        oc.rad[std::make_tuple(C_.l, C_.lp, C_.a, C_.b, dbits(w), pd.jt, pd.js, r)] = off;
        reac_off[((size_t)pd.c * 23 + pd.l) * 40 + (pd.jt * 2 + pd.js) * 10 + r] = off;
      }
      plans.push_back(std::move(gp));
    }
  }
  if (!plans.empty()) {
    const int L1 = h->L1;
    const long ntot = (long)hkr.size();
    cplx* nodes = need<cplx>(ws.grule, (size_t)ntot * (2 + L1 + 4 * L1 * L1));
    cplx* kr_all = nodes;
    cplx* w_all = kr_all + ntot;
    cplx* kz_all = w_all + ntot;                       // group g: [L1][Q_g] at L1 * node0
    cplx* sig_all = kz_all + (size_t)L1 * ntot;        // group g: [L1][L1][2][2][Q_g] at 4 L1^2 * node0
    FMM_CHECK(cudaMemcpyAsync(kr_all, hkr.data(), sizeof(cplx) * ntot, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(w_all, hw.data(), sizeof(cplx) * ntot, cudaMemcpyHostToDevice, st));
    // per group: 10 radial distances and 10 output offsets
    std::vector<char> blob(plans.size() * (sizeof(double) * 10 + sizeof(long) * 10), 0);
    size_t scratch = 0;
    for (size_t i = 0; i < plans.size(); ++i) {
      char* b = blob.data() + i * (sizeof(double) * 10 + sizeof(long) * 10);
      memcpy(b, plans[i].rho.data(), sizeof(double) * plans[i].rho.size());
      for (size_t k = 0; k < plans[i].rho.size(); ++k) {
        long o = (long)k * PP;                          // full radial matrix k of the group in scratch
        memcpy(b + sizeof(double) * 10 + sizeof(long) * k, &o, sizeof(long));
      }
      scratch = std::max(scratch, reac_group_scratch(p, plans[i].g.Q, h->rule.n_near, (int)plans[i].rho.size()));
    }
    char* dargs = need<char>(ws.gargs, blob.size());
    FMM_CHECK(cudaMemcpyAsync(dargs, blob.data(), blob.size(), cudaMemcpyHostToDevice, st));
    ws.m2l_reac.ensure(scratch);                        // sized once: no reallocation between launches
    cplx* full = need<cplx>(ws.out_tmp, (size_t)PP * 10 + 64);
    for (size_t i = 0; i < plans.size(); ++i) {
      const GroupPlan& gp = plans[i];
      const long n0 = gp.node0;
      const RuleNodes RN{kr_all + n0, w_all + n0, kz_all + (size_t)L1 * n0, sig_all + (size_t)4 * L1 * L1 * n0,
                         gp.g.Q, h->rule.n_near};
      group_rule_fill(h, RN, st);
      const double* drho = (const double*)(dargs + i * (sizeof(double) * 10 + sizeof(long) * 10));
      const long* doff = (const long*)(drho + 10);
      launch_reac_group(p, gp.g, RN, (int)gp.rho.size(), drho, doff, full, ws.m2l_reac, st);
      for (size_t k = 0; k < gp.rho.size(); ++k)
        launch_reac_split(p, full + (long)k * PP, oc.rad_buf.as<cplx>() + gp.split[k], st);
      n_classes += (long)gp.rho.size();
      t_nodes += (long)gp.g.Q * (long)gp.rho.size();
    }
    FMM_CHECK(cudaGetLastError());
  }
  if (!tab_cls.empty()) {
    tables_ops(h, tab_cls, oc.rad_buf.as<cplx>(), st);
    n_classes += (long)tab_cls.size();
  }
  h->stats.n_reac_table_classes = (long)tab_cls.size();
  // any still-missing offsets (classes computed by an earlier evaluation)
  for (int c = 0; c < nc; ++c) {
    if (comps[c].kind != CK_REAC) continue;
    for (int l = 2; l <= maxlev; ++l) {
      double w = cg[c].h2 / (double)(1 << l);
      for (int g = 0; g < 40; ++g) {
        size_t idx = ((size_t)c * 23 + l) * 40 + g;
        if (!used[idx] || reac_off[idx] >= 0) continue;
        const Comp& C_ = comps[c];
        reac_off[idx] = oc.rad.at(std::make_tuple(C_.l, C_.lp, C_.a, C_.b, dbits(w), (g / 10) / 2, (g / 10) % 2, g % 10));
      }
    }
  }
  FMM_CHECK(cudaStreamSynchronize(st));
  h->stats.ms_operators = ms_since(t1);
  h->stats.n_reac_classes = n_classes;
  h->stats.n_free_ops = (long)sep_free.size();
  h->stats.n_reac_T_nodes = t_nodes;
  // shifts in rotation form (p >= 5): coaxial operators per (component, level)
  const bool rot_shifts = p >= 5;
  long* d_rot_tab = nullptr;
  if (rot_shifts) {
    std::vector<long> m2m_az, l2l_az;
    rot_shift_tables(h, cg, has_level, maxlev, m2m_az, l2l_az, st);
    m2m_az.insert(m2m_az.end(), l2l_az.begin(), l2l_az.end());
    d_rot_tab = (long*)tc_need(ws.rot_tab, sizeof(long) * m2m_az.size() + 64);
    FMM_CHECK(cudaMemcpyAsync(d_rot_tab, m2m_az.data(), sizeof(long) * m2m_az.size(), cudaMemcpyHostToDevice, st));
  }
  // ---- passes
  auto t2 = Clock::now();
  long* dtabs = nullptr;
  {
    std::vector<long> tabs;
    tabs.insert(tabs.end(), m2m_base.begin(), m2m_base.end());
    tabs.insert(tabs.end(), l2l_base.begin(), l2l_base.end());
    tabs.insert(tabs.end(), m2l_base.begin(), m2l_base.end());
    tabs.insert(tabs.end(), reac_off.begin(), reac_off.end());
    dtabs = upload(ws.lvlscan, tabs, st);
  }
  cplx* M = need<cplx>(ws.M, (size_t)nb * P);
  cplx* L = need<cplx>(ws.L, (size_t)nb * P);
  std::vector<int> p2m_leaves, l2p_leaves, near_free, near_reac;
  std::vector<std::vector<int>> m2m_lvl(23), m2l_lvl(23);
  for (int l = 0; l <= maxlev; ++l)
    for (int b = lvl[l]; b < lvl[l + 1]; ++b) {
      bool src_ = bse[b] > bsb[b], tgt_ = bte[b] > btb[b];
      bool leaf = bnchild[b] == 0;
      if (src_ && l >= 2) {
        if (leaf) p2m_leaves.push_back(b);
        else m2m_lvl[l].push_back(b);
      }
      if (tgt_ && l >= 2) m2l_lvl[l].push_back(b);
      if (tgt_ && leaf) {
        (comps[bcomp[b]].kind == CK_FREE ? near_free : near_reac).push_back(b);
        if (l >= 2) l2p_leaves.push_back(b);
      }
    }
  // near-field leaves with the most pairs first (targets x U and W entries),
  // so that the long CTAs start in the first wave; each CTA sums only its own
  // targets, so the order does not change any result
  {
    const int* uo_h = lo_all.data() + (nb + 1);
    const int* wo_h = lo_all.data() + 2 * (size_t)(nb + 1);
    auto work = [&](int b) {
      return (long)(bte[b] - btb[b]) * (long)(uo_h[b + 1] - uo_h[b] + wo_h[b + 1] - wo_h[b] + 1);
    };
    auto by_work = [&](int a, int b) {
      const long wa = work(a), wb = work(b);
      return wa != wb ? wa > wb : a < b;
    };
    std::sort(near_free.begin(), near_free.end(), by_work);
    std::sort(near_reac.begin(), near_reac.end(), by_work);
  }
  // reaction near field: (leaf, first target) items of up to 4 targets, for
  // the leaves with U, W or X entries (their own or an ancestor's X list)
  std::vector<int> reac_items;
  {
    const int* uo_h = lo_all.data() + (nb + 1);
    const int* wo_h = lo_all.data() + 2 * (size_t)(nb + 1);
    const int* xo_h = lo_all.data() + 3 * (size_t)(nb + 1);
    for (int b : near_reac) {
      bool any = uo_h[b + 1] > uo_h[b] || wo_h[b + 1] > wo_h[b];
      for (int A = b; !any && A >= 0; A = bpar[A]) any = xo_h[A + 1] > xo_h[A];
      if (!any) continue;
      for (int t = btb[b]; t < bte[b]; t += 4) {
        reac_items.push_back(b);
        reac_items.push_back(t);
      }
    }
  }
  std::vector<int> sched;
  auto push = [&](const std::vector<int>& v) { long o = sched.size(); sched.insert(sched.end(), v.begin(), v.end()); return o; };
  long o_p2m = push(p2m_leaves), o_l2p = push(l2p_leaves), o_near_free = push(near_free),
       o_near_reac = push(reac_items);
  std::vector<long> o_m2m(23), o_m2l(23);
  for (int l = 0; l <= maxlev; ++l) { o_m2m[l] = push(m2m_lvl[l]); o_m2l[l] = push(m2l_lvl[l]); }
  int* dsched = upload(ws.lcnt, sched, st);
  FMM_CHECK(cudaMemsetAsync(err, 0, 4, st));
  E.mark(2, st);        // the scheduling above is host work: it counts to the operator stage
  // upward pass
  launch_p2m(p, dsched + o_p2m, (int)p2m_leaves.size(), B, dcg, ws.spos.as<double>(), ws.sq.as<cplx>(), M, st);
  for (int l = maxlev; l >= 2; --l) {
    if (rot_shifts) launch_m2m_rot(h, dsched + o_m2m[l], (int)m2m_lvl[l].size(), B, d_rot_tab, M, st);
    else launch_m2m(p, dsched + o_m2m[l], (int)m2m_lvl[l].size(), B, dtabs, oc.shift_buf.as<cplx>(), M, st);
  }
  FMM_CHECK(cudaGetLastError());
  E.mark(3, st);
  // downward pass
  OpIndex OI;
  OI.l2l_base = dtabs + nc * 23;
  OI.m2l_base = dtabs + 2 * nc * 23;
  OI.reac_off = dtabs + 3 * nc * 23;
  OI.phase = h->tab.phase.as<cplx>();
  OI.cgs = dcg;
  double gemm_flops = 0.0;
  const bool gemm_ran = lo_all[nb] > 0;
  h->stats.m2l_tensor_flops = 0.0;
  h->stats.m2l_tc_bytes = 0.0;
  run_m2l_gemm(h, nb, (long)lo_all[nb], m2l_lvl, dsched, o_m2l, maxlev, B, OI, loff, ws.vi.as<int>(),
               oc.free_buf.as<cplx>(), oc.rad_buf.as<cplx>(), oc.shift_buf.as<cplx>(), M, L, err, st, E.ev[10],
               E.ev[11], &gemm_flops, cg, rot_shifts ? d_rot_tab + (size_t)nc * 23 : nullptr);
  FMM_CHECK(cudaGetLastError());
  E.mark(4, st);
  long NT = comps.empty() ? 0 : comps.back().to + comps.back().nt;
  cplx* phi = need<cplx>(ws.phi, std::max<long>(1, NT));
  FMM_CHECK(cudaMemsetAsync(phi, 0, sizeof(cplx) * NT, st));
  launch_l2p(p, dsched + o_l2p, (int)l2p_leaves.size(), B, dcg, ws.tpos.as<double>(), L, phi, st);
  // near field
  cplx* coef = rule_coef(h, st);
  E.mark(5, st);
  std::vector<NearComp> ncs(nc);
  for (int c = 0; c < nc; ++c) {
    const Comp& C_ = comps[c];
    ncs[c].kind = C_.kind; ncs[c].l = C_.l; ncs[c].lp = C_.lp; ncs[c].a = C_.a; ncs[c].b = C_.b;
    ncs[c].k = C_.kt;
    ncs[c].dref = C_.dref;
    ncs[c].coef_off = ((((long)C_.l * h->L1 + C_.lp) * 2 + C_.a) * 2 + C_.b) * Q;
  }
  NearComp* dnc = upload(ws.segs, ncs, st);
  NearBoxes NB;
  NB.comp = B.comp; NB.lev = B.lev; NB.sb = B.sb; NB.se = B.se; NB.tb = B.tb; NB.te = B.te; NB.parent = B.parent;
  NB.uo = loff + (nb + 1); NB.ui = ws.ui.as<int>();
  NB.wo = loff + 2 * (nb + 1); NB.wi = ws.wi.as<int>();
  NB.xo = loff + 3 * (nb + 1); NB.xi = ws.xi.as<int>();
  // counters: free pairs, nodes, -, reaction pairs, nodes, surrogate pairs;
  // then the reaction near-field box: max rho, min z, max z (double bits);
  // then the near-field pairs of each component
  unsigned long long* counters = need<unsigned long long>(ws.iota, 10 + nc);
  FMM_CHECK(cudaMemsetAsync(counters, 0, 8 * (10 + nc), st));
  FMM_CHECK(cudaMemsetAsync(counters + 7, 0x7F, 8, st));      // min z starts above every finite value
  NB.comp_pairs = counters + 9;
  NB.tab_pairs = counters + 9 + nc;
  launch_near(dsched + o_near_free, (int)near_free.size(), NB, dnc, make_rule_view(h->rule, coef),
              ws.spos.as<double>(), ws.sq.as<cplx>(), ws.tpos.as<double>(), phi, counters, err, st,
              (h->flags & FMM_MIXED) != 0);
  E.mark(6, st);
  RuleView rv_reac = make_rule_view(h->rule, coef);
  rv_reac.surr = surrogate_view(h);
  rv_reac.ntab = near_table_view(h);
  rv_reac.tail_f32 = (h->flags & FMM_MIXED) ? 1 : 0;
  launch_near_reac(dsched + o_near_reac, (int)(reac_items.size() / 2), NB, dnc, rv_reac, ws.spos.as<double>(),
                   ws.sq.as<cplx>(), ws.tpos.as<double>(), phi, counters + 3, counters + 6, st);
  FMM_CHECK(cudaGetLastError());
  E.mark(7, st);
  for (int c = 0; c < nc; ++c)
    launch_scatter_add(comps[c].nt, ws.tidx.as<int>() + comps[c].to, phi + comps[c].to, out, st);
  if (h->flags & FMM_NORM_PAPER) launch_norm_paper(nt, tgt, medium_of(h), out, st);
  FMM_CHECK(cudaGetLastError());
  E.mark(8, st);
  int herr = 0;
  std::vector<unsigned long long> hcv(10 + nc);
  unsigned long long* hc = hcv.data();
  FMM_CHECK(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(hc, counters, 8 * (10 + nc), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  if (herr & 16) throw FmmError(FMM_ERR_TIMEOUT, "tensor-core M2L: a bounded wait on an mbarrier expired");
  if (herr & 32) throw FmmError(FMM_ERR_TIMEOUT, "near field: a bounded wait for the source copies expired");
  if (herr) throw FmmError(FMM_ERR_UNSUPPORTED, "reaction M2L pair without an operator");
  h->stats.ms_eval = ms_since(t2);
  h->stats.gpu_ms_tree = E.ms(0, 1);
  h->stats.gpu_ms_operators = E.ms(1, 2);
  h->stats.gpu_ms_upward = E.ms(2, 3);
  h->stats.gpu_ms_m2l = E.ms(3, 4);
  h->stats.gpu_ms_l2p = E.ms(4, 5);
  h->stats.gpu_ms_near_free = E.ms(5, 6);
  h->stats.gpu_ms_near_reac = E.ms(6, 7);
  h->stats.gpu_ms_sum = E.ms(7, 8);
  h->stats.gpu_ms_total = E.ms(0, 8);
  h->stats.gpu_ms_m2l_gemm = gemm_ran ? E.ms(10, 11) : 0.0;
  h->stats.m2l_gemm_flops = gemm_flops;
  h->stats.tune_zrot_kc = h->tune.zrot_kc;
  h->stats.tune_zrot_threads = h->tune.zrot_threads;
  h->stats.tune_zrot_ms = h->tune.zrot_ms;
  h->stats.tune_zrot_rule_ms = h->tune.zrot_rule_ms;
  h->stats.tune_zrot_candidates = (int)h->tune.zrot_trials.size();
  h->stats.n_free_pairs = (long)hc[0];
  h->stats.n_reac_pairs = (long)hc[3];
  h->stats.n_reac_nodes = (long)hc[4];
  h->stats.n_reac_surr_pairs = (long)hc[5];
  h->stats.n_reac_table_pairs = (long)hc[9 + nc];
  {
    double bx[3];
    memcpy(bx, hc + 6, sizeof(bx));
    const bool any = hc[3] > 0;
    h->stats.reac_near_rho_max = any ? bx[0] : 0.0;
    h->stats.reac_near_z_min = any ? bx[1] : 0.0;
    h->stats.reac_near_z_max = any ? bx[2] : 0.0;
  }
  h->stats.n_launches = g_fmm_launches - launches0;
  // work estimate per component (FP64-equivalent flops; used to split the
  // components over GPUs): M2L 8 complex MACs per operator entry and V pair in
  // the form the library runs, near field 30 per free-space pair and 60 per
  // contour node of a reaction pair, P2M and L2P 18 (p+1)^2 per point
  {
    const double P2 = (double)P;
    double free_pair = 0, reac_pair = 0;
    for (int n = 0; n <= p; ++n) free_pair += 2.0 * (2 * n + 1) * (2 * n + 1);
    for (int m = -p; m <= p; ++m) free_pair += (double)(p + 1 - abs(m)) * (p + 1 - abs(m));
    if (!rot_shifts) free_pair = P2 * P2;
    const double npp = (p + 1) * (p + 2) / 2.0, nmm = p * (p + 1) / 2.0;
    reac_pair = npp * npp + nmm * nmm;
    std::vector<long> vcount(nc, 0);
    for (int b = 0; b < nb; ++b) vcount[bcomp[b]] += lo_all[b + 1] - lo_all[b];
    const double nodes_per_pair = hc[3] ? (double)hc[4] / (double)hc[3] : 0.0;
    for (int c = 0; c < nc; ++c) {
      const bool reac = comps[c].kind == CK_REAC;
      const double pairs = (double)hc[9 + c];
      h->comp_work[c] = 8.0 * (reac ? reac_pair : free_pair) * vcount[c] +
                        (reac ? 60.0 * nodes_per_pair * pairs : 30.0 * pairs) +
                        18.0 * P2 * (double)(comps[c].ns + comps[c].nt);
    }
  }
}

extern "C" int fmm_layered_eval(fmm_layered_t* h, long ns, const double* src, const double* q, long nt,
                                const double* tgt, double* out, void* stream) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (ns < 0 || nt < 0 || (ns && (!src || !q)) || (nt && (!tgt || !out))) {
    h->err = "invalid argument";
    return FMM_ERR_ARG;
  }
  try {
    eval_impl(h, ns, src, q, nt, tgt, out, (cudaStream_t)stream);
  } catch (FmmError& e) {
    h->err = e.msg;
    return e.code;
  }
  h->nsrc_last = ns;
  h->ntgt_last = nt;
  return FMM_OK;
}

// Independent problems, each with its own handle, evaluated concurrently: one
// host thread per group of problems whose handles share a workspace (up to 16
// threads at a time; a handle with its own workspace is a group of one)
// drives those evaluations one after the other on one stream, so that the
// kernels of different groups overlap on the GPU while each thread waits on
// its own host steps.
extern "C" int fmm_layered_eval_batched(int n, fmm_layered_t* const* hs, const long* ns, const double* const* src,
                                        const double* const* q, const long* nt, const double* const* tgt,
                                        double* const* out, void* stream) {
  if (n < 0 || (n > 0 && (!hs || !ns || !src || !q || !nt || !tgt || !out))) return FMM_ERR_ARG;
  std::set<const fmm_layered_t*> seen;
  for (int i = 0; i < n; ++i) {
    fmm_layered* h = hs[i];
    if (!h || !seen.insert(h).second) return FMM_ERR_ARG;     // a handle serves one problem at a time
    h->err.clear();
    if (ns[i] < 0 || nt[i] < 0 || (ns[i] && (!src[i] || !q[i])) || (nt[i] && (!tgt[i] || !out[i]))) {
      h->err = "invalid argument";
      return FMM_ERR_ARG;
    }
  }
  if (n == 0) return FMM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return FMM_ERR_CUDA;
  if (cudaEventRecord(ready, st) != cudaSuccess) {
    cudaEventDestroy(ready);
    return FMM_ERR_CUDA;
  }
  std::vector<int> rc(n, FMM_OK);
  // problems whose handles share a workspace form one group, evaluated one
  // after the other by one thread on the stream of the group's first handle
  std::vector<std::vector<int>> groups;
  {
    std::map<const Workspace*, int> gi;
    for (int i = 0; i < n; ++i) {
      auto it = gi.find(hs[i]->wsp.get());
      if (it == gi.end()) {
        gi[hs[i]->wsp.get()] = (int)groups.size();
        groups.push_back({i});
      } else {
        groups[it->second].push_back(i);
      }
    }
  }
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      int g = next.fetch_add(1);
      if (g >= (int)groups.size()) break;
      cudaStream_t gst = nullptr;
      for (int i : groups[g]) {
        fmm_layered* h = hs[i];
        try {
          FMM_CHECK(cudaSetDevice(h->dev));
          if (!h->bstream) FMM_CHECK(cudaStreamCreateWithFlags(&h->bstream, cudaStreamNonBlocking));
          if (!h->bdone) FMM_CHECK(cudaEventCreateWithFlags(&h->bdone, cudaEventDisableTiming));
          if (!gst) {
            gst = h->bstream;
            FMM_CHECK(cudaStreamWaitEvent(gst, ready, 0));      // inputs written on the caller's stream
          }
          eval_impl(h, ns[i], src[i], q[i], nt[i], tgt[i], out[i], gst);
          FMM_CHECK(cudaEventRecord(h->bdone, gst));
          h->nsrc_last = ns[i];
          h->ntgt_last = nt[i];
        } catch (FmmError& e) {
          h->err = e.msg;
          rc[i] = e.code;
        } catch (std::exception& e) {
          h->err = e.what();
          rc[i] = FMM_ERR_OOM;
        }
      }
    }
  };
  int nth = std::min((int)groups.size(), 16);
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  int first = FMM_OK;
  for (int i = 0; i < n; ++i) {
    if (rc[i] == FMM_OK) {
      if (cudaStreamWaitEvent(st, hs[i]->bdone, 0) != cudaSuccess && first == FMM_OK) first = FMM_ERR_CUDA;
    } else if (first == FMM_OK) {
      first = rc[i];
    }
  }
  cudaEventDestroy(ready);
  return first;
}

extern "C" int fmm_layered_eval_host(fmm_layered_t* h, long ns, const double* src, const double* q, long nt,
                                     const double* tgt, double* out, void* stream) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (ns < 0 || nt < 0 || (ns && (!src || !q)) || (nt && (!tgt || !out))) {
    h->err = "invalid argument";
    return FMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf bs, bq, bt, bo;
  int rc = FMM_OK;
  try {
    double* ds = need<double>(bs, 3 * ns);
    double* dq = need<double>(bq, 2 * ns);
    double* dt = need<double>(bt, 3 * nt);
    double* dout = need<double>(bo, 2 * nt);
    if (ns) FMM_CHECK(cudaMemcpyAsync(ds, src, sizeof(double) * 3 * ns, cudaMemcpyHostToDevice, st));
    if (ns) FMM_CHECK(cudaMemcpyAsync(dq, q, sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, st));
    if (nt) FMM_CHECK(cudaMemcpyAsync(dt, tgt, sizeof(double) * 3 * nt, cudaMemcpyHostToDevice, st));
    eval_impl(h, ns, ds, dq, nt, dt, dout, st);
    if (nt) FMM_CHECK(cudaMemcpyAsync(out, dout, sizeof(double) * 2 * nt, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaStreamSynchronize(st));
  } catch (FmmError& e) {
    h->err = e.msg;
    rc = e.code;
  }
  bs.release(); bq.release(); bt.release(); bo.release();
  return rc;
}

// ---------------------------------------------------------------- components over GPUs
extern "C" int fmm_layered_set_components(fmm_layered_t* h, int first, int count) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (first < 0) {
    h->err = "first component must be >= 0";
    return FMM_ERR_ARG;
  }
  h->comp_first = first;
  h->comp_count = count < 0 ? -1 : count;
  return FMM_OK;
}

extern "C" int fmm_layered_component_work(const fmm_layered_t* h, double* work, int n) {
  if (!h || (n > 0 && !work)) return FMM_ERR_ARG;
  const int nc = (int)h->comp_work.size();
  if (n < nc) return FMM_ERR_ARG;
  for (int c = 0; c < nc; ++c) work[c] = h->comp_work[c];
  return nc;
}

extern "C" int fmm_layered_add_components(fmm_layered_t* h, double* out, void* stream) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (h->flags & FMM_NORM_PAPER) {
    h->err = "adding component potentials is defined in the physical normalization only (FMM_NORM_PAPER is set)";
    return FMM_ERR_UNSUPPORTED;
  }
  if (h->ntgt_last > 0 && !out) {
    h->err = "invalid argument";
    return FMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  try {
    const std::vector<Comp>& comps = h->comps;
    for (size_t c = 0; c < comps.size(); ++c)
      launch_scatter_add(comps[c].nt, h->W().tidx.as<int>() + comps[c].to, h->W().phi.as<cplx>() + comps[c].to, out, st);
    FMM_CHECK(cudaGetLastError());
  } catch (FmmError& e) {
    h->err = e.msg;
    return e.code;
  }
  return FMM_OK;
}

extern "C" int fmm_layered_measure_fp64_peak(double* gflops) {
  if (!gflops) return FMM_ERR_ARG;
  double v = measure_fp64_peak_impl();
  if (!(v > 0)) return FMM_ERR_CUDA;
  *gflops = v;
  return FMM_OK;
}

// ---------------------------------------------------------------- export
extern "C" int fmm_layered_num_components(const fmm_layered_t* h) {
  return h ? (int)h->comps.size() : FMM_ERR_ARG;
}

extern "C" int fmm_layered_component_info(const fmm_layered_t* hc, int c, long long* info, double* root) {
  fmm_layered* h = const_cast<fmm_layered*>(hc);
  if (!h || c < 0 || c >= (int)h->comps.size() || !info || !root) return FMM_ERR_ARG;
  const Comp& C_ = h->comps[c];
  std::vector<int> comp(h->nboxes);
  cudaMemcpy(comp.data(), h->W().bcomp.ptr, 4 * h->nboxes, cudaMemcpyDeviceToHost);
  std::vector<int> lev(h->nboxes);
  cudaMemcpy(lev.data(), h->W().blevel.ptr, 4 * h->nboxes, cudaMemcpyDeviceToHost);
  long nbc = 0;
  int nlev = 0;
  for (int b = 0; b < h->nboxes; ++b)
    if (comp[b] == c) { ++nbc; nlev = std::max(nlev, lev[b] + 1); }
  info[0] = C_.kind; info[1] = C_.l; info[2] = C_.lp; info[3] = C_.a; info[4] = C_.b;
  info[5] = C_.ns; info[6] = C_.nt; info[7] = nbc; info[8] = nlev; info[9] = 0;
  root[0] = C_.c[0]; root[1] = C_.c[1]; root[2] = C_.c[2]; root[3] = C_.h;
  return FMM_OK;
}

extern "C" int fmm_layered_tree_export(const fmm_layered_t* hc, int c, int* level, long long* prefix,
                                       int* src_begin, int* src_end, int* tgt_begin, int* tgt_end, int* parent,
                                       int* src_perm, int* tgt_perm, int* list_off, int* v_idx, int* u_idx,
                                       int* w_idx, int* x_idx) {
  fmm_layered* h = const_cast<fmm_layered*>(hc);
  if (!h || c < 0 || c >= (int)h->comps.size()) return FMM_ERR_ARG;
  const Comp& C_ = h->comps[c];
  // the evaluation may have run on any stream: let it finish before reading its trees
  if (cudaDeviceSynchronize() != cudaSuccess) return FMM_ERR_CUDA;
  std::vector<int> comp, lev, sb, se, tb, te, par;
  std::vector<unsigned long long> pre;
  tree_host_copy(h, comp, lev, pre, sb, se, tb, te, par);
  int nb = h->nboxes;
  std::vector<int> local(nb, -1);
  std::vector<int> glob;
  for (int b = 0; b < nb; ++b)
    if (comp[b] == c) { local[b] = (int)glob.size(); glob.push_back(b); }
  int nbc = (int)glob.size();
  for (int i = 0; i < nbc; ++i) {
    int b = glob[i];
    if (level) level[i] = lev[b];
    if (prefix) prefix[i] = (long long)pre[b];
    if (src_begin) src_begin[i] = sb[b] - (int)C_.so;
    if (src_end) src_end[i] = se[b] - (int)C_.so;
    if (tgt_begin) tgt_begin[i] = tb[b] - (int)C_.to;
    if (tgt_end) tgt_end[i] = te[b] - (int)C_.to;
    if (parent) parent[i] = par[b] < 0 ? -1 : local[par[b]];
  }
  if (src_perm && C_.ns)
    cudaMemcpy(src_perm, h->W().slocal.as<int>() + C_.so, 4 * C_.ns, cudaMemcpyDeviceToHost);
  if (tgt_perm && C_.nt)
    cudaMemcpy(tgt_perm, h->W().tlocal.as<int>() + C_.to, 4 * C_.nt, cudaMemcpyDeviceToHost);
  if (list_off) {
    std::vector<int> off(4 * (size_t)(nb + 1));
    cudaMemcpy(off.data(), h->W().loff.ptr, 4 * off.size(), cudaMemcpyDeviceToHost);
    int* idxs[4] = {v_idx, u_idx, w_idx, x_idx};
    DevBuf* bufs[4] = {&h->W().vi, &h->W().ui, &h->W().wi, &h->W().xi};
    for (int k = 0; k < 4; ++k) {
      const int* o = off.data() + (size_t)k * (nb + 1);
      std::vector<int> all(o[nb]);
      if (idxs[k] && o[nb]) cudaMemcpy(all.data(), bufs[k]->ptr, 4 * (size_t)o[nb], cudaMemcpyDeviceToHost);
      int* lo = list_off + (size_t)k * (nbc + 1);
      lo[0] = 0;
      for (int i = 0; i < nbc; ++i) {
        int b = glob[i];
        int n = o[b + 1] - o[b];
        lo[i + 1] = lo[i] + n;
        if (idxs[k])
          for (int e = 0; e < n; ++e) idxs[k][lo[i] + e] = local[all[o[b] + e]];
      }
    }
  }
  return FMM_OK;
}

// Host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "fmm_math.cuh"
#include "surrogate.cuh"
#include "near_table.cuh"
#include "../../include/fmm_layered.h"

#define FMM_CHECK(call)                                                    \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) throw FmmError(FMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct FmmError {
  int code;
  std::string msg;
  FmmError(int c, std::string m) : code(c), msg(std::move(m)) {}
};

// Growable device buffer (bytes).  Freed at destroy.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  void ensure(size_t nbytes) {
    if (nbytes <= bytes) return;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
    size_t want = nbytes + nbytes / 4 + 256;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
      ptr = nullptr;
      throw FmmError(FMM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(want) + " bytes failed");
    }
    bytes = want;
  }
  template <class T> T* as() const { return (T*)ptr; }
  // grow keeping the first `keep` bytes (stream-ordered copy)
  void grow_keep(size_t nbytes, size_t keep, cudaStream_t st) {
    if (nbytes <= bytes) return;
    size_t want = nbytes + nbytes / 2 + 256;
    void* np = nullptr;
    if (cudaMalloc(&np, want) != cudaSuccess)
      throw FmmError(FMM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(want) + " bytes failed");
    if (ptr && keep) cudaMemcpyAsync(np, ptr, keep, cudaMemcpyDeviceToDevice, st);
    if (ptr) { cudaStreamSynchronize(st); cudaFree(ptr); }
    ptr = np;
    bytes = want;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
};

enum { CK_FREE = 0, CK_REAC = 1 };

// Reaction near-field integrals are taken on the real tail up to
// ta + FMM_NEAR_TAIL_DECAY / H (H = vertical distance zt + zs of target and
// image from the interface), where the integrand has decayed below e^{-30}.
#define FMM_NEAR_TAIL_DECAY 30.0

// Layer of a point of height z (the number of interfaces above it: layer l is
// d_l < z < d_{l-1}), whether z lies exactly on an interface, and its
// distances to the interface below (z - d_l) and above (d_{l-1} - z) within
// its layer (INFINITY where the layer has none).  Shared by the
// classification of the FMM and by the allocation-free direct sum.
struct PointLayer {
  int l;
  bool on_iface;
  double gap_below, gap_above;
};
__host__ __device__ inline PointLayer classify_height(double z, const double* d, int L1) {
  PointLayer r{0, false, INFINITY, INFINITY};
  for (int j = 0; j < L1 - 1; ++j) {
    if (z == d[j]) r.on_iface = true;
    if (z < d[j]) ++r.l;
  }
  if (r.l < L1 - 1) r.gap_below = z - d[r.l];
  if (r.l > 0) r.gap_above = d[r.l - 1] - z;
  return r;
}

enum { AR_UP = 0, AR_DOWN = 1 };

// One FMM component (a free-space FMM of a layer or one reaction FMM).
struct Comp {
  int kind, l, lp, a, b;
  double ks, kt;            // source-side and target-side wave numbers
  double c[3], h;           // root box
  double dref;              // reference interface (reaction)
  int zs_lo, zs_hi, zt_lo, zt_hi;   // clamps of the integer z coordinate
  long so, ns, to, nt;      // segments in the concatenated point arrays
};

// Quadrature rule on the library's contour: Gamma1 (k_rho = -i s, 0 <= s <= b),
// Gamma2 (k_rho = t - i b, 0 <= t <= ta), Gamma3 (k_rho = ta - i s, s from b
// to 0), then the real axis [ta, ...) in panels of length `panel`.
struct Rule {
  double b = 0, ta = 0, panel = 2.0;
  int n_near = 0;           // complex nodes before the real tail
  int per_panel = 14;       // nodes per tail panel
  int n_tail_panels = 0;    // panels present
  DevBuf kr, w;             // cplx [Q]
  DevBuf kz;                // cplx [L1][Q]
  DevBuf sigma;             // cplx [L1][L1][2][2][Q]
  int Q() const { return n_near + per_panel * n_tail_panels; }
  // number of nodes needed to integrate up to t_max on the tail
  int nodes_to(double tmax) const;
  // does the rule reach t_max (no growth needed)?
  bool covers(double tmax) const { return tmax <= ta + panel * n_tail_panels; }
  // end of the tail needed by near-field pairs at vertical distance H
  double near_tmax(double H) const { return ta + FMM_NEAR_TAIL_DECAY / H; }
};

// Contour nodes of one integration (the handle's rule, or a rule built for
// one group of reaction M2L classes): kr, w [Q]; kz [L1][Q]; sigma
// [L1][L1][2][2][Q]; nodes [0, n_near) complex, the rest on the real tail.
struct RuleNodes {
  const cplx *kr, *w, *kz, *sigma;
  int Q, n_near;
};

struct Tables {             // expansion-order dependent tables built at create
  DevBuf gaunt;             // double [P][P][2p+1], G(n,m; nu,-mu; q)
  DevBuf phase;             // cplx [49][2p+1], azimuthal phases of the reaction M2L offsets
};

struct Workspace {
  // classification
  DevBuf slayer, tlayer, sorder, torder, iota, ltmp, counts, bbox, gap, flags;
  // concatenated component points, gathered (unsorted) ...
  DevBuf spos_u, sq_u, skey_u, sval_u, sidx_u, tpos_u, tkey_u, tval_u, tidx_u;
  // ... and sorted by (component, key)
  DevBuf skey, sperm, spos, sq, sidx, slocal, tkey, tperm, tpos, tidx, tlocal;
  DevBuf segs, segl, segs_keys;
  // boxes
  DevBuf bcomp, blevel, bprefix, bsb, bse, btb, bte, bparent, bchild0, bnchild, bcoord;
  DevBuf lvlcnt, lvlscan, lvl_begin;
  // lists (CSR over boxes): V, U, W, X
  DevBuf lcnt, loff, vi, ui, wi, xi;
  // expansions
  DevBuf M, L;
  // operators
  DevBuf m2l_free, m2m_op, l2l_op, m2l_reac, op_tab;
  DevBuf phi;           // per component-target results (sorted order)
  // M2L as batched GEMMs
  DevBuf g_owner, g_keys, g_vals, g_inv, g_Y, g_Z, g_runs, g_bat;
  // tensor-core M2L (mixed precision): run tables, operand tiles, scales, work items
  DevBuf tc_runs, tc_jobs, tc_a, tc_sig, tc_parts, tc_items, tc_etab;
  // rotation-form free-space M2L: run info, operator jobs, batches, run starts
  DevBuf rot_info, rot_jobs, rot_bat, rot_rs, rot_tab;
  DevBuf out_tmp;
  DevBuf sort_tmp;
  DevBuf grule;         // contour nodes of the reaction M2L groups being integrated
  DevBuf gargs;         // their radial distances and output offsets
};

// Translation operators kept across evaluations: they depend only on the box
// width of a level, the wave numbers and (reaction) the layer pair, arrows and
// the box positions relative to the interface.
struct OpCache {
  DevBuf free_buf, shift_buf, rad_buf;
  long free_used = 0, shift_used = 0, rad_used = 0;      // elements (cplx)
  long free_virtual = 0;    // class offsets of free-space operators that are not built (rotation form)
  std::map<std::pair<uint64_t, uint64_t>, long> free_m2l;              // (k, w) -> 343 slots
  std::map<std::tuple<uint64_t, uint64_t, int>, long> shift;           // (k, w, kind) -> 8 octants
  std::map<std::tuple<int, int, int, int, uint64_t, int, int, int>, long> rad;  // (l,l',a,b,w,jt,js,r)
  void clear() {
    free_used = shift_used = rad_used = free_virtual = 0;
    free_m2l.clear();
    shift.clear();
    rad.clear();
  }
};

// FP16 hi/lo copies of translation operators for the tensor-core M2L, keyed
// by (FP64 operator offset, reaction, basis block, first output row).
struct TcOpRef { long dst_off, scale_off; int N_pad, R16, RB, r0; };
struct TcCache {
  DevBuf bbuf, sbuf;                      // operator tiles (bytes), row exponents (ints)
  DevBuf phase_f;                         // FP32 copy of the rotation table e^{i m phi}
  bool phase_ready = false;
  long b_used = 0, s_used = 0, b_used_done = 0, s_done = 0;
  std::map<std::tuple<long, int, int, int>, TcOpRef> ops;
  std::vector<bool> pending_reac;
};

// Rotation form of the free-space M2L: rotation matrices of the 343 offset
// directions and the coaxial operators keyed by (k, box width, |offset|^2).
struct RotCache {
  bool ready = false;
  DevBuf w, az_buf;
  long az_used = 0;
  std::map<std::tuple<uint64_t, uint64_t, int>, long> az;
};

// Learned surrogate of the reaction components: training data, networks and
// the per-cell verdict of the held-out check.
struct SurrState {
  bool trained = false;
  double rho_max = 0, z_min = 0, z_max = 0, bound = 0;
  // winf: inference parameters [slot][2][SURR_NINF] (BF16 hi parts, then lo)
  DevBuf coef, slots, X, Y, Xh, Yh, wf, m, v, winf, gpart, acc, ok, gram, musd;
  std::vector<double> cell_err;           // [slot][64] held-out relative RMS error, -1 if not judged
  std::vector<unsigned char> cell_ok;     // [slot][64] within the bound
  void release() {
    DevBuf* all[] = {&coef, &slots, &X, &Y, &Xh, &Yh, &wf, &m, &v, &winf, &gpart, &acc, &ok, &gram, &musd};
    for (DevBuf* b : all) b->release();
  }
};

// Tabulated reaction M2L integrals (FMM_TABLES; tables.cu): the S integrals
// of every reaction component on the class rays, the CSR sums that turn them
// into operator entries, and per-evaluation job buffers.
struct TabState {
  bool built = false;
  int ntab = 0, nslot = 0;
  double kmax = 0, build_ms = 0;
  size_t bytes = 0;
  std::vector<int> slot_of;             // [(l * L1 + l') * 4 + a * 2 + b] -> slot, -1 if none
  std::vector<long> term_base;          // [(l * L1 + l') * 2 + a] -> offset into term_off, -1 if none
  DevBuf idx, vals, term_off, term_tab, term_coef, jobs, full, split_offs;
  // near-field kernel table (near_table.cuh)
  DevBuf nvals, nslot_map, ncheb;
  double near_build_ms = 0;
  void release() {
    DevBuf* all[] = {&idx, &vals, &term_off, &term_tab, &term_coef, &jobs, &full, &split_offs, &nvals, &nslot_map, &ncheb};
    for (DevBuf* b : all) b->release();
  }
};

// Tile choices of the M2L autotuner (rotation-form kernel k_zrot): made on
// the first evaluation that has free-space translations, kept per handle.
struct TuneState {
  bool zrot_done = false;
  int zrot_kc = 0, zrot_threads = 0;
  float zrot_ms = 0, zrot_rule_ms = 0;
  std::vector<float> zrot_trials;
};

struct fmm_layered {
  int L1 = 0;               // number of layers
  std::vector<double> k, d, eps;
  int p = 0, leaf = 0;
  unsigned flags = 0;
  int dev = 0;
  DevBuf d_k, d_d, d_eps;
  Rule rule;
  Tables tab;
  // device workspace of an evaluation; handles may share one
  // (fmm_layered_share_workspace), which then serializes their evaluations
  std::shared_ptr<Workspace> wsp = std::make_shared<Workspace>();
  Workspace& W() const { return *wsp; }
  OpCache cache;
  TcCache tc;
  RotCache rot;
  SurrState surr;
  TabState tabs;
  TuneState tune;
  fmm_stats_t stats{};
  std::string err;
  // components evaluated: [comp_first, comp_first + comp_count) of the full
  // ordered list (comp_count < 0: all)
  int comp_first = 0, comp_count = -1;
  // state of the last evaluation (for export)
  int n_comp_all = 0;                 // components of the full list
  int comp_first_eval = 0;            // global index of comps[0]
  std::vector<double> comp_work;      // work estimate per evaluated component
  std::vector<Comp> comps;
  std::vector<int> lvl_begin;         // global box index where each level starts
  int nboxes = 0;
  long nsrc_last = 0, ntgt_last = 0;
  // stream and completion event of this handle's problem in a batched call
  cudaStream_t bstream = nullptr;
  cudaEvent_t bdone = nullptr;
};

// Count of this library's kernel launches made by the calling host thread.
// Per thread, so that the problems of a
// batched call, each evaluated by its own host thread, count their own.
extern thread_local long g_fmm_launches;
#define LAUNCH(...) do { ++g_fmm_launches; __VA_ARGS__; } while (0)

inline void* tc_need(DevBuf& b, size_t n) {
  b.ensure(n ? n : 1);
  return b.ptr;
}

// ---- plain-data structures passed to kernels
struct SepJob { double b[3]; double k; int kind; long out_off; };
struct ReacGroup {
  int l, lp, a, b;
  double kl, klp;
  int Q;                  // quadrature nodes used (near + tail)
  double zt, zs;          // distances of the target and image box centres from the interface
  long sig_off;           // sigma^{ab}_{l l'} row in the rule's sigma array
};
struct BoxGeom { const int *comp, *lev, *sb, *se, *tb, *te, *parent, *child0, *nchild, *coord; };
struct CompGeom {
  double lo[3];          // c - h
  double h2;             // root width 2h
  double ks, kt;
  int kind, free_idx, reac_idx;
  int a;
  double dref;
};
struct OpIndex {
  const long* m2l_base;   // [comp * 23 + level] free space: offset of the 343-slot block
  const long* l2l_base;   // [comp * 23 + level] offset of the 8 L2L operators
  const long* reac_off;   // [(comp * 23 + level) * 40 + (jt * 2 + js) * 10 + r] radial reaction operator
  const cplx* phase;      // [(dy + 3) * 7 + (dx + 3)][m + p] = e^{i m atan2(dy, dx)}
  const CompGeom* cgs;
};
struct RuleView {
  const cplx *kr, *coef;   // coef[(l,l',a,b)][q] = (i/4pi) w k_rho sigma / k_lz
  const cplx* kz;          // [L1][Q]
  int Q, n_near, per_panel, n_panels;
  double ta, panel;
  SurrView surr;           // learned surrogate of the reaction components (w == nullptr: none)
  NearTabView ntab;        // tabulated near-field reaction kernel (vals == nullptr: none)
  int tail_f32;            // reaction near field: real-axis tail in FP32 (mixed form)
};
struct NearComp { int kind, l, lp, a, b; double k; double dref; long coef_off; };
struct NearBoxes {
  const int *comp, *lev, *sb, *se, *tb, *te, *parent;
  const int *uo, *ui, *wo, *wi, *xo, *xi;
  unsigned long long* comp_pairs;     // near-field pairs per component (added; may be null)
  unsigned long long* tab_pairs;      // reaction pairs taken from the kernel table (added; may be null)
};
struct DirectMedium { int L1; double k[FMM_MAXL], d[FMM_MAXL]; };


// medium.cu
void gauss_legendre_pub(int n, std::vector<double>& x, std::vector<double>& w);
void rule_init(fmm_layered* h);
void rule_extend(fmm_layered* h, double tmax, cudaStream_t st);
// nodes for the reaction M2L classes of one group: the handle's complex
// contour, then a real tail to ta + (30 + 7p)/H in panels scaled to the group
int group_tail(const fmm_layered* h, double H, double rho_max, std::vector<cplx>& kr, std::vector<cplx>& w);
void group_rule_fill(fmm_layered* h, const RuleNodes& G, cudaStream_t st);

// tables.cu: tabulated reaction M2L integrals (FMM_TABLES)
struct TabClass { int l, lp, a, b, jt, js, r; double w; long split_off; };
void tables_build(fmm_layered* h, cudaStream_t st);
bool tables_cover(const fmm_layered* h, double w);
void tables_ops(fmm_layered* h, const std::vector<TabClass>& cls, cplx* rad, cudaStream_t st);
void tables_operator_host(fmm_layered* h, const TabClass& c, double* out, cudaStream_t st);
NearTabView near_table_view(const fmm_layered* h);

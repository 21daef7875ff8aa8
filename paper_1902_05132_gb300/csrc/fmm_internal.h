// Host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fmm_math.cuh"
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
};

struct Tables {             // expansion-order dependent tables built at create
  DevBuf gaunt;             // double [P][P][2p+1], G(n,m; nu,-mu; q)
};

struct Workspace {
  // classification
  DevBuf slayer, tlayer, sorder, torder, iota, ltmp, counts, bbox, gap, flags;
  // concatenated component points, gathered (unsorted) ...
  DevBuf spos_u, sq_u, skey_u, sval_u, sidx_u, tpos_u, tkey_u, tval_u, tidx_u;
  // ... and sorted by (component, key)
  DevBuf skey, sperm, spos, sq, sidx, slocal, tkey, tperm, tpos, tidx, tlocal;
  DevBuf segs, segl;
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
  DevBuf out_tmp;
  DevBuf cub_tmp;
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
  Workspace ws;
  fmm_stats_t stats{};
  std::string err;
  // state of the last evaluation (for export)
  std::vector<Comp> comps;
  std::vector<int> lvl_begin;         // global box index where each level starts
  int nboxes = 0;
  long nsrc_last = 0, ntgt_last = 0;
};

// Count of this library's kernel launches (CUB's internal launches excluded).
extern long g_fmm_launches;
#define LAUNCH(...) do { ++g_fmm_launches; __VA_ARGS__; } while (0)

// ---- plain-data structures passed to kernels
struct SepJob { double b[3]; double k; int kind; long out_off; };
struct ReacJob {
  int l, lp, a, b;
  double kl, klp;
  int Q;                 // nodes used
  double zt, zs;         // distances of target and image centres from the interface
  double rho, phi;       // horizontal offset of the class
  long out_off;          // element offset of the operator (OpT layout)
  long sig_off;          // offset of sigma^{ab}_{l l'} in the rule's sigma array
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
struct OpIndex { const long* m2l_base; const long* l2l_base; const CompGeom* cgs; };
struct RuleView {
  const cplx *kr, *coef;   // coef[(l,l',a,b)][q] = (i/4pi) w k_rho sigma / k_lz
  const cplx* kz;          // [L1][Q]
  int Q, n_near, per_panel, n_panels;
  double ta, panel;
};
struct NearComp { int kind, l, lp, a, b; double k; double dref; long coef_off; };
struct NearBoxes { const int *comp, *lev, *sb, *se, *tb, *te, *parent; const int *uo, *ui, *wo, *wi, *xo, *xi; };
struct DirectMedium { int L1; double k[FMM_MAXL], d[FMM_MAXL]; };
struct ExpandJob { long src, dst; double phi; };

// medium.cu
void gauss_legendre_pub(int n, std::vector<double>& x, std::vector<double>& w);
void rule_init(fmm_layered* h);
void rule_extend(fmm_layered* h, double tmax, cudaStream_t st);

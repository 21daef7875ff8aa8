// Classification, equivalent polarization sources, Morton-key octrees and
// interaction lists for every FMM component of one evaluation.
//
// Definitions (identical, operation for operation, to the ones the tests
// check against):
//  * layer of a point: number of interfaces above it (layer l is
//    d_l < z < d_{l-1}); z equal to an interface is an error.
//  * components: free space for every layer holding sources and targets,
//    then reaction (l, l', a, b) in lexicographic order (arrow up = 0) for
//    every target layer l and source layer l' that hold points (eqs.
//    generalreact, totaldensity); the sources of a reaction component are the
//    equivalent polarization sources of eq. (eqpolarizedsource):
//    z* = d_l - D'_b(z') (a = up) or d_{l-1} + D'_b(z') (a = down),
//    D'_up = z' - d_l', D'_down = d_{l'-1} - z'.
//  * root box: c = (min + max) * 0.5 per axis over sources and targets, with
//    c_z = d_l (a = up) or d_{l-1} (a = down) for reaction so that the root is
//    split by the interface (Sec. 3.4); half-width
//    h = max_axis max(max - c, c - min) * (1 + 2^-20) (1 if zero).
//  * key: i = clamp(floor((x - (c - h)) * (2^21 / (2h))), 0, 2^21 - 1) per axis
//    with every operation rounded separately (no contraction), the z index of
//    reaction targets clamped to their half of the root and that of images to
//    the other half; bits interleaved x lowest.
//  * stable sort by (key, position in the component's list).
//  * a box of level l < 21 is refined when it holds more than `leaf` sources
//    or more than `leaf` targets, or, in a reaction tree, when it touches the
//    interface (the root's mid-plane) and holds any point; empty children are
//    dropped.  The second rule keeps every target leaf at least one box away
//    from every image leaf, so reaction components are evaluated entirely by
//    M2L unless points lie within 2^-21 root widths of the interface.  With
//    FMM_TREE_COUNTS the second rule is off (refinement by the counts alone),
//    and target leaves next to the interface meet image leaves in their U, W
//    and X lists: the reaction near field of eq. generalcomponentsimag.
//  * lists of a target box T (boxes with sources only, closed boxes touching
//    = adjacent): V(T) children of the parent's colleagues not adjacent to T;
//    for leaf T, U(T) source leaves adjacent to T (T included) and W(T)
//    descendants of T's colleagues whose parent is adjacent to T but which are
//    not; X(T) source leaves coarser than T adjacent to parent(T) but not to T.
//    Every list is sorted by box number.

#include <algorithm>
#include <cmath>
#include <vector>

#include "fmm_internal.h"
#include "sort.h"

#define FLAG_ON_INTERFACE 1
#define FLAG_NONFINITE 2
#define FLAG_LIST_OVERFLOW 4
#define LIST_STACK 512

__device__ __host__ inline unsigned long long enc_double(double x) {
  unsigned long long u;
  memcpy(&u, &x, 8);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}
__host__ inline double dec_double(unsigned long long e) {
  unsigned long long u = (e >> 63) ? (e & 0x7FFFFFFFFFFFFFFFULL) : ~e;
  double x;
  memcpy(&x, &u, 8);
  return x;
}

__device__ inline unsigned long long spread3(unsigned v) {
  unsigned long long x = v & 0x1FFFFF;
  x = (x | (x << 32)) & 0x1F00000000FFFFULL;
  x = (x | (x << 16)) & 0x1F0000FF0000FFULL;
  x = (x | (x << 8)) & 0x100F00F00F00F00FULL;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}
__device__ inline unsigned compact3(unsigned long long x) {
  x &= 0x1249249249249249ULL;
  x = (x ^ (x >> 2)) & 0x10C30C30C30C30C3ULL;
  x = (x ^ (x >> 4)) & 0x100F00F00F00F00FULL;
  x = (x ^ (x >> 8)) & 0x1F0000FF0000FFULL;
  x = (x ^ (x >> 16)) & 0x1F00000000FFFFULL;
  x = (x ^ (x >> 32)) & 0x1FFFFF;
  return (unsigned)x;
}
__device__ inline unsigned long long morton3(unsigned ix, unsigned iy, unsigned iz) {
  return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

// ------------------------------------------------------------- classification
// bbox layout: [set (0 src, 1 tgt)][layer][axis][min, max] (encoded doubles);
// gap layout: [set][layer][side (0: z - d_l, 1: d_{l-1} - z)] (encoded).
__global__ void k_iota(long n, int* __restrict__ out) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)i;
}

__global__ void k_classify(long n, const double* __restrict__ xyz, const double* __restrict__ q, int set,
                           int L1, const double* __restrict__ d, unsigned char* __restrict__ layer,
                           unsigned* __restrict__ counts, unsigned long long* __restrict__ bbox,
                           unsigned long long* __restrict__ gap, int* __restrict__ flags) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  bool fin = isfinite(x) && isfinite(y) && isfinite(z);
  if (q) fin = fin && isfinite(q[2 * i]) && isfinite(q[2 * i + 1]);
  if (!fin) {
    atomicOr(flags, FLAG_NONFINITE);
    layer[i] = 0;
    return;
  }
  const PointLayer pl = classify_height(z, d, L1);
  if (pl.on_iface) atomicOr(flags, FLAG_ON_INTERFACE);
  const int l = pl.l;
  layer[i] = (unsigned char)l;
  atomicAdd(&counts[set * L1 + l], 1u);
  double v[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    size_t base = (((size_t)set * L1 + l) * 3 + a) * 2;
    unsigned long long e = enc_double(v[a]);
    atomicMin(&bbox[base], e);
    atomicMax(&bbox[base + 1], e);
  }
  size_t g = ((size_t)set * L1 + l) * 2;
  if (l < L1 - 1) atomicMin(&gap[g], enc_double(pl.gap_below));
  if (l > 0) atomicMin(&gap[g + 1], enc_double(pl.gap_above));
}

// ------------------------------------------------------------- gather
struct CompDev {
  int kind, l, lp, a, b;
  double dl, dlp, dlm1, dlpm1;   // d_l, d_l', d_{l-1}, d_{l'-1} (when defined)
  double lo[3], s;               // c - h, 2^21 / (2h)
  int zlo, zhi;                  // clamp of the z index
};

__device__ inline unsigned long long point_key(const CompDev& c, double x, double y, double z) {
  double v[3] = {x, y, z};
  unsigned idx[3];
  for (int a = 0; a < 3; ++a) {
    double t = __dsub_rn(v[a], c.lo[a]);
    double u = __dmul_rn(t, c.s);
    double f = floor(u);
    if (f < 0.0) f = 0.0;
    if (f > 2097151.0) f = 2097151.0;
    idx[a] = (unsigned)f;
  }
  if ((int)idx[2] < c.zlo) idx[2] = c.zlo;
  if ((int)idx[2] > c.zhi) idx[2] = c.zhi;
  return morton3(idx[0], idx[1], idx[2]);
}

// Sources of one component: positions (images for reaction), charges, keys.
__global__ void k_gather_src(long n, const int* __restrict__ order, const double* __restrict__ xyz,
                             const double* __restrict__ q, CompDev c, long off,
                             double* __restrict__ pos, cplx* __restrict__ qo, unsigned long long* __restrict__ key,
                             int* __restrict__ val, int* __restrict__ idx) {
  long j = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  int g = order[j];
  double x = xyz[3 * g], y = xyz[3 * g + 1], z = xyz[3 * g + 2];
  if (c.kind == CK_REAC) {
    double Ds = (c.b == AR_UP) ? (z - c.dlp) : (c.dlpm1 - z);
    z = (c.a == AR_UP) ? (c.dl - Ds) : (c.dlm1 + Ds);
  }
  long o = off + j;
  pos[3 * o] = x; pos[3 * o + 1] = y; pos[3 * o + 2] = z;
  qo[o] = C(q[2 * g], q[2 * g + 1]);
  key[o] = point_key(c, x, y, z);
  val[o] = (int)o;
  idx[o] = g;
}

__global__ void k_gather_tgt(long n, const int* __restrict__ order, const double* __restrict__ xyz, CompDev c,
                             long off, double* __restrict__ pos, unsigned long long* __restrict__ key,
                             int* __restrict__ val, int* __restrict__ idx) {
  long j = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  int g = order[j];
  double x = xyz[3 * g], y = xyz[3 * g + 1], z = xyz[3 * g + 2];
  long o = off + j;
  pos[3 * o] = x; pos[3 * o + 1] = y; pos[3 * o + 2] = z;
  key[o] = point_key(c, x, y, z);
  val[o] = (int)o;
  idx[o] = g;
}

// Apply the sort permutation: out[i] = in[val[i]].
__global__ void k_permute(long n, const int* __restrict__ val, const double* __restrict__ pin,
                          const cplx* __restrict__ qin, const int* __restrict__ iin,
                          double* __restrict__ pout, cplx* __restrict__ qout, int* __restrict__ iout,
                          int* __restrict__ local_out, const long* __restrict__ seg_begin, int nseg) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = val[i];
  pout[3 * i] = pin[3 * s]; pout[3 * i + 1] = pin[3 * s + 1]; pout[3 * i + 2] = pin[3 * s + 2];
  if (qin) qout[i] = qin[s];
  iout[i] = iin[s];
  // position of the point within its component's (layer-ordered) list
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (seg_begin[mid] <= s) lo = mid; else hi = mid - 1;
  }
  local_out[i] = (int)(s - seg_begin[lo]);
}

// ------------------------------------------------------------- tree levels
__device__ inline int lower_bound_u64(const unsigned long long* a, int lo, int hi, unsigned long long v) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ inline bool refine_box(int level, int leaf, int ns, int nt, bool split_iface, int iz) {
  if (level >= 21) return false;
  if (ns > leaf || nt > leaf) return true;
  if (split_iface && ns + nt > 0) {
    if (level == 0) return true;
    int half = 1 << (level - 1);
    if (iz == half - 1 || iz == half) return true;
  }
  return false;
}

// Children of box b (one warp per box): lane o = 0..8 finds the first source
// key at or above the start of child octant o's key range (o = 8: the end of
// the box's range), lane 16 + o the same among the target keys, so child o
// holds sources [s(o), s(o+1)) and targets [t(o), t(o+1)).  The searches run
// side by side instead of one after the other.
__device__ inline unsigned child_bounds(int b, int level, const int* __restrict__ sb, const int* __restrict__ se,
                                        const int* __restrict__ tb, const int* __restrict__ te,
                                        const unsigned long long* __restrict__ prefix,
                                        const unsigned long long* __restrict__ skey,
                                        const unsigned long long* __restrict__ tkey, int lane, int* s_lo, int* s_hi,
                                        int* t_lo, int* t_hi) {
  const int shift = 3 * (21 - (level + 1));
  const unsigned long long p3 = prefix[b] << 3;
  int v = 0;
  if (lane <= 8) v = lower_bound_u64(skey, sb[b], se[b], (p3 + (unsigned long long)lane) << shift);
  else if (lane >= 16 && lane <= 24) v = lower_bound_u64(tkey, tb[b], te[b], (p3 + (unsigned long long)(lane - 16)) << shift);
  const int o = lane & 7;
  *s_lo = __shfl_sync(0xffffffffu, v, o);
  *s_hi = __shfl_sync(0xffffffffu, v, o + 1);
  *t_lo = __shfl_sync(0xffffffffu, v, 16 + o);
  *t_hi = __shfl_sync(0xffffffffu, v, 17 + o);
  // bit o set: child octant o holds a source or a target
  return __ballot_sync(0xffffffffu, lane < 8 && (*s_hi > *s_lo || *t_hi > *t_lo)) & 0xFFu;
}

__global__ void k_count_children(int lb, int le, int level, int leaf, const int* __restrict__ sb,
                                 const int* __restrict__ se, const int* __restrict__ tb,
                                 const int* __restrict__ te, const unsigned long long* __restrict__ prefix,
                                 const unsigned long long* __restrict__ skey,
                                 const unsigned long long* __restrict__ tkey, int* __restrict__ nchild,
                                 const int* __restrict__ comp, const int* __restrict__ comp_kind,
                                 const int* __restrict__ coord, int split_iface) {
  const int b = lb + (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= le) return;                       // whole warps leave together
  const int ns = se[b] - sb[b], nt = te[b] - tb[b];
  int cnt = 0;
  if (refine_box(level, leaf, ns, nt, split_iface && comp_kind[comp[b]] == CK_REAC, coord[3 * b + 2])) {
    int s0, s1, t0, t1;
    cnt = __popc(child_bounds(b, level, sb, se, tb, te, prefix, skey, tkey, lane, &s0, &s1, &t0, &t1));
  }
  if (lane == 0) nchild[b - lb] = cnt;
}

__global__ void k_write_children(int lb, int le, int level, int nb_next_base, const int* __restrict__ scan,
                                 const int* __restrict__ nchild_lvl, int* __restrict__ comp,
                                 int* __restrict__ lev, unsigned long long* __restrict__ prefix,
                                 int* __restrict__ sb, int* __restrict__ se, int* __restrict__ tb,
                                 int* __restrict__ te, int* __restrict__ parent, int* __restrict__ child0,
                                 int* __restrict__ nchild, int* __restrict__ coord,
                                 const unsigned long long* __restrict__ skey,
                                 const unsigned long long* __restrict__ tkey) {
  const int b = lb + (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= le) return;
  const int n = nchild_lvl[b - lb];
  const int base = nb_next_base + scan[b - lb];
  if (lane == 0) {
    child0[b] = n ? base : -1;
    nchild[b] = n;
  }
  if (!n) return;
  int s0, s1, t0, t1;
  const unsigned mask = child_bounds(b, level, sb, se, tb, te, prefix, skey, tkey, lane, &s0, &s1, &t0, &t1);
  if (lane < 8 && ((mask >> lane) & 1u)) {
    const int c = base + __popc(mask & ((1u << lane) - 1u));
    const unsigned long long cp = (prefix[b] << 3) | (unsigned long long)lane;
    comp[c] = comp[b];
    lev[c] = level + 1;
    prefix[c] = cp;
    sb[c] = s0; se[c] = s1; tb[c] = t0; te[c] = t1;
    parent[c] = b;
    coord[3 * c] = compact3(cp);
    coord[3 * c + 1] = compact3(cp >> 1);
    coord[3 * c + 2] = compact3(cp >> 2);
  }
}

// ------------------------------------------------------------- lists
struct TreeView {
  const int *comp, *lev, *sb, *se, *tb, *te, *parent, *child0, *nchild, *coord;
  const unsigned long long* prefix;
  const int* lvl_begin;   // [23]
};

__device__ inline int find_box(const TreeView& T, int comp, int level, int ix, int iy, int iz) {
  int n = 1 << level;
  if (ix < 0 || iy < 0 || iz < 0 || ix >= n || iy >= n || iz >= n) return -1;
  unsigned long long key = morton3(ix, iy, iz);
  int lo = T.lvl_begin[level], hi = T.lvl_begin[level + 1];
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int cm = T.comp[mid];
    if (cm < comp || (cm == comp && T.prefix[mid] < key)) lo = mid + 1; else hi = mid;
  }
  if (lo < T.lvl_begin[level + 1] && T.comp[lo] == comp && T.prefix[lo] == key) return lo;
  return -1;
}

__device__ inline bool adjacent(const TreeView& T, int b1, int b2) {
  int l1 = T.lev[b1], l2 = T.lev[b2];
  int L = max(l1, l2);
  long f1 = 1L << (L - l1), f2 = 1L << (L - l2);
  for (int a = 0; a < 3; ++a) {
    long lo1 = (long)T.coord[3 * b1 + a] * f1, hi1 = lo1 + f1;
    long lo2 = (long)T.coord[3 * b2 + a] * f2, hi2 = lo2 + f2;
    if (lo1 > hi2 || lo2 > hi1) return false;
  }
  return true;
}

__device__ inline bool is_leaf(const TreeView& T, int b) { return T.nchild[b] == 0; }
__device__ inline bool has_src(const TreeView& T, int b) { return T.se[b] > T.sb[b]; }

template <bool FILL>
__device__ inline void emit(int* out, int& n, int v) {
  if (FILL) out[n] = v;
  ++n;
}

__device__ inline void sort_ints(int* a, int n) {
  for (int i = 1; i < n; ++i) {
    int v = a[i], j = i - 1;
    while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
    a[j + 1] = v;
  }
}

// pass 0: counts into cnt[4][nb]; pass 1: fill lists at the given offsets.
template <bool FILL>
__global__ void k_lists(int nb, TreeView T, int* __restrict__ cnt, const int* __restrict__ vo,
                        const int* __restrict__ uo, const int* __restrict__ wo, const int* __restrict__ xo,
                        int* __restrict__ vi, int* __restrict__ ui, int* __restrict__ wi, int* __restrict__ xi,
                        int* __restrict__ flags) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nb) return;
  int nv = 0, nu = 0, nw = 0, nx = 0;
  int* V = FILL ? vi + vo[t] : nullptr;
  int* U = FILL ? ui + uo[t] : nullptr;
  int* W = FILL ? wi + wo[t] : nullptr;
  int* X = FILL ? xi + xo[t] : nullptr;
  if (T.te[t] > T.tb[t]) {
    int comp = T.comp[t], l = T.lev[t];
    if (l >= 2) {
      int P = T.parent[t];
      int px = T.coord[3 * P], py = T.coord[3 * P + 1], pz = T.coord[3 * P + 2];
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int Cb = find_box(T, comp, l - 1, px + dx, py + dy, pz + dz);
            if (Cb < 0) continue;
            for (int k = 0; k < T.nchild[Cb]; ++k) {
              int S = T.child0[Cb] + k;
              if (has_src(T, S) && !adjacent(T, S, t)) emit<FILL>(V, nv, S);
            }
          }
      // X list: leaves coarser than t adjacent to parent(t) but not to t
      for (int A = P; A >= 0 && T.lev[A] >= 1; A = T.parent[A]) {
        int ax = T.coord[3 * A], ay = T.coord[3 * A + 1], az = T.coord[3 * A + 2], la = T.lev[A];
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dx && !dy && !dz) continue;
              int S = find_box(T, comp, la, ax + dx, ay + dy, az + dz);
              if (S < 0 || !is_leaf(T, S) || !has_src(T, S)) continue;
              if (adjacent(T, S, P) && !adjacent(T, S, t)) emit<FILL>(X, nx, S);
            }
      }
    }
    if (is_leaf(T, t)) {
      int stack[LIST_STACK];
      int sp = 0;
      int tx = T.coord[3 * t], ty = T.coord[3 * t + 1], tz = T.coord[3 * t + 2];
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int Cb = find_box(T, comp, l, tx + dx, ty + dy, tz + dz);
            if (Cb < 0) continue;
            if (is_leaf(T, Cb)) {
              if (has_src(T, Cb)) emit<FILL>(U, nu, Cb);
            } else if (sp < LIST_STACK) {
              stack[sp++] = Cb;
            } else {
              atomicOr(flags, FLAG_LIST_OVERFLOW);
            }
          }
      while (sp > 0) {
        int Cb = stack[--sp];
        for (int k = 0; k < T.nchild[Cb]; ++k) {
          int S = T.child0[Cb] + k;
          if (adjacent(T, S, t)) {
            if (is_leaf(T, S)) {
              if (has_src(T, S)) emit<FILL>(U, nu, S);
            } else if (sp < LIST_STACK) {
              stack[sp++] = S;
            } else {
              atomicOr(flags, FLAG_LIST_OVERFLOW);
            }
          } else if (has_src(T, S)) {
            emit<FILL>(W, nw, S);
          }
        }
      }
      for (int A = T.parent[t]; A >= 0 && T.lev[A] >= 1; A = T.parent[A]) {
        int ax = T.coord[3 * A], ay = T.coord[3 * A + 1], az = T.coord[3 * A + 2], la = T.lev[A];
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dx && !dy && !dz) continue;
              int S = find_box(T, comp, la, ax + dx, ay + dy, az + dz);
              if (S < 0 || !is_leaf(T, S) || !has_src(T, S)) continue;
              if (adjacent(T, S, t)) emit<FILL>(U, nu, S);
            }
      }
    }
  }
  if (FILL) {
    sort_ints(V, nv);
    sort_ints(U, nu);
    sort_ints(W, nw);
    sort_ints(X, nx);
  } else {
    cnt[t] = nv;
    cnt[nb + t] = nu;
    cnt[2 * nb + t] = nw;
    cnt[3 * nb + t] = nx;
  }
}

// ------------------------------------------------------------- host driver
template <class T>
static T* need(DevBuf& b, size_t n) {
  b.ensure(sizeof(T) * (n ? n : 1));
  return b.as<T>();
}

// off[k][b] = all[k nb + b] - all[k nb] for b <= nb (list k's CSR offsets
// from the scan of the four lists' counts); tot[k] = off[k][nb]
__global__ void k_list_offsets(int nb, const int* __restrict__ all, int* __restrict__ off, int* __restrict__ tot) {
  long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= 4 * ((long)nb + 1)) return;
  const int k = (int)(e / (nb + 1)), b = (int)(e % (nb + 1));
  const int v = all[(long)k * nb + b] - all[(long)k * nb];
  off[e] = v;
  if (b == nb) tot[k] = v;
}

static void exclusive_scan(Workspace& ws, const int* in, int* out, long n, cudaStream_t st) {
  dev_exclusive_scan(in, out, n, ws.sort_tmp, st);
}

// keys for the stable partition of points by layer: (layer, position)
__global__ void k_layer_keys(long n, const unsigned char* __restrict__ layer, unsigned long long* __restrict__ key,
                             int* __restrict__ val) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = layer[i];
  val[i] = (int)i;
}

// component of each sorted point (by its position in the concatenated,
// component-ordered list) as the key of the last, stable pass
__global__ void k_comp_keys(long n, const int* __restrict__ pos, const long* __restrict__ seg_begin, int nseg,
                            unsigned long long* __restrict__ key) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = pos[i];
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (seg_begin[mid] <= s) lo = mid; else hi = mid - 1;
  }
  key[i] = (unsigned long long)lo;
}

__global__ void k_gather_keys(long n, const int* __restrict__ pos, const unsigned long long* __restrict__ in,
                              unsigned long long* __restrict__ out) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[pos[i]];
}

struct ClassifyOut {
  std::vector<unsigned> counts;           // [2][L1]
  std::vector<double> bbox;               // [2][L1][3][2]
  std::vector<double> gap;                // [2][L1][2]
};

// Host copy of the box arrays of the last evaluation (used by the export).
void tree_host_copy(fmm_layered* h, std::vector<int>& comp, std::vector<int>& lev,
                    std::vector<unsigned long long>& prefix, std::vector<int>& sb, std::vector<int>& se,
                    std::vector<int>& tb, std::vector<int>& te, std::vector<int>& parent) {
  Workspace& ws = h->W();
  int nb = h->nboxes;
  comp.resize(nb); lev.resize(nb); prefix.resize(nb); sb.resize(nb); se.resize(nb);
  tb.resize(nb); te.resize(nb); parent.resize(nb);
  cudaMemcpy(comp.data(), ws.bcomp.ptr, 4 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(lev.data(), ws.blevel.ptr, 4 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(prefix.data(), ws.bprefix.ptr, 8 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(sb.data(), ws.bsb.ptr, 4 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(se.data(), ws.bse.ptr, 4 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(tb.data(), ws.btb.ptr, 4 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(te.data(), ws.bte.ptr, 4 * nb, cudaMemcpyDeviceToHost);
  cudaMemcpy(parent.data(), ws.bparent.ptr, 4 * nb, cudaMemcpyDeviceToHost);
}

// Build all component trees and lists.  Returns the classification summary
// through `gap_out` ([2][L1][2] minimal distances to interfaces).
void build_trees(fmm_layered* h, long ns, const double* src, const double* q, long nt, const double* tgt,
                 std::vector<double>& gap_out, cudaStream_t st) {
  Workspace& ws = h->W();
  const int L1 = h->L1;
  // ---- classification
  unsigned char* sl = need<unsigned char>(ws.slayer, ns);
  unsigned char* tl = need<unsigned char>(ws.tlayer, nt);
  unsigned* counts = need<unsigned>(ws.counts, 2 * L1);
  unsigned long long* bbox = need<unsigned long long>(ws.bbox, 2 * L1 * 6);
  unsigned long long* gap = need<unsigned long long>(ws.gap, 2 * L1 * 2);
  int* flags = need<int>(ws.flags, 1);
  {
    std::vector<unsigned long long> init(2 * L1 * 6);
    for (int i = 0; i < 2 * L1 * 3; ++i) {
      init[2 * i] = ~0ULL;
      init[2 * i + 1] = 0ULL;
    }
    std::vector<unsigned long long> ginit(2 * L1 * 2, ~0ULL);
    FMM_CHECK(cudaMemcpyAsync(bbox, init.data(), 8 * init.size(), cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(gap, ginit.data(), 8 * ginit.size(), cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemsetAsync(counts, 0, 4 * 2 * L1, st));
    FMM_CHECK(cudaMemsetAsync(flags, 0, 4, st));
  }
  if (ns) LAUNCH(k_classify<<<(ns + 255) / 256, 256, 0, st>>>(ns, src, q, 0, L1, h->d_d.as<double>(), sl, counts, bbox, gap, flags));
  if (nt) LAUNCH(k_classify<<<(nt + 255) / 256, 256, 0, st>>>(nt, tgt, nullptr, 1, L1, h->d_d.as<double>(), tl, counts, bbox, gap, flags));
  FMM_CHECK(cudaGetLastError());
  // stable partition of points by layer
  int* sorder = need<int>(ws.sorder, ns);
  int* torder = need<int>(ws.torder, nt);
  {
    // stable radix sort on the layer byte, values = positions
    const long ni = std::max(ns, nt);
    unsigned long long* kbuf = need<unsigned long long>(ws.ltmp, 2 * (size_t)ni);
    int* vbuf = need<int>(ws.iota, ni);
    for (int set = 0; set < 2; ++set) {
      long n = set ? nt : ns;
      if (!n) continue;
      LAUNCH(k_layer_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, set ? tl : sl, kbuf, vbuf));
      dev_sort_pairs(kbuf, vbuf, kbuf + ni, set ? torder : sorder, n, 0, 8, ws.sort_tmp, st);
    }
  }
  ClassifyOut co;
  co.counts.resize(2 * L1);
  std::vector<unsigned long long> hb(2 * L1 * 6), hg(2 * L1 * 2);
  int hflags = 0;
  FMM_CHECK(cudaMemcpyAsync(co.counts.data(), counts, 4 * 2 * L1, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(hb.data(), bbox, 8 * hb.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(hg.data(), gap, 8 * hg.size(), cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  if (hflags & FLAG_NONFINITE) throw FmmError(FMM_ERR_NONFINITE, "non-finite coordinate or charge");
  if (hflags & FLAG_ON_INTERFACE) throw FmmError(FMM_ERR_ON_INTERFACE, "a point lies exactly on an interface");
  co.bbox.resize(hb.size());
  for (size_t i = 0; i < hb.size(); ++i) co.bbox[i] = dec_double(hb[i]);
  gap_out.resize(hg.size());
  for (size_t i = 0; i < hg.size(); ++i) gap_out[i] = (hg[i] == ~0ULL) ? INFINITY : dec_double(hg[i]);
  std::vector<long> soff(L1 + 1, 0), toff(L1 + 1, 0);
  for (int l = 0; l < L1; ++l) {
    soff[l + 1] = soff[l] + co.counts[l];
    toff[l + 1] = toff[l] + co.counts[L1 + l];
  }
  auto BB = [&](int set, int l, int axis, int mm) { return co.bbox[(((size_t)set * L1 + l) * 3 + axis) * 2 + mm]; };
  // ---- components (fixed order)
  std::vector<Comp>& comps = h->comps;
  comps.clear();
  const double* dd = h->d.data();
  for (int l = 0; l < L1; ++l)
    if (co.counts[l] && co.counts[L1 + l]) {
      Comp c{};
      c.kind = CK_FREE; c.l = c.lp = l; c.a = c.b = 0;
      c.ks = c.kt = h->k[l];
      c.ns = co.counts[l]; c.nt = co.counts[L1 + l];
      comps.push_back(c);
    }
  if (L1 > 1)
    for (int l = 0; l < L1; ++l) {
      if (!co.counts[L1 + l]) continue;
      for (int lp = 0; lp < L1; ++lp) {
        if (!co.counts[lp]) continue;
        for (int a = 0; a < 2; ++a) {
          if (a == AR_UP ? !(l < L1 - 1) : !(l > 0)) continue;
          for (int b = 0; b < 2; ++b) {
            if (b == AR_UP ? !(lp < L1 - 1) : !(lp > 0)) continue;
            Comp c{};
            c.kind = CK_REAC; c.l = l; c.lp = lp; c.a = a; c.b = b;
            c.ks = h->k[lp]; c.kt = h->k[l];
            c.ns = co.counts[lp]; c.nt = co.counts[L1 + l];
            comps.push_back(c);
          }
        }
      }
    }
  // the selected range of components (fmm_layered_set_components)
  h->n_comp_all = (int)comps.size();
  {
    const int first = std::min(std::max(h->comp_first, 0), h->n_comp_all);
    const int last = h->comp_count < 0 ? h->n_comp_all : std::min(h->n_comp_all, first + h->comp_count);
    comps = std::vector<Comp>(comps.begin() + first, comps.begin() + std::max(first, last));
    h->comp_first_eval = first;
  }
  const int nc = (int)comps.size();
  if (nc == 0) {
    h->nboxes = 0;
    h->lvl_begin.assign(23, 0);
    h->stats.n_components = 0;
    h->stats.n_boxes = 0;
    h->stats.max_level = 0;
    h->stats.n_v_pairs = 0;
    return;
  }
  long so = 0, to = 0;
  std::vector<CompDev> cdev(nc);
  for (int ci = 0; ci < nc; ++ci) {
    Comp& c = comps[ci];
    c.so = so; c.to = to;
    so += c.ns; to += c.nt;
    int sl_ = (c.kind == CK_FREE) ? c.l : c.lp;
    double mn[3], mx[3];
    for (int a = 0; a < 2; ++a) {
      mn[a] = std::min(BB(0, sl_, a, 0), BB(1, c.l, a, 0));
      mx[a] = std::max(BB(0, sl_, a, 1), BB(1, c.l, a, 1));
    }
    double smn = BB(0, sl_, 2, 0), smx = BB(0, sl_, 2, 1);
    if (c.kind == CK_REAC) {
      // image z is monotone in z': evaluate the map at the extremes
      auto img = [&](double z) {
        double Ds = (c.b == AR_UP) ? (z - dd[c.lp]) : (dd[c.lp - 1] - z);
        return (c.a == AR_UP) ? (dd[c.l] - Ds) : (dd[c.l - 1] + Ds);
      };
      double i0 = img(smn), i1 = img(smx);
      smn = std::min(i0, i1);
      smx = std::max(i0, i1);
    }
    mn[2] = std::min(smn, BB(1, c.l, 2, 0));
    mx[2] = std::max(smx, BB(1, c.l, 2, 1));
    for (int a = 0; a < 3; ++a) c.c[a] = (mn[a] + mx[a]) * 0.5;
    if (c.kind == CK_REAC) {
      c.dref = (c.a == AR_UP) ? dd[c.l] : dd[c.l - 1];
      c.c[2] = c.dref;
    }
    double hh = 0;
    for (int a = 0; a < 3; ++a) hh = std::max(hh, std::max(mx[a] - c.c[a], c.c[a] - mn[a]));
    hh = hh * (1.0 + 9.5367431640625e-07);
    if (hh == 0.0) hh = 1.0;
    c.h = hh;
    const int half = 1 << 20;
    if (c.kind == CK_REAC) {
      if (c.a == AR_UP) { c.zt_lo = half; c.zt_hi = 2 * half - 1; c.zs_lo = 0; c.zs_hi = half - 1; }
      else { c.zt_lo = 0; c.zt_hi = half - 1; c.zs_lo = half; c.zs_hi = 2 * half - 1; }
    } else {
      c.zt_lo = c.zs_lo = 0;
      c.zt_hi = c.zs_hi = 2 * half - 1;
    }
    CompDev& cd = cdev[ci];
    cd.kind = c.kind; cd.l = c.l; cd.lp = c.lp; cd.a = c.a; cd.b = c.b;
    cd.dl = (c.l < L1 - 1) ? dd[c.l] : 0; cd.dlm1 = (c.l > 0) ? dd[c.l - 1] : 0;
    cd.dlp = (c.lp < L1 - 1) ? dd[c.lp] : 0; cd.dlpm1 = (c.lp > 0) ? dd[c.lp - 1] : 0;
    for (int a = 0; a < 3; ++a) cd.lo[a] = c.c[a] - c.h;
    cd.s = 2097152.0 / (2.0 * c.h);
  }
  const long NS = so, NT = to;
  // ---- gather points per component
  double* spos_u = need<double>(ws.spos_u, 3 * NS);
  cplx* sq_u = need<cplx>(ws.sq_u, NS);
  unsigned long long* skey_u = need<unsigned long long>(ws.skey_u, NS);
  int* sval_u = need<int>(ws.sval_u, NS);
  int* sidx_u = need<int>(ws.sidx_u, NS);
  double* tpos_u = need<double>(ws.tpos_u, 3 * NT);
  unsigned long long* tkey_u = need<unsigned long long>(ws.tkey_u, NT);
  int* tval_u = need<int>(ws.tval_u, NT);
  int* tidx_u = need<int>(ws.tidx_u, NT);
  for (int ci = 0; ci < nc; ++ci) {
    Comp& c = comps[ci];
    CompDev cs = cdev[ci];
    int sl_ = (c.kind == CK_FREE) ? c.l : c.lp;
    cs.zlo = c.zs_lo; cs.zhi = c.zs_hi;
    if (c.ns) LAUNCH(k_gather_src<<<(c.ns + 255) / 256, 256, 0, st>>>(c.ns, sorder + soff[sl_], src, q, cs, c.so, spos_u, sq_u, skey_u, sval_u, sidx_u));
    CompDev ct = cdev[ci];
    ct.zlo = c.zt_lo; ct.zhi = c.zt_hi;
    if (c.nt) LAUNCH(k_gather_tgt<<<(c.nt + 255) / 256, 256, 0, st>>>(c.nt, torder + toff[c.l], tgt, ct, c.to, tpos_u, tkey_u, tval_u, tidx_u));
  }
  FMM_CHECK(cudaGetLastError());
  // ---- segmented stable sort by key (radix sort is stable; values are the
  // positions in the component's layer-ordered list)
  std::vector<int> segSi(nc + 1), segTi(nc + 1);
  std::vector<long> segS(nc + 1), segT(nc + 1);
  for (int ci = 0; ci < nc; ++ci) {
    segS[ci] = comps[ci].so; segT[ci] = comps[ci].to;
    segSi[ci] = (int)comps[ci].so; segTi[ci] = (int)comps[ci].to;
  }
  segS[nc] = NS; segT[nc] = NT; segSi[nc] = (int)NS; segTi[nc] = (int)NT;
  int* dsegs = need<int>(ws.segs, 2 * (nc + 1));
  long* dsegl = need<long>(ws.segl, 2 * (nc + 1));
  FMM_CHECK(cudaMemcpyAsync(dsegs, segSi.data(), 4 * (nc + 1), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(dsegs + nc + 1, segTi.data(), 4 * (nc + 1), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(dsegl, segS.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
  FMM_CHECK(cudaMemcpyAsync(dsegl + nc + 1, segT.data(), 8 * (nc + 1), cudaMemcpyHostToDevice, st));
  unsigned long long* skey = need<unsigned long long>(ws.skey, NS);
  unsigned long long* tkey = need<unsigned long long>(ws.tkey, NT);
  int* sperm = need<int>(ws.sperm, NS);
  int* tperm = need<int>(ws.tperm, NT);
  for (int set = 0; set < 2; ++set) {
    // stable sort by the 63-bit key, then (stable) by component: the order
    // (component, key, position in the component's list)
    long n = set ? NT : NS;
    if (!n) continue;
    unsigned long long* ku = set ? tkey_u : skey_u;
    unsigned long long* kd = set ? tkey : skey;
    int* vu = set ? tval_u : sval_u;
    int* vd = set ? tperm : sperm;
    // keep the unsorted keys: the passes overwrite their input
    unsigned long long* kcopy = need<unsigned long long>(ws.segs_keys, 2 * (size_t)n);
    FMM_CHECK(cudaMemcpyAsync(kcopy, ku, 8 * (size_t)n, cudaMemcpyDeviceToDevice, st));
    dev_sort_pairs(kcopy, vu, kd, vd, n, 0, 63, ws.sort_tmp, st);
    if (nc > 1) {
      unsigned long long* ck = kcopy + n;
      LAUNCH(k_comp_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, vd, dsegl + (set ? nc + 1 : 0), nc, ck));
      FMM_CHECK(cudaMemcpyAsync(vu, vd, 4 * (size_t)n, cudaMemcpyDeviceToDevice, st));
      dev_sort_pairs(ck, vu, kcopy, vd, n, 0, nc > 256 ? 16 : 8, ws.sort_tmp, st);
      LAUNCH(k_gather_keys<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, vd, ku, kd));
    }
  }
  double* spos = need<double>(ws.spos, 3 * NS);
  cplx* sqs = need<cplx>(ws.sq, NS);
  int* sidx = need<int>(ws.sidx, NS);
  int* slocal = need<int>(ws.slocal, NS);
  double* tpos = need<double>(ws.tpos, 3 * NT);
  int* tidx = need<int>(ws.tidx, NT);
  int* tlocal = need<int>(ws.tlocal, NT);
  if (NS) LAUNCH(k_permute<<<(NS + 255) / 256, 256, 0, st>>>(NS, sperm, spos_u, sq_u, sidx_u, spos, sqs, sidx, slocal, dsegl, nc));
  if (NT) LAUNCH(k_permute<<<(NT + 255) / 256, 256, 0, st>>>(NT, tperm, tpos_u, nullptr, tidx_u, tpos, nullptr, tidx, tlocal, dsegl + nc + 1, nc));
  FMM_CHECK(cudaGetLastError());

  // ---- tree levels
  size_t cap = std::max<size_t>(4096, (size_t)(2 * (NS + NT) / std::max(1, h->leaf) + 16 * nc));
  auto grow_boxes = [&](size_t need_boxes, size_t keep) {
    if (need_boxes * 4 <= ws.bcomp.bytes && need_boxes * 12 <= ws.bcoord.bytes) return;
    size_t n = std::max(need_boxes, cap);
    ws.bcomp.grow_keep(4 * n, 4 * keep, st);
    ws.blevel.grow_keep(4 * n, 4 * keep, st);
    ws.bprefix.grow_keep(8 * n, 8 * keep, st);
    ws.bsb.grow_keep(4 * n, 4 * keep, st);
    ws.bse.grow_keep(4 * n, 4 * keep, st);
    ws.btb.grow_keep(4 * n, 4 * keep, st);
    ws.bte.grow_keep(4 * n, 4 * keep, st);
    ws.bparent.grow_keep(4 * n, 4 * keep, st);
    ws.bchild0.grow_keep(4 * n, 4 * keep, st);
    ws.bnchild.grow_keep(4 * n, 4 * keep, st);
    ws.bcoord.grow_keep(12 * n, 12 * keep, st);
    cap = n;
  };
  grow_boxes(cap, 0);
  {
    std::vector<int> comp(nc), lev(nc, 0), sb(nc), se(nc), tb(nc), te(nc), par(nc, -1), coord(3 * nc, 0);
    std::vector<unsigned long long> pre(nc, 0);
    for (int ci = 0; ci < nc; ++ci) {
      comp[ci] = ci;
      sb[ci] = (int)comps[ci].so; se[ci] = (int)(comps[ci].so + comps[ci].ns);
      tb[ci] = (int)comps[ci].to; te[ci] = (int)(comps[ci].to + comps[ci].nt);
    }
    FMM_CHECK(cudaMemcpyAsync(ws.bcomp.ptr, comp.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.blevel.ptr, lev.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.bprefix.ptr, pre.data(), 8 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.bsb.ptr, sb.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.bse.ptr, se.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.btb.ptr, tb.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.bte.ptr, te.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.bparent.ptr, par.data(), 4 * nc, cudaMemcpyHostToDevice, st));
    FMM_CHECK(cudaMemcpyAsync(ws.bcoord.ptr, coord.data(), 12 * nc, cudaMemcpyHostToDevice, st));
  }
  std::vector<int> kinds(nc);
  for (int ci = 0; ci < nc; ++ci) kinds[ci] = comps[ci].kind;
  int* dkind = need<int>(ws.ltmp, nc);
  FMM_CHECK(cudaMemcpyAsync(dkind, kinds.data(), 4 * nc, cudaMemcpyHostToDevice, st));
  std::vector<int>& lvl = h->lvl_begin;
  lvl.assign(1, 0);
  lvl.push_back(nc);
  int level = 0;
  while (true) {
    int lb = lvl[level], le = lvl[level + 1];
    int n = le - lb;
    if (n == 0) break;
    int* cntl = need<int>(ws.lvlcnt, n + 1);
    int* scn = need<int>(ws.lvlscan, n + 1);
    LAUNCH(k_count_children<<<(n + 3) / 4, 128, 0, st>>>(lb, le, level, h->leaf, ws.bsb.as<int>(), ws.bse.as<int>(),
                                                      ws.btb.as<int>(), ws.bte.as<int>(), ws.bprefix.as<unsigned long long>(),
                                                      skey, tkey, cntl, ws.bcomp.as<int>(), dkind, ws.bcoord.as<int>(),
                                                      (h->flags & FMM_TREE_COUNTS) ? 0 : 1));
    exclusive_scan(ws, cntl, scn, n, st);
    int last_cnt = 0, last_scan = 0;
    FMM_CHECK(cudaMemcpyAsync(&last_cnt, cntl + n - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaMemcpyAsync(&last_scan, scn + n - 1, 4, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaStreamSynchronize(st));
    int total = last_cnt + last_scan;
    grow_boxes((size_t)le + total, (size_t)le);
    LAUNCH(k_write_children<<<(n + 3) / 4, 128, 0, st>>>(lb, le, level, le, scn, cntl, ws.bcomp.as<int>(), ws.blevel.as<int>(),
                                                      ws.bprefix.as<unsigned long long>(), ws.bsb.as<int>(), ws.bse.as<int>(),
                                                      ws.btb.as<int>(), ws.bte.as<int>(), ws.bparent.as<int>(),
                                                      ws.bchild0.as<int>(), ws.bnchild.as<int>(), ws.bcoord.as<int>(), skey, tkey));
    FMM_CHECK(cudaGetLastError());
    if (total == 0) break;
    lvl.push_back(le + total);
    ++level;
  }
  h->nboxes = lvl.back();
  while ((int)lvl.size() < 23) lvl.push_back(h->nboxes);
  const int nb = h->nboxes;
  // ---- lists
  int* dlvl = need<int>(ws.lvl_begin, 23);
  FMM_CHECK(cudaMemcpyAsync(dlvl, lvl.data(), 4 * 23, cudaMemcpyHostToDevice, st));
  TreeView T;
  T.comp = ws.bcomp.as<int>(); T.lev = ws.blevel.as<int>(); T.sb = ws.bsb.as<int>(); T.se = ws.bse.as<int>();
  T.tb = ws.btb.as<int>(); T.te = ws.bte.as<int>(); T.parent = ws.bparent.as<int>(); T.child0 = ws.bchild0.as<int>();
  T.nchild = ws.bnchild.as<int>(); T.coord = ws.bcoord.as<int>(); T.prefix = ws.bprefix.as<unsigned long long>();
  T.lvl_begin = dlvl;
  int* cnt = need<int>(ws.lcnt, 4 * (size_t)nb + 4);
  int* off = need<int>(ws.loff, 4 * ((size_t)nb + 1));
  FMM_CHECK(cudaMemsetAsync(flags, 0, 4, st));
  LAUNCH(k_lists<false><<<(nb + 127) / 128, 128, 0, st>>>(nb, T, cnt, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr, nullptr, flags));
  FMM_CHECK(cudaGetLastError());
  // offsets of the four lists: one scan over the counts of all four
  // (cnt[4][nb], then one zero), each list's offsets relative to its start
  FMM_CHECK(cudaMemsetAsync(cnt + (size_t)4 * nb, 0, 4, st));
  int* scanall = need<int>(ws.lvlscan, 4 * (size_t)nb + 8);
  int* dtot = scanall + 4 * (size_t)nb + 1;
  exclusive_scan(ws, cnt, scanall, 4 * (long)nb + 1, st);
  LAUNCH(k_list_offsets<<<(unsigned)((4 * ((long)nb + 1) + 255) / 256), 256, 0, st>>>(nb, scanall, off, dtot));
  std::vector<int> tot(4);
  FMM_CHECK(cudaMemcpyAsync(tot.data(), dtot, 16, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  int* vi = need<int>(ws.vi, tot[0]);
  int* ui = need<int>(ws.ui, tot[1]);
  int* wi = need<int>(ws.wi, tot[2]);
  int* xi = need<int>(ws.xi, tot[3]);
  LAUNCH(k_lists<true><<<(nb + 127) / 128, 128, 0, st>>>(nb, T, nullptr, off, off + (nb + 1), off + 2 * (size_t)(nb + 1),
                                                  off + 3 * (size_t)(nb + 1), vi, ui, wi, xi, flags));
  FMM_CHECK(cudaGetLastError());
  FMM_CHECK(cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, st));
  FMM_CHECK(cudaStreamSynchronize(st));
  if (hflags & FLAG_LIST_OVERFLOW) throw FmmError(FMM_ERR_UNSUPPORTED, "interaction-list traversal stack overflow");
  h->stats.n_components = nc;
  h->stats.n_boxes = nb;
  h->stats.max_level = level;
  h->stats.n_v_pairs = tot[0];
}

"""Plain CPU FMM for the layered Green's function (Sec. 3.4, Algorithm 1).

One FMM per component:
  * free space, layer l: targets and sources of layer l, kernel
    e^{ik_l r} / (4 pi r), j != i (bitwise-identical points skipped);
  * reaction (l, l', a, b): targets of layer l, equivalent polarization
    sources (images, eq. eqpolarizedsource) of the sources of layer l',
    kernel u~^{ab}_{l l'} (eq. generalcomponentsimag).
The potential is the sum of all components (eq. totalinteraction).

Tree (reading c8 of the ambiguities; the paper leaves it to DASHMM):
  root centre c = ((min x + max x)/2, (min y + max y)/2, c_z) with
  c_z = (min z + max z)/2 for free space and c_z = d_l (a = up) or d_{l-1}
  (a = down) for reaction, so that the root box is split by the interface
  (Sec. 3.4, "equally divided by the interface"); half-width
  h = max over axes of max(max - c, c - min), times (1 + 2^-20).
  Key of a point: i = min(2^21 - 1, floor((x - (c - h)) * (2^21 / (2h)))) per
  axis (FP64, round to nearest, each operation rounded separately), bits
  interleaved x lowest; in reaction trees targets are clamped to the target
  half (i_z >= 2^20 when targets lie above the interface) and images to the
  other half.  Stable sort by (key, original index), sources and targets
  separately.  A box at level l < 21 is refined iff it holds more than ``leaf``
  sources or more than ``leaf`` targets, or -- in a reaction tree, unless the
  count-only rule is asked for (``split_interface=False``) -- it touches
  the interface (its closed z-extent contains the root's mid-plane) and holds
  any point; empty children are dropped.  The second rule separates every
  target leaf from every image leaf by at least one box, so the reaction
  components need no near-field evaluation as long as no point lies within
  2^-21 of the root width of the interface (design reading; the paper leaves
  the refinement to DASHMM).  Under the count-only rule, target leaves next
  to the interface have image leaves in their U, W and X lists, evaluated by
  the Sommerfeld quadrature (the near field of Algorithm 1's last step).
  Boxes are numbered by (level, key prefix).
Lists (Cheng-Greengard-Rokhlin style, source boxes with >= 1 source, target
  boxes with >= 1 target; closed boxes touching = adjacent):
  V(T): children of the parent's colleagues not adjacent to T (M2L);
  U(T), leaf T: source leaves adjacent to T, T included (direct);
  W(T), leaf T: descendants of T's colleagues whose parent is adjacent to T
        but which are not (direct, exact kernel);
  X(T): source leaves S coarser than T, adjacent to parent(T), not adjacent
        to T (direct to every target below T, exact kernel).
  Every list is sorted by box number.

Expansions (all with the paper's coefficient convention, eq. melecoeffree):
  P2M  M_nm = sum_j q_j 4 pi j_n(k r_j) conj(Y_n^m)        (k = source k)
  M2M  M~ = conj(S^(b)) M,  b = c_child - c_parent          (eq. metome)
  M2L  free space: L_nm = (ik/4pi) sum S_{nu n}^{mu m}(c_t - c_s) M_{nu mu}
       (Thm. 2.3 with the index order the derivation gives; the printed
       S_{n nu}^{m mu} of eq. metole is its transpose), S from the Gaunt
       formula eq. (singularseparation);
       reaction: L = T M with T of eq. (me2lesimplified) -- see reaction_T;
  L2L  L~ = S^(b)^T L, b = c_child - c_parent               (eq. metome)
  L2P  Phi = sum L_nm j_n(k r) Y_n^m                         (k = target k)

Pins: tests/test_oracle_fmm.py (tree/list invariants and completeness,
translation operators against direct evaluation, reaction M2L against the
quadrature kernel, FMM against the direct sum with geometric decay in p,
the printed ME convergence rates of Fig. meconvergence).
"""
import math
from collections import defaultdict

import numpy as np

from . import specfun as sf
from .gaunt import gaunt_table
from .green import FOUR_PI, Ztilde, free_kernel, image_z, j0_on_rule, oracle_rule
from .media import UP, DOWN

NBITS = 21
MAXLEV = 21


# ======================================================================= tree
def _spread_bits(v):
    v = v.astype(np.uint64)
    out = np.zeros_like(v)
    for b in range(NBITS):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def morton(ix, iy, iz):
    return _spread_bits(ix) | (_spread_bits(iy) << np.uint64(1)) | (_spread_bits(iz) << np.uint64(2))


def demorton(key, level):
    """Integer coordinates (ix, iy, iz) at ``level`` of a level prefix."""
    key = int(key)
    ix = iy = iz = 0
    for b in range(level):
        ix |= ((key >> (3 * b)) & 1) << b
        iy |= ((key >> (3 * b + 1)) & 1) << b
        iz |= ((key >> (3 * b + 2)) & 1) << b
    return ix, iy, iz


def root_box(src, tgt, cz_fixed=None):
    """Root centre and half-width (see module docstring)."""
    pts = np.concatenate([src, tgt], axis=0)
    mn = pts.min(axis=0)
    mx = pts.max(axis=0)
    c = (mn + mx) * 0.5
    if cz_fixed is not None:
        c[2] = cz_fixed
    hax = np.maximum(mx - c, c - mn)
    h = float(np.max(hax)) * (1.0 + 2.0 ** -20)
    if h == 0.0:
        h = 1.0
    return c, h


def point_keys(pos, c, h, zclamp=None):
    """Morton keys of points; ``zclamp`` = (lo, hi) bounds on i_z."""
    s = 2097152.0 / (2.0 * h)
    lo = c - h
    t = (pos - lo[None, :]) * s
    i = np.floor(t)
    i = np.clip(i, 0, 2 ** NBITS - 1).astype(np.int64)
    if zclamp is not None:
        i[:, 2] = np.clip(i[:, 2], zclamp[0], zclamp[1])
    return morton(i[:, 0], i[:, 1], i[:, 2])


class Tree:
    """Adaptive octree over one component's sources and targets."""

    def __init__(self, src, tgt, leaf, c, h, zclamp_src=None, zclamp_tgt=None, split_interface=False):
        self.c = np.asarray(c, float)
        self.h = float(h)
        self.leaf = int(leaf)
        self.split_interface = bool(split_interface)
        ks = point_keys(src, self.c, self.h, zclamp_src) if len(src) else np.zeros(0, np.uint64)
        kt = point_keys(tgt, self.c, self.h, zclamp_tgt) if len(tgt) else np.zeros(0, np.uint64)
        # stable sort by (key, original index)
        self.sperm = np.lexsort((np.arange(len(ks)), ks)) if len(ks) else np.zeros(0, int)
        self.tperm = np.lexsort((np.arange(len(kt)), kt)) if len(kt) else np.zeros(0, int)
        self.skeys = ks[self.sperm]
        self.tkeys = kt[self.tperm]
        self._build()

    def _prefix(self, keys, level):
        return keys >> np.uint64(3 * (NBITS - level))

    def _build(self):
        lev, pre, s0, s1, t0, t1, par = [], [], [], [], [], [], []
        cur = [(0, 0, len(self.skeys), 0, len(self.tkeys), -1)]   # prefix, s0, s1, t0, t1, parent
        level = 0
        while cur:
            base = len(lev)
            nxt = []
            for j, (p, a0, a1, b0, b1, pa) in enumerate(cur):
                lev.append(level)
                pre.append(p)
                s0.append(a0); s1.append(a1); t0.append(b0); t1.append(b1); par.append(pa)
                me = base + j
                touches = False
                if self.split_interface and (a1 - a0) + (b1 - b0) > 0:
                    iz = demorton(p, level)[2]
                    half = 1 << (level - 1) if level >= 1 else 0
                    touches = level == 0 or iz == half - 1 or iz == half
                if ((a1 - a0) > self.leaf or (b1 - b0) > self.leaf or touches) and level < MAXLEV:
                    sp_ = self._prefix(self.skeys[a0:a1], level + 1)
                    tp_ = self._prefix(self.tkeys[b0:b1], level + 1)
                    for o in range(8):
                        cp = (p << 3) | o
                        c_s0 = a0 + int(np.searchsorted(sp_, np.uint64(cp), "left"))
                        c_s1 = a0 + int(np.searchsorted(sp_, np.uint64(cp), "right"))
                        c_t0 = b0 + int(np.searchsorted(tp_, np.uint64(cp), "left"))
                        c_t1 = b0 + int(np.searchsorted(tp_, np.uint64(cp), "right"))
                        if c_s1 > c_s0 or c_t1 > c_t0:
                            nxt.append((cp, c_s0, c_s1, c_t0, c_t1, me))
            cur = nxt
            level += 1
        self.level = np.array(lev, dtype=np.int64)
        self.prefix = np.array(pre, dtype=np.uint64)
        self.src_begin = np.array(s0, dtype=np.int64)
        self.src_end = np.array(s1, dtype=np.int64)
        self.tgt_begin = np.array(t0, dtype=np.int64)
        self.tgt_end = np.array(t1, dtype=np.int64)
        self.parent = np.array(par, dtype=np.int64)
        nb = len(lev)
        self.children = [[] for _ in range(nb)]
        for b in range(1, nb):
            self.children[self.parent[b]].append(b)
        self.is_leaf = np.array([len(ch) == 0 for ch in self.children])
        self.nlevels = int(self.level.max()) + 1
        self.lookup = {(int(self.level[b]), int(self.prefix[b])): b for b in range(nb)}
        self.coords = np.array([demorton(self.prefix[b], self.level[b]) for b in range(nb)],
                               dtype=np.int64).reshape(nb, 3)
        self.nsrc = self.src_end - self.src_begin
        self.ntgt = self.tgt_end - self.tgt_begin

    # -- geometry
    def width(self, level):
        return 2.0 * self.h / (2 ** level)

    def center(self, b):
        w = self.width(int(self.level[b]))
        return (self.c - self.h) + (self.coords[b] + 0.5) * w

    def adjacent(self, b1, b2):
        l1, l2 = int(self.level[b1]), int(self.level[b2])
        L = max(l1, l2)
        f1, f2 = 1 << (L - l1), 1 << (L - l2)
        lo1 = self.coords[b1] * f1
        hi1 = lo1 + f1
        lo2 = self.coords[b2] * f2
        hi2 = lo2 + f2
        return bool(np.all(lo1 <= hi2) and np.all(lo2 <= hi1))

    def colleagues(self, b):
        """Same-level boxes adjacent to b (b included)."""
        l = int(self.level[b])
        out = []
        n = 1 << l
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    ix, iy, iz = self.coords[b] + np.array([dx, dy, dz])
                    if 0 <= ix < n and 0 <= iy < n and 0 <= iz < n:
                        key = int(morton(np.array([ix]), np.array([iy]), np.array([iz]))[0])
                        o = self.lookup.get((l, key))
                        if o is not None:
                            out.append(o)
        return sorted(out)

    def ancestors(self, b):
        out = []
        while self.parent[b] >= 0:
            b = int(self.parent[b])
            out.append(b)
        return out      # parent first

    def subtree_leaves(self, b):
        if self.is_leaf[b]:
            return [b]
        out = []
        for c in self.children[b]:
            out.extend(self.subtree_leaves(c))
        return out


def build_lists(tree):
    """U, V, W, X lists (dict box -> sorted list of boxes)."""
    nb = len(tree.level)
    U, V, W, X = {}, {}, {}, {}
    for T in range(nb):
        if tree.ntgt[T] == 0:
            continue
        l = int(tree.level[T])
        # V list
        vl = []
        if l >= 2:
            P = int(tree.parent[T])
            for C in tree.colleagues(P):
                for S in tree.children[C]:
                    if tree.nsrc[S] > 0 and not tree.adjacent(S, T):
                        vl.append(S)
        if vl:
            V[T] = sorted(vl)
        # X list
        xl = []
        if l >= 2:
            P = int(tree.parent[T])
            for A in tree.ancestors(T):       # levels l-1 .. 0
                if tree.level[A] < 1:
                    continue
                for S in tree.colleagues(A):
                    if S != A and tree.is_leaf[S] and tree.nsrc[S] > 0 \
                            and tree.adjacent(S, P) and not tree.adjacent(S, T):
                        xl.append(S)
        if xl:
            X[T] = sorted(set(xl))
        if not tree.is_leaf[T]:
            continue
        ul, wl = [], []
        # same level and finer
        stack = []
        for C in tree.colleagues(T):
            if tree.is_leaf[C]:
                if tree.nsrc[C] > 0:
                    ul.append(C)
            else:
                stack.append(C)
        while stack:
            C = stack.pop()
            for S in tree.children[C]:
                if tree.adjacent(S, T):
                    if tree.is_leaf[S]:
                        if tree.nsrc[S] > 0:
                            ul.append(S)
                    else:
                        stack.append(S)
                elif tree.nsrc[S] > 0:
                    wl.append(S)
        # coarser leaves adjacent to T
        for A in tree.ancestors(T):
            if tree.level[A] < 1:
                continue
            for S in tree.colleagues(A):
                if S != A and tree.is_leaf[S] and tree.nsrc[S] > 0 and tree.adjacent(S, T):
                    ul.append(S)
        if ul:
            U[T] = sorted(set(ul))
        if wl:
            W[T] = sorted(wl)
    return U, V, W, X


# ================================================================ operators
def _sign(e):
    return -1.0 if (e % 2) else 1.0


_idx_cache = {}


def _sep_index(p):
    """Index arrays for the Gaunt-formula separation matrices."""
    if p in _idx_cache:
        return _idx_cache[p]
    G = gaunt_table(p)
    ns, ms = sf.nm_table(p)
    P = sf.ncoef(p)
    ii, jj, qq, yy, gg = [], [], [], [], []
    for i in range(P):
        for j in range(P):
            n, m, nu, mu = ns[i], ms[i], ns[j], ms[j]
            for q in range(abs(n - nu), n + nu + 1):
                if abs(mu - m) <= q and G[i, j, q] != 0.0:
                    ii.append(i); jj.append(j); qq.append(q)
                    yy.append(sf.nm(q, mu - m)); gg.append(G[i, j, q])
    ii, jj, qq, yy, gg = map(np.array, (ii, jj, qq, yy, gg))
    pref = np.array([4 * math.pi * _sign(ms[i]) * (1j ** int((ns[j] - ns[i]) % 4))
                     for i, j in zip(ii, jj)])
    coef = pref * gg * np.array([1j ** int(q % 4) for q in qq])
    _idx_cache[p] = (ii, jj, qq, yy, coef)
    return _idx_cache[p]


def sep_matrix(p, k, b, regular):
    """S_{n nu}^{m mu}(b) (regular=False, eq. singularseparation) or
    S^_{n nu}^{m mu}(b) (regular=True, eq. spmhat3d), rows (n,m), cols (nu,mu)."""
    ii, jj, qq, yy, coef = _sep_index(p)
    r, th, ph = sf.cart2sph(np.asarray(b, float))
    if regular:
        z = sf.sph_jn_all(2 * p, k * r).astype(complex)
    else:
        z = sf.sph_hn_all(2 * p, k * r)
    Y = sf.ylm_all(2 * p, th, ph)
    P = sf.ncoef(p)
    vals = coef * z[qq] * np.conj(Y[yy])
    flat = ii * P + jj
    S = (np.bincount(flat, weights=vals.real, minlength=P * P)
         + 1j * np.bincount(flat, weights=vals.imag, minlength=P * P))
    return S.reshape(P, P)


def p2m(p, k, c, pos, q):
    """Multipole coefficients of point sources about c (eq. melecoeffree)."""
    if len(pos) == 0:
        return np.zeros(sf.ncoef(p), complex)
    r, th, ph = sf.cart2sph(pos - c[None, :])
    J = sf.expand_n(sf.sph_jn_all(p, k * r), p)
    return FOUR_PI * np.sum(q[:, None] * J * np.conj(sf.ylm_all(p, th, ph)), axis=0)


def l2p(p, k, c, pos, L):
    """Evaluate a local expansion about c at points (eq. freespace3dlocexp)."""
    r, th, ph = sf.cart2sph(pos - c[None, :])
    J = sf.expand_n(sf.sph_jn_all(p, k * r), p)
    return (J * sf.ylm_all(p, th, ph)) @ L


def m2m(p, k, c_child, c_parent, M):
    return np.conj(sep_matrix(p, k, c_child - c_parent, True)) @ M


def l2l(p, k, c_parent, c_child, L):
    return sep_matrix(p, k, c_child - c_parent, True).T @ L


def free_m2l_matrix(p, k, c_t, c_s):
    """Matrix mapping M (about c_s) to L (about c_t) for e^{ikr}/(4 pi r)."""
    return (1j * k / FOUR_PI) * sep_matrix(p, k, c_t - c_s, False).T


def reaction_T(medium, l, lp, a, b, p, c_t, c_s, rule, sig=None):
    """Reaction M2L matrix (see reaction_T_radial); full matrix for one pair."""
    dx, dy = c_t[0] - c_s[0], c_t[1] - c_s[1]
    I = reaction_T_radial(medium, l, lp, a, b, p, math.hypot(dx, dy), c_t[2], c_s[2], rule, sig)
    return I * reaction_T_phase(p, math.atan2(dy, dx))


def reaction_T_phase(p, phi):
    """e^{i (m'-m) phi} on the (n,m) x (n',m') layout."""
    _, ms = sf.nm_table(p)
    return np.exp(1j * (ms[None, :] - ms[:, None]) * phi)


def reaction_T_radial(medium, l, lp, a, b, p, rho, z_t, z_s, rule, sig=None):
    """Reaction M2L matrix T (rows (n,m), cols (n',m')) for targets in layer l
    about c_t and image sources of layer l' about c_s.

    Re-derived from eqs. (mekernelimage), (extfunkhecke), (me2lesimplified):
      T = i^{n+n'+1} i^{m'-m} e^{i(m'-m) phi_ts} s_t s_s
          int k_rho J_{m'-m}(k_rho rho_ts) Z~^a(z_t, z_s) sigma^{ab} / k_lz
              P^_n^m(k_lz / k_l) P^_{n'}^{m'}(k_l'z / k_l') dk_rho,
    (rho_ts, phi_ts) the polar coordinates of the horizontal part of c_t - c_s,
    s_t = 1, s_s = (-1)^{n'} for a = up; s_t = (-1)^{n+m}, s_s = (-1)^{m'} for
    a = down.  The printed eq. (metoleimage2) carries (-1)^{n'} for both a;
    for a = down the source plane wave is e^{i k_l'z (z_s - d_{l-1})}, whose
    Funk-Hecke expansion about c_s gives (-1)^{m'} (as in the paper's own
    first derivation of eq. expfuncreaction), so the oracle uses (-1)^{m'}."""
    kr, w, ne = rule
    kz = medium.kz(kr)
    if sig is None:
        sig = medium.sigma(kr, l, lp)[(a, b)]
    ns, ms = sf.nm_table(p)
    Pl = sf.phat_all(p, kz[l] / medium.k[l], s=kr / medium.k[l])        # (Q, P)
    Plp = sf.phat_all(p, kz[lp] / medium.k[lp], s=kr / medium.k[lp])
    Z = Ztilde(medium, l, lp, a, kz, z_t, z_s)
    base = w * kr * Z * sig / kz[l]                                   # (Q,)
    if a == UP:
        st = np.ones(len(ns))
        ss = np.array([_sign(n) for n in ns])
    else:
        st = np.array([_sign(n + m) for n, m in zip(ns, ms)])
        ss = np.array([_sign(m) for m in ms])
    A = Pl * (1j ** (ns % 4))[None, :] * st[None, :]
    B = Plp * (1j ** (ns % 4))[None, :] * ss[None, :]
    Jall = besselj_on_rule(2 * p, kr, ne, rho)                       # (Q, 4p+1)
    T = np.zeros((len(ns), len(ns)), dtype=complex)
    for m in range(-p, p + 1):
        im = np.nonzero(ms == m)[0]
        d = ms - m                                                    # per column
        Bw = B * base[:, None] * Jall[:, d + 2 * p]
        phase = 1j * (1j ** (d % 4))
        T[im, :] = (A[:, im].T @ Bw) * phase[None, :]
    return T


def besselj_on_rule(dmax, kr, ne, rho):
    """J_d(k_rho rho) for d = -dmax..dmax on all nodes, shape (Q, 2 dmax + 1);
    complex arguments on the ellipse, real on the tail (scipy jv)."""
    Q = len(kr)
    out = np.zeros((Q, 2 * dmax + 1), dtype=complex)
    if rho == 0.0:
        out[:, dmax] = 1.0
        return out
    ds = np.arange(0, dmax + 1)
    ze = kr[:ne] * rho
    zt = kr[ne:].real * rho
    for d in ds:
        v = np.empty(Q, dtype=complex)
        v[:ne] = sf.besselj(d, ze)
        v[ne:] = sf.besselj(d, zt)
        out[:, dmax + d] = v
        out[:, dmax - d] = v * (-1.0) ** d
    return out


def t_rule(medium, H, rho, p):
    """Oracle rule for a reaction M2L class with vertical centre gap H:
    the integrand grows like k_rho^{2p} and decays like e^{-k_rho H}; the real
    tail runs to ~5 times the peak (2p/H), i.e. T = a + (40 + 10p)/H."""
    return oracle_rule(medium, H / (1.0 + 0.25 * p), max(rho, 1e-3))


# ============================================================== components
class Component:
    def __init__(self, kind, l, lp=None, a=None, b=None):
        self.kind, self.l, self.lp, self.a, self.b = kind, l, lp, a, b

    def __repr__(self):
        if self.kind == "free":
            return f"free[{self.l}]"
        return f"reac[{self.l}{self.lp}{'ud'[self.a]}{'ud'[self.b]}]"


def components(medium, nsrc_layer, ntgt_layer):
    """Free-space components (layers with targets and sources) then reaction
    components in (l, l', a, b) order."""
    out = []
    for l in range(medium.L + 1):
        if ntgt_layer[l] and nsrc_layer[l]:
            out.append(Component("free", l))
    if medium.L > 0:
        for l in range(medium.L + 1):
            if not ntgt_layer[l]:
                continue
            for lp in range(medium.L + 1):
                if not nsrc_layer[lp]:
                    continue
                for a in medium.arrows_target(l):
                    for b in medium.arrows_source(lp):
                        out.append(Component("reac", l, lp, a, b))
    return out


def component_tree(medium, comp, src, tgt, leaf, split_interface=True):
    """Root box, key clamps and tree of one component (src: images for
    reaction); ``split_interface`` selects the interface rule of reaction
    trees (see the module docstring)."""
    if comp.kind == "free":
        c, h = root_box(src, tgt)
        return Tree(src, tgt, leaf, c, h)
    cz = medium.d[comp.l] if comp.a == UP else medium.d[comp.l - 1]
    c, h = root_box(src, tgt, cz_fixed=cz)
    half = 2 ** (NBITS - 1)
    if comp.a == UP:      # targets above the interface, images below
        zt, zs = (half, 2 ** NBITS - 1), (0, half - 1)
    else:
        zt, zs = (0, half - 1), (half, 2 ** NBITS - 1)
    return Tree(src, tgt, leaf, c, h, zclamp_src=zs, zclamp_tgt=zt, split_interface=split_interface)


# ============================================================== evaluation
class FMM:
    """Plain CPU FMM of Algorithm 1 for all components.

    ``targets`` (optional) restricts the downward pass and the direct terms to
    a subset of target indices: every returned value is computed exactly as in
    the full run (the full upward pass is always done).
    ``split_interface=False`` builds the reaction trees by the point counts
    alone (count-only rule)."""

    def __init__(self, medium, p, leaf, split_interface=True):
        self.medium = medium
        self.p = int(p)
        self.leaf = int(leaf)
        self.split_interface = bool(split_interface)

    def evaluate(self, src, q, tgt, targets=None, stats=None):
        med = self.medium
        src = np.asarray(src, float)
        tgt = np.asarray(tgt, float)
        q = np.asarray(q, complex)
        ls = med.layer_of(src[:, 2])
        lt = med.layer_of(tgt[:, 2])
        sel = np.arange(len(tgt)) if targets is None else np.asarray(targets)
        want = np.zeros(len(tgt), bool)
        want[sel] = True
        out = np.zeros(len(tgt), dtype=complex)
        ns_l = [int(np.sum(ls == l)) for l in range(med.L + 1)]
        nt_l = [int(np.sum(lt == l)) for l in range(med.L + 1)]
        for comp in components(med, ns_l, nt_l):
            js = np.nonzero(ls == (comp.l if comp.kind == "free" else comp.lp))[0]
            it = np.nonzero(lt == comp.l)[0]
            spos = src[js].copy()
            if comp.kind == "reac":
                spos[:, 2] = image_z(med, comp.l, comp.lp, comp.a, comp.b, src[js, 2])
            vals = self._component(comp, spos, q[js], tgt[it], want[it], stats)
            out[it] += vals
        return out[sel]

    # ------------------------------------------------------------------
    def _component(self, comp, spos, q, tpos, want, stats):
        med, p = self.medium, self.p
        tree = component_tree(med, comp, spos, tpos, self.leaf, self.split_interface)
        U, V, W, X = build_lists(tree)
        if stats is not None:
            stats.setdefault("components", []).append(
                (repr(comp), len(tree.level), sum(map(len, V.values())),
                 sum(map(len, U.values()))))
        if comp.kind == "free":
            ks = kt = med.k[comp.l]
        else:
            ks, kt = med.k[comp.lp], med.k[comp.l]
        S_sorted = spos[tree.sperm]
        q_sorted = q[tree.sperm]
        T_sorted = tpos[tree.tperm]
        want_sorted = want[tree.tperm]
        nb = len(tree.level)
        # boxes whose targets are wanted (and their ancestors)
        need = np.zeros(nb, bool)
        for b in range(nb):
            if tree.ntgt[b] and np.any(want_sorted[tree.tgt_begin[b]:tree.tgt_end[b]]):
                need[b] = True
        # upward pass
        M = {}
        shift = {}
        for b in sorted(range(nb), key=lambda x: -tree.level[x]):
            if tree.nsrc[b] == 0:
                continue
            cb = tree.center(b)
            if tree.is_leaf[b]:
                s0, s1 = tree.src_begin[b], tree.src_end[b]
                M[b] = p2m(p, ks, cb, S_sorted[s0:s1], q_sorted[s0:s1])
            else:
                acc = np.zeros(sf.ncoef(p), complex)
                for c in tree.children[b]:
                    if c in M:
                        okey = ("m2m", int(tree.level[c]), tuple(tree.coords[c] & 1))
                        if okey not in shift:
                            shift[okey] = np.conj(sep_matrix(p, ks, tree.center(c) - cb, True))
                        acc += shift[okey] @ M[c]
                M[b] = acc
        # downward pass
        Lx = {}
        cache = {}
        for b in sorted(range(nb), key=lambda x: tree.level[x]):
            if not need[b]:
                continue
            cb = tree.center(b)
            acc = np.zeros(sf.ncoef(p), complex)
            pa = int(tree.parent[b])
            if pa >= 0 and pa in Lx:
                okey = ("l2l", int(tree.level[b]), tuple(tree.coords[b] & 1))
                if okey not in shift:
                    shift[okey] = sep_matrix(p, kt, cb - tree.center(pa), True).T
                acc += shift[okey] @ Lx[pa]
            for S in V.get(b, []):
                acc += self._m2l(comp, tree, b, S, cache) @ M[S]
            Lx[b] = acc
        rule = None
        if comp.kind == "reac":
            # one rule for the component: smallest vertical gap and largest
            # lateral distance of any target/image pair
            dref = med.d[comp.l] if comp.a == UP else med.d[comp.l - 1]
            H = float(np.min(np.abs(tpos[:, 2] - dref)) + np.min(np.abs(spos[:, 2] - dref)))
            rho = 2.0 * math.sqrt(2.0) * tree.h
            kr, w, ne = oracle_rule(med, H, rho)
            kz = med.kz(kr)
            rule = (kr, w, ne, kz, med.sigma(kr, comp.l, comp.lp)[(comp.a, comp.b)])
        res = np.zeros(len(T_sorted), dtype=complex)
        for b in range(nb):
            if not need[b]:
                continue
            t0, t1 = tree.tgt_begin[b], tree.tgt_end[b]
            idx = np.arange(t0, t1)[want_sorted[t0:t1]]
            if tree.is_leaf[b]:
                res[idx] += l2p(p, kt, tree.center(b), T_sorted[idx], Lx[b])
                for S in U.get(b, []) + W.get(b, []):
                    s0, s1 = tree.src_begin[S], tree.src_end[S]
                    res[idx] += self._direct(comp, T_sorted[idx], S_sorted[s0:s1], q_sorted[s0:s1], rule)
            for S in X.get(b, []):
                s0, s1 = tree.src_begin[S], tree.src_end[S]
                res[idx] += self._direct(comp, T_sorted[idx], S_sorted[s0:s1], q_sorted[s0:s1], rule)
        out = np.zeros(len(tpos), dtype=complex)
        out[tree.tperm] = res
        return out

    def _m2l(self, comp, tree, T, S, cache):
        p, med = self.p, self.medium
        lev = int(tree.level[T])
        d = tree.coords[T] - tree.coords[S]
        if comp.kind == "free":
            key = (lev, int(d[0]), int(d[1]), int(d[2]))
            if key not in cache:
                cache[key] = free_m2l_matrix(p, med.k[comp.l], tree.center(T), tree.center(S))
            return cache[key]
        key = (lev, int(d[0]), int(d[1]), int(tree.coords[T][2]), int(tree.coords[S][2]))
        if key not in cache:
            ct, cs = tree.center(T), tree.center(S)
            rkey = ("radial", lev, int(d[0] ** 2 + d[1] ** 2), key[3], key[4])
            if rkey not in cache:
                H = abs(ct[2] - cs[2])
                rho = math.hypot(ct[0] - cs[0], ct[1] - cs[1])
                rule = t_rule(med, H, rho, p)
                cache[rkey] = reaction_T_radial(med, comp.l, comp.lp, comp.a, comp.b, p,
                                                rho, ct[2], cs[2], rule)
            phi = math.atan2(ct[1] - cs[1], ct[0] - cs[0])
            cache[key] = cache[rkey] * reaction_T_phase(p, phi)
        return cache[key]

    def _direct(self, comp, tpos, spos, q, rule=None):
        med = self.medium
        if len(tpos) == 0 or len(spos) == 0:
            return np.zeros(len(tpos), complex)
        if comp.kind == "free":
            diff = tpos[:, None, :] - spos[None, :, :]
            R = np.sqrt(np.sum(diff * diff, axis=-1))
            same = np.all(diff == 0.0, axis=-1)
            Rs = np.where(same, 1.0, R)
            k = med.k[comp.l]
            G = np.where(same, 0.0, np.exp(1j * k * Rs) / (FOUR_PI * Rs))
            return G @ q
        l, lp, a = comp.l, comp.lp, comp.a
        kr, w, ne, kz, sig = rule
        f = w * kr * sig / kz[l]
        out = np.zeros(len(tpos), complex)
        for i in range(len(tpos)):
            t = tpos[i]
            rr = np.hypot(t[0] - spos[:, 0], t[1] - spos[:, 1])
            J = j0_on_rule(kr, ne, rr)
            Z = Ztilde(med, l, lp, a, kz, t[2], spos[:, 2][:, None])
            out[i] = 1j / FOUR_PI * np.sum(q[:, None] * J * Z * f[None, :])
        return out


def reaction_me_basis(medium, l, lp, a, b, p, r, c_s, rule):
    """Expansion functions F~_nm(r, c_s) of the image-form multipole expansion
    (eq. mebasis), so that u~(r, r_s) = sum_nm M_nm F~_nm(r, c_s) with
    M_nm = 4 pi j_n(k_l' |r_s - c_s|) conj(Y_n^m) (eq. melayerupgoingimage).
    After the alpha integral (identity for J_n, Sec. 3.5):
      F~_nm = (i/4pi) s_s i^n i^m e^{i m phi} int k_rho J_m(k_rho rho)
              Z~^a(z, z_s) sigma / k_lz P^_n^m(k_l'z / k_l') dk_rho,
    (rho, phi) the polar coordinates of the horizontal part of r - c_s and
    s_s = (-1)^n (a = up) or (-1)^m (a = down) as in reaction_T."""
    kr, w, ne = rule
    kz = medium.kz(kr)
    sig = medium.sigma(kr, l, lp)[(a, b)]
    ns, ms = sf.nm_table(p)
    Plp = sf.phat_all(p, kz[lp] / medium.k[lp], s=kr / medium.k[lp])
    Z = Ztilde(medium, l, lp, a, kz, r[2], c_s[2])
    dx, dy = r[0] - c_s[0], r[1] - c_s[1]
    rho, phi = math.hypot(dx, dy), math.atan2(dy, dx)
    Jall = besselj_on_rule(p, kr, ne, rho)
    base = w * kr * Z * sig / kz[l]
    ss = np.array([_sign(n) for n in ns]) if a == UP else np.array([_sign(m) for m in ms])
    integ = np.sum(base[:, None] * Jall[:, ms + p] * Plp, axis=0)
    return (1j / FOUR_PI) * ss * (1j ** (ns % 4)) * (1j ** (ms % 4)) * np.exp(1j * ms * phi) * integ

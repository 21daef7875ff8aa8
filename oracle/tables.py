"""Tabulated Sommerfeld integrals and polynomial interpolation of the reaction
M2L operators (Sec. 3.5: eqs. uniformintegral, identitypolyexp, M2Ltable,
metoletableform) -- oracle, test infrastructure only.

The reaction M2L matrix (eq. me2lesimplified) needs O(p^4) Sommerfeld
integrals per translation.  Sec. 3.5 writes every one of them as a short sum
of a few integrals that do not depend on (n, m, n', m'):

  P^_n^m(k_lz/k_l) = (k_l/k_lz)^mu  sum_s b^s_{n|m|} (k_rho/k_l)^{|m|+2s} tau_m,
      mu = (n+|m|) mod 2, tau_m = (-1)^m for m < 0, 1 otherwise
      (Rodrigues' formula and eq. identitypolyexp),
  S_{q,t,mu,nu}(rho, zt, zs) = int k_rho^{t+1} J_q(k_rho rho) Z~(zt, zs)
                               sigma / k_lz (k_l/k_lz)^mu (k_l'/k_l'z)^nu dk_rho
      (eq. M2Ltable, q the Bessel order, t the power of k_rho),
  I_{nm,n'm'} = sum_s A^s_{nn'mm'} S_{m'-m, |m|+|m'|+2s, mu, nu}
      (eq. metoletableform; J_{-q} = (-1)^q J_q),
  A^s = sum_{s1+s2=s} tau_m tau_m' b^{s1}_{n|m|} b^{s2}_{n'|m'|}
                       / (k_l^{|m|+2 s1} k_l'^{|m'|+2 s2})          (eq. asslegendreexpcoef),
and the radial M2L matrix (the matrix of ``fmm.reaction_T_radial``) is
  T_{nm,n'm'} = i^{n+n'+1} i^{m'-m} s_t s_s I_{nm,n'm'}
with the signs s_t, s_s of that function.  Here the coefficients b are
derived afresh from Rodrigues' formula: an odd polynomial x f(x^2) is
written (1/x)(1 - s^2) f(1 - s^2) with x = k_z/k, s = k_rho/k, so that odd
degrees carry the factor k/k_z as in the paper.

Tables (the paper tabulates S on a 3-D grid in (rho, z, z') over "the domain
of interest" and interpolates with polynomials, Sec. 3.5 and Sec. 4).  The
domain of interest of the library's M2L is the set of class points the trees
produce: a reaction V pair at level l joins boxes of width w whose centres are
(jt + 1/2) w and (js + 1/2) w from the interface (jt, js in {0, 1}) and
rho = w * sqrt(dx^2 + dy^2) apart horizontally (ten values of dx^2 + dy^2).
These 40 rays through the origin of (rho, zt, zs) are the tabulated domain;
along each ray the coordinate is u = log2(k_max w), k_max the largest wave
number of the medium, u in [-8, 1.5].  The ray is cut into panels (whole
octaves for u < -3, half octaves up to -1, quarter octaves beyond), and
on each panel the values S * w^(t+2) are kept at 12 Chebyshev points of the
first kind and interpolated by the barycentric formula (a polynomial of
degree 11).  The factor w^(t+2) removes the w^-(t+2) growth of the integrals
as w -> 0, so that the interpolated function is smooth in u.
"""
import math

import numpy as np
from numpy.polynomial import polynomial as npoly

from . import specfun as sf
from .fmm import besselj_on_rule, t_rule
from .media import UP

RHO2 = (0, 1, 2, 4, 5, 8, 9, 10, 13, 18)          # dx^2 + dy^2 of the radial classes
NCHEB = 12                                        # interpolation points per panel
U_EDGES = tuple([-8.0, -7.0, -6.0, -5.0, -4.0, -3.0, -2.5, -2.0, -1.5, -1.0]
                + [-1.0 + 0.25 * i for i in range(1, 11)])


# ------------------------------------------------------ Legendre power forms
def legendre_power(n, m):
    """(mu, beta) with P^_n^m(x) = (1/x)^mu s^m sum_j beta_j s^{2j}, m >= 0,
    s = sqrt(1 - x^2): Rodrigues' formula P^_n^m = c_nm/(2^n n!) s^m
    d^{n+m}/dx^{n+m} (x^2 - 1)^n, the derivative written in powers of
    x^2 = 1 - s^2 (eq. identitypolyexp and the expansion after it)."""
    c = math.sqrt((2 * n + 1) / (4.0 * math.pi) * math.factorial(n - m) / math.factorial(n + m))
    poly = npoly.polypow([-1.0, 0.0, 1.0], n)
    der = npoly.polyder(poly, n + m) * c / (2.0 ** n * math.factorial(n))   # degree n - m in x
    mu = (n - m) % 2
    beta = np.zeros(n + 2)
    for j, cj in enumerate(der):
        if j % 2 != mu:
            continue
        i = (j - mu) // 2 + mu          # x^{2i'} -> (1-s^2)^{i'};  x^{2i'+1} -> (1/x)(1-s^2)^{i'+1}
        b = npoly.polypow([1.0, -1.0], i)
        beta[:len(b)] += cj * b
    return mu, np.trim_zeros(beta, "b")


class Expansion:
    """Index set of the S integrals and the coefficients A^s for order p and
    the wave numbers (k_l, k_l') of one layer pair."""

    def __init__(self, p, kl, klp):
        self.p = p
        ns, ms = sf.nm_table(p)
        self.ns = [int(v) for v in ns]
        self.ms = [int(v) for v in ms]
        forms = {(n, m): legendre_power(n, m) for n in range(p + 1) for m in range(n + 1)}
        keys = set()
        terms = {}
        P = len(self.ns)
        for i in range(P):
            n, m = self.ns[i], self.ms[i]
            mu, be = forms[(n, abs(m))]
            tau = (-1) ** abs(m) if m < 0 else 1
            for j in range(P):
                n2, m2 = self.ns[j], self.ms[j]
                nu, be2 = forms[(n2, abs(m2))]
                tau2 = (-1) ** abs(m2) if m2 < 0 else 1
                q = abs(m2 - m)
                sgn_q = (-1) ** q if m2 - m < 0 else 1       # J_{-q} = (-1)^q J_q
                A = {}
                for s1, c1 in enumerate(be):
                    for s2, c2 in enumerate(be2):
                        t = abs(m) + abs(m2) + 2 * (s1 + s2)
                        A[t] = A.get(t, 0.0) + tau * tau2 * sgn_q * c1 * c2 / (
                            kl ** (abs(m) + 2 * s1) * klp ** (abs(m2) + 2 * s2))
                lst = []
                for t, a in sorted(A.items()):
                    keys.add((q, t, mu, nu))
                    lst.append(((q, t, mu, nu), a))
                terms[(i, j)] = lst
        self.index = sorted(keys)
        pos = {k: x for x, k in enumerate(self.index)}
        self.terms = {ij: [(pos[k], a) for k, a in lst] for ij, lst in terms.items()}
        self.tpow = np.array([k[1] for k in self.index])


# ----------------------------------------------------------- the integrals
def s_integrals(medium, comp, p, ex, rho, zt, zs, rule=None):
    """S_{q,t,mu,nu}(rho, zt, zs) of eq. M2Ltable for every index of ``ex``,
    by the oracle's contour quadrature.  ``comp`` = (l, l', a, b); zt, zs are
    the distances of the target and of the image from the reference
    interface, so that Z~ = e^{i k_lz zt + i k_l'z zs} (eq. zexponentialimage)."""
    l, lp, a, b = comp
    if rule is None:
        rule = t_rule(medium, zt + zs, max(rho, 1e-3), p)
    kr, w, ne = rule
    kz = medium.kz(kr)
    sig = medium.sigma(kr, l, lp)[(a, b)]
    base = w * kr * np.exp(1j * kz[l] * zt + 1j * kz[lp] * zs) * sig / kz[l]
    J = besselj_on_rule(2 * p, kr, ne, rho)[:, 2 * p:]           # J_q, q = 0..2p
    rl, rlp = medium.k[l] / kz[l], medium.k[lp] / kz[lp]
    tmax = int(ex.tpow.max())
    kpow = kr[:, None] ** np.arange(tmax + 1)[None, :]
    q = np.array([k[0] for k in ex.index])
    mu = np.array([k[2] for k in ex.index])
    nu = np.array([k[3] for k in ex.index])
    X = base[:, None] * kpow[:, ex.tpow] * J[:, q] * rl[:, None] ** mu[None, :] * rlp[:, None] ** nu[None, :]
    return X.sum(axis=0)


def t_from_s(ex, comp, S):
    """Radial reaction M2L matrix from the S integrals (eq. metoletableform and
    the phases of eq. me2lesimplified); layout of fmm.reaction_T_radial."""
    a = comp[2]
    P = len(ex.ns)
    T = np.zeros((P, P), dtype=complex)
    for i in range(P):
        n, m = ex.ns[i], ex.ms[i]
        st = 1 if a == UP else (-1) ** ((n + m) % 2)
        for j in range(P):
            n2, m2 = ex.ns[j], ex.ms[j]
            ss = (-1) ** n2 if a == UP else (-1) ** (m2 % 2)
            acc = 0j
            for x, c in ex.terms[(i, j)]:
                acc += c * S[x]
            T[i, j] = acc * st * ss * 1j ** ((n + n2 + 1 + (m2 - m)) % 4)
    return T


# ---------------------------------------------------------- the tables
def cheb_points(n=NCHEB):
    """Chebyshev points of the first kind on [-1, 1], x_j = cos((2j+1) pi / 2n)."""
    j = np.arange(n)
    return np.cos((2 * j + 1) * np.pi / (2 * n))


def panel_of(u):
    """Index of the panel holding u (panels are half-open, the last closed);
    None outside [U_EDGES[0], U_EDGES[-1]]."""
    if not (U_EDGES[0] <= u <= U_EDGES[-1]):
        return None
    for k in range(len(U_EDGES) - 1):
        if u < U_EDGES[k + 1]:
            return k
    return len(U_EDGES) - 2


def ray(jt, js, r):
    """(rho, zt, zs) per unit box width of the class (jt, js, r)."""
    return math.sqrt(RHO2[r]), jt + 0.5, js + 0.5


def panel_nodes(medium, comp, p, ex, jt, js, r, k):
    """Tabulated values on panel k of ray (jt, js, r): S * w^(t+2) at the
    panel's Chebyshev points, shape (NCHEB, len(ex.index))."""
    kmax = float(np.max(medium.k))
    u0, u1 = U_EDGES[k], U_EDGES[k + 1]
    rh, zt, zs = ray(jt, js, r)
    out = []
    for x in cheb_points():
        u = u0 + 0.5 * (u1 - u0) * (x + 1.0)
        w = 2.0 ** u / kmax
        out.append(s_integrals(medium, comp, p, ex, rh * w, zt * w, zs * w) * w ** (ex.tpow + 2))
    return np.array(out)


def barycentric(values, x):
    """Polynomial through (cheb_points(), values) at x in [-1, 1]
    (barycentric formula with the weights (-1)^j sin((2j+1) pi / 2n))."""
    n = values.shape[0]
    j = np.arange(n)
    xj = cheb_points(n)
    lam = (-1.0) ** j * np.sin((2 * j + 1) * np.pi / (2 * n))
    d = x - xj
    if np.any(d == 0.0):
        return values[int(np.argmin(np.abs(d)))]
    c = lam / d
    return (c.reshape((-1,) + (1,) * (values.ndim - 1)) * values).sum(axis=0) / c.sum()


def table_T(medium, comp, p, w, jt, js, r, ex=None, nodes=None):
    """Radial reaction M2L matrix of class (jt, js, r) at box width w from the
    interpolated tables; None if u = log2(k_max w) is outside the tables.
    ``nodes`` may pass panel_nodes(...) of the panel that holds u."""
    l, lp = comp[0], comp[1]
    if ex is None:
        ex = Expansion(p, medium.k[l], medium.k[lp])
    kmax = float(np.max(medium.k))
    u = math.log2(kmax * w)
    k = panel_of(u)
    if k is None:
        return None
    if nodes is None:
        nodes = panel_nodes(medium, comp, p, ex, jt, js, r, k)
    u0, u1 = U_EDGES[k], U_EDGES[k + 1]
    x = 2.0 * (u - u0) / (u1 - u0) - 1.0
    S = barycentric(nodes, x) / w ** (ex.tpow + 2)
    return t_from_s(ex, comp, S)


def degree_weights(medium, comp, p, w):
    """Size of the degree-n coefficients of expansions of boxes of width w,
    (k rho_b)^n / (2n+1)!! with rho_b = (sqrt 3 / 2) w (the bound of |j_n| in
    eq. melecoeffree): outer product for targets (k_l) and images (k_l').
    Used to weigh operator errors by their effect on the potentials."""
    l, lp = comp[0], comp[1]
    ns, _ = sf.nm_table(p)
    rb = math.sqrt(3.0) / 2.0 * w

    def dfact(n):
        return float(np.prod(np.arange(2 * n + 1, 0, -2, dtype=float)))
    st = np.array([(medium.k[l] * rb) ** n / dfact(n) for n in ns])
    ss = np.array([(medium.k[lp] * rb) ** n / dfact(n) for n in ns])
    return st[:, None] * ss[None, :]


# ------------------------------------------------ near-field kernel table
# The reaction near field (Algorithm 1, last step; eq. generalcomponentsimag)
# needs the kernel u~^{ab}_{ll'} = (i/4pi) S_{0,0,0,0}(rho, zt, zs) at arbitrary
# target-image pairs.  Its table is a true 3-D one, in the coordinates
#   u = log2(k_max R), R = sqrt(rho^2 + H^2), H = zt + zs,
#   theta = atan(rho / H) in [0, atan 6],   f = zt / H in [0, 1],
# holding R * u~ (which tends to a constant as R -> 0) at 10 x 16 x 8
# Chebyshev points of the first kind per panel: whole octaves of u from -7
# to 1, half octaves from 1 to 3.  Pairs outside (R out of range or
# rho > 6 H) are not tabulated.
NF_EDGES = tuple([-7.0 + i for i in range(9)] + [1.5, 2.0, 2.5, 3.0])
NF_NODES = (10, 16, 8)
NF_THETA_MAX = math.atan(6.0)


def near_coords(medium, rho, zt, zs):
    kmax = float(np.max(medium.k))
    H = zt + zs
    R = math.hypot(rho, H)
    return math.log2(kmax * R), math.atan2(rho, H), zt / H, R


def near_panel(u, theta):
    if not (NF_EDGES[0] <= u <= NF_EDGES[-1]) or theta > NF_THETA_MAX:
        return None
    for k in range(len(NF_EDGES) - 1):
        if u < NF_EDGES[k + 1]:
            return k
    return len(NF_EDGES) - 2


def near_panel_nodes(medium, comp, k):
    """R * u~ at the panel's nodes, shape NF_NODES (u, theta, f), by the
    oracle's quadrature of the kernel (green.reaction_image_kernel)."""
    from .green import oracle_rule, reaction_image_kernel
    l, lp, a, b = comp
    d = medium.d[l] if a == UP else medium.d[l - 1]
    kmax = float(np.max(medium.k))
    nu, nt, nf = NF_NODES
    us = NF_EDGES[k] + 0.5 * (NF_EDGES[k + 1] - NF_EDGES[k]) * (cheb_points(nu) + 1.0)
    ts = 0.5 * NF_THETA_MAX * (cheb_points(nt) + 1.0)
    fs = 0.5 * (cheb_points(nf) + 1.0)
    out = np.zeros(NF_NODES, dtype=complex)
    for i, uu in enumerate(us):
        R = 2.0 ** uu / kmax
        for j, th in enumerate(ts):
            H, rho = R * math.cos(th), R * math.sin(th)
            rule = oracle_rule(medium, H, max(rho, 1e-3))
            for m, f in enumerate(fs):
                zt, zs = f * H, (1.0 - f) * H
                zt_abs = d + zt if a == UP else d - zt
                zs_abs = d - zs if a == UP else d + zs
                v = reaction_image_kernel(medium, l, lp, a, b, np.array([0.0, 0.0, zt_abs]),
                                          np.array([[rho, 0.0, zs_abs]]), rule)
                out[i, j, m] = R * v[0]
    return out


def near_table_value(medium, comp, rho, zt, zs, nodes=None):
    """Interpolated near-field reaction kernel u~ of one pair; None outside
    the table.  ``nodes`` may pass near_panel_nodes of the pair's panel."""
    u, th, f, R = near_coords(medium, rho, zt, zs)
    k = near_panel(u, th)
    if k is None:
        return None
    if nodes is None:
        nodes = near_panel_nodes(medium, comp, k)
    xu = 2.0 * (u - NF_EDGES[k]) / (NF_EDGES[k + 1] - NF_EDGES[k]) - 1.0
    xt = 2.0 * th / NF_THETA_MAX - 1.0
    xf = 2.0 * f - 1.0
    v = barycentric(nodes, xu)                 # (nt, nf)
    v = barycentric(v, xt)                     # (nf,)
    v = barycentric(v, xf)
    return v / R

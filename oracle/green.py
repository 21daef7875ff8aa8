"""Layered Green's function by Sommerfeld integrals (Secs. 2.2, 3.1-3.3).

Physical normalization: the free-space part is e^{ik|r-r'|} / (4 pi |r-r'|)
(eq. domaingreenfn).  The reaction part for a target in layer l and a source
in layer l' is

  G^r(r, r') = (1 / 2pi) int_C k_rho J_0(k_rho rho) u^r(k_rho; z, z') dk_rho
             = sum_{a,b} u^{ab}_{l l'}(r, r'),
  u^{ab}_{l l'} = (i / 4pi) int_C k_rho J_0(k_rho rho)
                  e^{i k_lz D_a(z)} e^{i k_l'z D'_b(z')} sigma^{ab}_{l l'} / k_lz dk_rho

(eqs. greenfuncomponent, generalcomponents, with the alpha-integral done in
closed form: int_0^{2pi} e^{i k_rho rho cos(alpha - phi)} d alpha = 2 pi J_0).
D_up(z) = z - d_l, D_down(z) = d_{l-1} - z, D'_up(z') = z' - d_l',
D'_down(z') = d_{l'-1} - z'.

Oracle contour (deliberately not the CUDA library's): a semi-ellipse in the
fourth quadrant from 0 to a = 1.5 max_j k_j + 1 with depth 0.3 a, followed by
the real axis [a, T] where every k_jz is positive imaginary and the integrand
decays like e^{-k_rho h}; T = a + 40 / h_min.  Both pieces use composite
Gauss-Legendre panels (numpy.polynomial.legendre.leggauss).

Pins: tests/test_oracle_green.py (Sommerfeld identity against e^{ikr}/r,
equal-k image closed forms, transmission conditions, reciprocity, agreement
with an independent contour and rule).
"""
import math

import numpy as np
from scipy import special as sp

from .media import UP, DOWN

FOUR_PI = 4.0 * math.pi


# ---------------------------------------------------------------- quadrature
def _gl(n):
    return np.polynomial.legendre.leggauss(n)


def ellipse_rule(a, depth, npanel=4, n=16):
    """Nodes/weights on k_rho(t) = a/2 (1 - cos t) - i depth sin t, t in [0, pi]."""
    x, w = _gl(n)
    edges = np.linspace(0.0, math.pi, npanel + 1)
    ks, ws = [], []
    for i in range(npanel):
        lo, hi = edges[i], edges[i + 1]
        t = 0.5 * (lo + hi) + 0.5 * (hi - lo) * x
        wt = 0.5 * (hi - lo) * w
        kr = 0.5 * a * (1.0 - np.cos(t)) - 1j * depth * np.sin(t)
        dk = 0.5 * a * np.sin(t) - 1j * depth * np.cos(t)
        ks.append(kr)
        ws.append(wt * dk)
    return np.concatenate(ks), np.concatenate(ws)


def tail_rule(a, T, panel, n=20):
    """Composite Gauss-Legendre on the real axis [a, a + m*panel] >= T."""
    x, w = _gl(n)
    m = max(1, int(math.ceil((T - a) / panel)))
    lo = a + panel * np.arange(m)
    kr = (lo[:, None] + 0.5 * panel * (1.0 + x[None, :])).ravel()
    wt = np.tile(0.5 * panel * w, m)
    return kr.astype(complex), wt.astype(complex)


def oracle_rule(medium, h_min, rho_max, npanel_e=6, n_e=16, n_t=20):
    """Full oracle contour rule for integrands decaying like e^{-k_rho h},
    h >= h_min, with Bessel argument k_rho * rho, rho <= rho_max.
    Returns (kr, w, n_ellipse)."""
    a = 1.5 * float(np.max(medium.k)) + 1.0
    ke, we = ellipse_rule(a, 0.3 * a, npanel_e, n_e)
    panel = min(2.0, 6.0 / max(rho_max, 1e-300))
    T = a + 40.0 / h_min
    kt, wt = tail_rule(a, T, panel, n_t)
    return np.concatenate([ke, kt]), np.concatenate([we, wt]), len(ke)


def j0_complex(z):
    """J_0(z) for complex z, |z| <= 12, by its power series
    sum_k (-z^2/4)^k / (k!)^2 (summed to 60 terms); scipy's jv beyond."""
    z = np.asarray(z, dtype=complex)
    small = np.abs(z) <= 12.0
    out = np.empty_like(z)
    zs = z[small]
    u = -(zs * zs) / 4.0
    term = np.ones_like(zs)
    acc = np.ones_like(zs)
    for k in range(1, 60):
        term = term * u / (k * k)
        acc = acc + term
    out[small] = acc
    if np.any(~small):
        out[~small] = sp.jv(0, z[~small])
    return out


def j0_on_rule(kr, n_ellipse, rho):
    """J_0(k_rho rho) for all nodes; rho[...] real >= 0 -> shape rho.shape + (Q,)."""
    rho = np.asarray(rho, dtype=float)
    out = np.empty(rho.shape + kr.shape, dtype=complex)
    out[..., :n_ellipse] = j0_complex(rho[..., None] * kr[:n_ellipse])
    out[..., n_ellipse:] = sp.j0(rho[..., None] * kr[n_ellipse:].real)
    return out


# ---------------------------------------------------------------- kernels
def free_kernel(k, r, rp):
    """e^{ik|r-r'|} / (4 pi |r-r'|)."""
    R = np.linalg.norm(np.asarray(r, float) - np.asarray(rp, float), axis=-1)
    return np.exp(1j * k * R) / (FOUR_PI * R)


def free_kernel_dz(k, r, rp):
    """d/dz of e^{ik|r-r'|} / (4 pi |r-r'|) with respect to the target z."""
    diff = np.asarray(r, float) - np.asarray(rp, float)
    R = np.linalg.norm(diff, axis=-1)
    return (1j * k * R - 1.0) * np.exp(1j * k * R) / (FOUR_PI * R ** 3) * diff[..., 2]


def sommerfeld_free(k, rho, z, rule):
    """Right-hand side of the Sommerfeld identity (eq. sommerfeldid after the
    alpha integral): (i / 4 pi) int k_rho J_0(k_rho rho) e^{i k_z |z|} / k_z.
    Equals e^{ikr}/(4 pi r), r = sqrt(rho^2 + z^2)."""
    kr, w, ne = rule
    kz = np.sqrt(k * k - kr * kr + 0j)
    kz = np.where(kz.imag < 0, -kz, kz)
    J = j0_on_rule(kr, ne, np.asarray(rho))
    f = kr * np.exp(1j * kz * abs(z)) / kz
    return 1j / FOUR_PI * np.sum(J * (w * f), axis=-1)


def reaction_component(medium, l, lp, a, b, r, rp, rule):
    """u^{ab}_{l l'}(r, r') for one target r (layer l) and sources rp[..., 3]
    (layer l') on the given rule (eq. generalcomponents)."""
    kr, w, ne = rule
    kz = medium.kz(kr)
    sig = medium.sigma(kr, l, lp)[(a, b)]
    r = np.asarray(r, float)
    rp = np.asarray(rp, float)
    rho = np.hypot(r[0] - rp[..., 0], r[1] - rp[..., 1])
    J = j0_on_rule(kr, ne, rho)
    Dt = medium.delta_t(a, l, r[2])
    Ds = medium.delta_s(b, lp, rp[..., 2])
    f = w * kr * np.exp(1j * kz[l] * Dt) * sig / kz[l]
    src = np.exp(1j * kz[lp][None, :] * np.asarray(Ds)[..., None]) if np.ndim(Ds) else \
        np.exp(1j * kz[lp] * Ds)
    return 1j / FOUR_PI * np.sum(J * f * src, axis=-1)


def image_z(medium, l, lp, a, b, zp):
    """z of the equivalent polarization source (eq. eqpolarizedsource):
    d_l - D'_b(z') for a = up, d_{l-1} + D'_b(z') for a = down."""
    Ds = medium.delta_s(b, lp, np.asarray(zp, float))
    return (medium.d[l] - Ds) if a == UP else (medium.d[l - 1] + Ds)


def Ztilde(medium, l, lp, a, kz, z, zs):
    """Z~^a_{l l'}(z, z_s) of eq. (zexponentialimage) on the nodes (kz = medium.kz)."""
    if a == UP:
        d = medium.d[l]
        return np.exp(1j * kz[l] * (z - d) + 1j * kz[lp] * (d - zs))
    d = medium.d[l - 1]
    return np.exp(1j * kz[l] * (d - z) + 1j * kz[lp] * (zs - d))


def reaction_image_kernel(medium, l, lp, a, b, r, rs, rule, sig=None):
    """u~^{ab}_{l l'}(r, r_s) with an image source r_s (eq. generalcomponentsimag),
    one target r, sources rs[..., 3]."""
    kr, w, ne = rule
    kz = medium.kz(kr)
    if sig is None:
        sig = medium.sigma(kr, l, lp)[(a, b)]
    r = np.asarray(r, float)
    rs = np.asarray(rs, float)
    rho = np.hypot(r[0] - rs[..., 0], r[1] - rs[..., 1])
    J = j0_on_rule(kr, ne, rho)
    Z = Ztilde(medium, l, lp, a, kz, r[2], np.asarray(rs[..., 2])[..., None])
    f = w * kr * sig / kz[l]
    return 1j / FOUR_PI * np.sum(J * Z * f, axis=-1)


def reaction_total_spectral(medium, l, lp, r, rp, rule, dz=False):
    """G^r(r, r') from the full spectral reaction field of the 2L x 2L solve
    (no split into components): (1/2pi) int k_rho J_0 u^r dk_rho, with
    u^r = A_l e^{i k_lz (z - d_l)} + B_l e^{i k_lz (d_{l-1} - z)} and the
    source wave amplitudes (i/2k_l'z) e^{...} of the two excitations.
    With dz=True returns dG^r/dz (target z) instead; r may lie on the
    boundary of its layer l (used by the transmission-condition pin)."""
    kr, w, ne = rule
    kz = medium.kz(kr)
    resp = medium.unit_responses(kr, lp)
    r = np.asarray(r, float)
    rp = np.asarray(rp, float)
    c = 1j / (2.0 * kz[lp])
    uhat = np.zeros(np.shape(rp)[:-1] + kr.shape, dtype=complex)
    zp = rp[..., 2][..., None]
    for exc, (A, B) in resp.items():
        if exc == "dn":
            amp = c * np.exp(1j * kz[lp] * (zp - medium.d[lp]))
        else:
            amp = c * np.exp(1j * kz[lp] * (medium.d[lp - 1] - zp))
        field = 0.0
        fu = (1j * kz[l]) if dz else 1.0
        if l < medium.L:
            field = field + fu * A[l] * np.exp(1j * kz[l] * (r[2] - medium.d[l]))
        if l > 0:
            field = field + (-fu if dz else 1.0) * B[l] * np.exp(1j * kz[l] * (medium.d[l - 1] - r[2]))
        uhat = uhat + amp * field
    rho = np.hypot(r[0] - rp[..., 0], r[1] - rp[..., 1])
    J = j0_on_rule(kr, ne, rho)
    return np.sum(J * (w * kr) * uhat, axis=-1) / (2.0 * math.pi)


# ---------------------------------------------------------------- direct sum
def _h_of_sources(medium, lp, zs):
    """min over allowed b of D'_b(z') for each source."""
    return np.min(np.stack([medium.delta_s(b, lp, zs) for b in medium.arrows_source(lp)]), axis=0)


def _h_of_target(medium, l, z):
    return min(medium.delta_t(a, l, z) for a in medium.arrows_target(l))


def reaction_block(medium, l, lp, tgt, src, q, chunk=512):
    """sum_j q_j G^r(t_i, s_j) for targets in layer l and sources in layer l'.

    Sources are sorted by their distance to the nearest relevant interface and
    processed in chunks; each chunk truncates the real tail where its slowest
    term has decayed (T = a + 40 / h_chunk), on a panel grid shared by all
    chunks so that sigma is evaluated once per node."""
    tgt = np.asarray(tgt, float)
    src = np.asarray(src, float)
    q = np.asarray(q, complex)
    nt = len(tgt)
    out = np.zeros(nt, dtype=complex)
    if nt == 0 or len(src) == 0:
        return out
    hs = _h_of_sources(medium, lp, src[:, 2])
    order = np.argsort(hs, kind="stable")
    src, q, hs = src[order], q[order], hs[order]
    ht_all = np.array([_h_of_target(medium, l, z) for z in tgt[:, 2]])
    rho_max = float(np.hypot(np.ptp(np.concatenate([tgt[:, 0], src[:, 0]])),
                             np.ptp(np.concatenate([tgt[:, 1], src[:, 1]]))))
    h_glob = float(np.min(ht_all) + hs[0])
    kr, w, ne = oracle_rule(medium, h_glob, max(rho_max, 1e-3))
    kz = medium.kz(kr)
    sig = medium.sigma(kr, l, lp)
    a_list = medium.arrows_target(l)
    b_list = medium.arrows_source(lp)
    a0 = 1.5 * float(np.max(medium.k)) + 1.0
    # per-source factor U_a(j, q) = sum_b sigma^{ab} e^{i k_l'z D'_b(z_j)} q_j
    Ds = {b: medium.delta_s(b, lp, src[:, 2]) for b in b_list}
    for i in range(nt):
        t = tgt[i]
        ht = ht_all[i]
        for c0 in range(0, len(src), chunk):
            c1 = min(len(src), c0 + chunk)
            h = ht + hs[c0]
            T = a0 + 40.0 / h
            nq = int(np.searchsorted(kr[ne:].real, T, side="right")) + ne
            # round up to whole panels of the shared grid
            nq = min(len(kr), ne + int(math.ceil((nq - ne) / 20.0)) * 20)
            krq, wq = kr[:nq], w[:nq]
            rho = np.hypot(t[0] - src[c0:c1, 0], t[1] - src[c0:c1, 1])
            J = j0_on_rule(krq, ne, rho)                      # (nc, nq)
            acc = np.zeros((c1 - c0, nq), dtype=complex)
            for a in a_list:
                ft = np.exp(1j * kz[l, :nq] * medium.delta_t(a, l, t[2]))
                ua = 0.0
                for b in b_list:
                    ua = ua + sig[(a, b)][None, :nq] * np.exp(
                        1j * kz[lp, None, :nq] * Ds[b][c0:c1, None])
                acc += ft[None, :] * ua
            f = wq * krq / kz[l, :nq]
            out[i] += 1j / FOUR_PI * np.sum(q[c0:c1, None] * J * acc * f[None, :])
    return out


def direct_sum(medium, src, q, tgt, targets=None):
    """Phi(t_i) = sum_j q_j G(t_i, s_j) in physical normalization (eq.
    totalinteraction with e^{ikr}/(4 pi r) for the free part).

    Free-space term only for source and target in the same layer, skipped when
    the two points are bitwise identical (the paper's j != i).  Reaction terms
    always included (self image too).  ``targets`` selects a subset of target
    indices (default all)."""
    src = np.asarray(src, float)
    tgt = np.asarray(tgt, float)
    q = np.asarray(q, complex)
    if targets is not None:
        tgt = tgt[np.asarray(targets)]
    ls = medium.layer_of(src[:, 2])
    lt = medium.layer_of(tgt[:, 2])
    out = np.zeros(len(tgt), dtype=complex)
    for l in range(medium.L + 1):
        it = np.nonzero(lt == l)[0]
        if len(it) == 0:
            continue
        js = np.nonzero(ls == l)[0]
        k = medium.k[l]
        for c0 in range(0, len(it), 256):
            ii = it[c0:c0 + 256]
            diff = tgt[ii, None, :] - src[None, js, :]
            R = np.sqrt(np.sum(diff * diff, axis=-1))
            same = np.all(diff == 0.0, axis=-1)
            Rs = np.where(same, 1.0, R)
            val = np.where(same, 0.0, np.exp(1j * k * Rs) / (FOUR_PI * Rs))
            out[ii] += val @ q[js]
        if medium.L > 0:
            for lp in range(medium.L + 1):
                js = np.nonzero(ls == lp)[0]
                if len(js):
                    out[it] += reaction_block(medium, l, lp, tgt[it], src[js], q[js])
    return out

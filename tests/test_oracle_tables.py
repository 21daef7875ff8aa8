"""Pins of the oracle's tabulated-integral form of the reaction M2L
(oracle/tables.py; Sec. 3.5, eqs. identitypolyexp, M2Ltable,
metoletableform).

What pins it, independently of the code under test:
  * the power forms of P^_n^m against the oracle's recurrence values
    (specfun.phat_all) on the real interval and on the complex contour with
    the branch k_rho/k of Sec. 2.2 -- a wrong b coefficient, sign tau_m or
    factor k/k_z fails;
  * the S expansion with exact integrals against the direct radial matrix
    of eq. me2lesimplified (fmm.reaction_T_radial, which integrates the
    Legendre products node by node) -- a dropped term, wrong A^s, wrong
    power of i, wrong J_{-q} sign fails;
  * the interpolated tables against the same direct matrix at box widths
    inside panels of each width (whole, half, quarter octave), with errors
    weighted by the size of the expansion coefficients they multiply;
  * the barycentric formula reproduces the node values and any polynomial of
    degree < 12 exactly;
  * the near-field kernel table (R u~ on Chebyshev points in log2(k_max R),
    atan(rho/H), zt/H) against the quadrature kernel of eq.
    generalcomponentsimag at random pairs.
"""
import math

import numpy as np
import pytest

from oracle import fmm as F
from oracle import specfun as sf
from oracle import tables as tb
from oracle.media import DOWN, UP, Medium

MED = Medium([0.8, 1.2, 1.6], [0.0, -1.2], [1.0, 2.0, 3.0])


def _power_form(n, m, x, s):
    mu, beta = tb.legendre_power(n, abs(m))
    tau = (-1) ** abs(m) if m < 0 else 1
    return tau * (1.0 / x) ** mu * s ** abs(m) * sum(bj * s ** (2 * j) for j, bj in enumerate(beta))


def test_legendre_power_forms_real_and_contour():
    p = 10
    x = np.array([-0.93, -0.41, 0.17, 0.55, 0.91])
    ref = sf.phat_all(p, x)
    s = np.sqrt(1.0 - x * x)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            assert np.allclose(_power_form(n, m, x, s), ref[:, sf.nm(n, m)], rtol=1e-10, atol=1e-12)
    # complex: k_rho on the oracle contour and the real tail, x = k_z/k, s = k_rho/k
    kr, _, _ = F.t_rule(MED, 0.5, 0.3, 4)
    kr = kr[::37]
    k = MED.k[1]
    kz = MED.kz(kr)[1]
    refc = sf.phat_all(p, kz / k, s=kr / k)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            got = _power_form(n, m, kz / k, kr / k)
            scale = np.abs(refc[:, sf.nm(n, m)]).max()
            assert np.abs(got - refc[:, sf.nm(n, m)]).max() <= 1e-9 * scale, (n, m)


def test_index_set_size_and_ranges():
    # q = |m' - m| <= 2p, t = |m| + |m'| + 2s <= 2p + 2, t = q (mod 2)
    for p in (4, 8):
        ex = tb.Expansion(p, 1.0, 1.3)
        qs = [k[0] for k in ex.index]
        ts = [k[1] for k in ex.index]
        assert max(qs) == 2 * p and min(qs) == 0
        assert max(ts) <= 2 * p + 2
        assert all((k[0] - k[1]) % 2 == 0 and k[1] >= k[0] for k in ex.index)
        # the paper counts 4(p+1)(2p+1) tables; the set actually reached is smaller
        assert len(ex.index) <= 4 * (p + 1) * (2 * p + 1)


def _direct_T(comp, p, rho, zt, zs, rule):
    l, lp, a, b = comp
    d = MED.d[l] if a == UP else MED.d[l - 1]
    zt_abs = d + zt if a == UP else d - zt
    zs_abs = d - zs if a == UP else d + zs
    return F.reaction_T_radial(MED, l, lp, a, b, p, rho, zt_abs, zs_abs, rule)


@pytest.mark.parametrize("comp,p", [((0, 1, UP, DOWN), 5), ((2, 1, DOWN, DOWN), 5), ((1, 1, DOWN, UP), 8),
                                    ((0, 0, UP, UP), 8), ((0, 1, UP, DOWN), 10), ((2, 1, DOWN, DOWN), 12)])
def test_s_expansion_reproduces_direct_operator(comp, p):
    l, lp = comp[0], comp[1]
    ex = tb.Expansion(p, MED.k[l], MED.k[lp])
    rho, zt, zs = math.sqrt(5.0) * 0.2, 0.5 * 0.2, 1.5 * 0.2
    rule = F.t_rule(MED, zt + zs, rho, p)
    S = tb.s_integrals(MED, comp, p, ex, rho, zt, zs, rule)
    T1 = tb.t_from_s(ex, comp, S)
    T0 = _direct_T(comp, p, rho, zt, zs, rule)
    # same nodes on both sides: agreement to rounding of the expansion
    assert np.abs(T1 - T0).max() <= 1e-11 * np.abs(T0).max()


@pytest.mark.parametrize("comp,u,jt,js,r", [
    ((0, 1, UP, DOWN), -4.4, 0, 1, 3),      # whole-octave panel
    ((2, 1, DOWN, DOWN), -3.4, 1, 1, 7),
    ((1, 1, DOWN, UP), -1.7, 1, 0, 9),      # half-octave panel
    ((0, 1, UP, DOWN), -0.6, 0, 1, 2),      # quarter-octave panels
    ((2, 1, DOWN, DOWN), 0.6, 0, 0, 9),
    ((1, 1, DOWN, UP), 1.3, 1, 1, 4),
])
def test_interpolated_tables_match_direct_operator(comp, u, jt, js, r):
    p = 8
    l, lp = comp[0], comp[1]
    ex = tb.Expansion(p, MED.k[l], MED.k[lp])
    w = 2.0 ** u / max(MED.k)
    T1 = tb.table_T(MED, comp, p, w, jt, js, r, ex)
    rh, zt, zs = tb.ray(jt, js, r)
    rule = F.t_rule(MED, (zt + zs) * w, max(rh * w, 1e-3), p)
    T0 = _direct_T(comp, p, rh * w, zt * w, zs * w, rule)
    Wt = tb.degree_weights(MED, comp, p, w)
    err = np.abs((T1 - T0) * Wt).max() / np.abs(T0 * Wt).max()
    assert err < 1e-11, err


def test_outside_tables_is_none():
    ex = tb.Expansion(4, MED.k[0], MED.k[1])
    assert tb.table_T(MED, (0, 1, UP, DOWN), 4, 2.0 ** 2 / max(MED.k), 0, 0, 9, ex) is None
    assert tb.table_T(MED, (0, 1, UP, DOWN), 4, 2.0 ** -9 / max(MED.k), 0, 0, 9, ex) is None
    assert tb.panel_of(tb.U_EDGES[0]) == 0 and tb.panel_of(tb.U_EDGES[-1]) == len(tb.U_EDGES) - 2


def test_barycentric_exact_for_low_degree_polynomials():
    rng = np.random.default_rng(3)
    c = rng.normal(size=(tb.NCHEB, 3)) + 1j * rng.normal(size=(tb.NCHEB, 3))
    xn = tb.cheb_points()
    vals = np.array([np.polynomial.polynomial.polyval(x, c) for x in xn])
    for x in (-0.97, -0.2, 0.31, 0.88):
        want = np.polynomial.polynomial.polyval(x, c)
        assert np.allclose(tb.barycentric(vals, x), want, rtol=1e-12, atol=1e-12)
    assert np.array_equal(tb.barycentric(vals, xn[4]), vals[4])


# ---- near-field kernel table (oracle/tables.py, near_*): the interpolated
# kernel against the quadrature kernel of eq. generalcomponentsimag at random
# pairs inside a whole-octave and a half-octave panel, and outside the table.
@pytest.mark.parametrize("comp,k", [((0, 1, UP, DOWN), 5), ((1, 1, DOWN, UP), 10), ((2, 2, DOWN, DOWN), 4)])
def test_near_table_matches_quadrature_kernel(comp, k):
    from oracle import green as G
    l, lp, a, b = comp
    d = MED.d[l] if a == UP else MED.d[l - 1]
    nodes = tb.near_panel_nodes(MED, comp, k)
    rng = np.random.default_rng(11 + k)
    kmax = max(MED.k)
    for _ in range(3):
        u = rng.uniform(tb.NF_EDGES[k], tb.NF_EDGES[k + 1])
        th = rng.uniform(0.0, tb.NF_THETA_MAX)
        f = rng.uniform(0.0, 1.0)
        R = 2.0 ** u / kmax
        H, rho = R * math.cos(th), R * math.sin(th)
        zt, zs = f * H, (1.0 - f) * H
        got = tb.near_table_value(MED, comp, rho, zt, zs, nodes)
        zt_abs = d + zt if a == UP else d - zt
        zs_abs = d - zs if a == UP else d + zs
        rule = G.oracle_rule(MED, H, max(rho, 1e-3))
        ref = G.reaction_image_kernel(MED, l, lp, a, b, np.array([0.0, 0.0, zt_abs]),
                                      np.array([[rho, 0.0, zs_abs]]), rule)[0]
        assert abs(got - ref) <= 1e-9 * abs(ref), (u, th, f, abs(got - ref) / abs(ref))


def test_near_table_domain():
    assert tb.near_table_value(MED, (0, 1, UP, DOWN), 7.0, 0.5, 0.5) is None     # rho > 6 H
    assert tb.near_panel(3.5, 0.1) is None and tb.near_panel(-7.5, 0.1) is None
    assert tb.near_panel(-7.0, 0.0) == 0 and tb.near_panel(3.0, 0.0) == len(tb.NF_EDGES) - 2

"""Pins for oracle.green (Sommerfeld integrals, Secs. 2.2, 3.1-3.3)."""
import math

import numpy as np

from oracle import green
from oracle.media import Medium, UP, DOWN


def test_sommerfeld_identity():
    # eq. (sommerfeldid) after the alpha integral:
    # e^{ikr}/(4 pi r) = (i/4pi) int k_rho J_0(k_rho rho) e^{i k_z |z|}/k_z dk_rho.
    for k in (0.5, 1.0, 2.0, 3.0):
        med = Medium([k])
        for rho, z in [(0.0, 0.1), (0.3, 0.2), (1.5, 0.5), (2.8, 0.1), (0.1, 1.0), (2.8, 2.0)]:
            r = math.hypot(rho, z)
            ex = np.exp(1j * k * r) / (4 * math.pi * r)
            v = green.sommerfeld_free(k, rho, z, green.oracle_rule(med, abs(z), max(rho, 1e-3)))
            assert abs(v - ex) <= 5e-13 * abs(ex), (k, rho, z)


def _gamma12_rule(b, T, n1=30, n2=24, panel=1.0):
    """The contour of Sec. 3.5 (Gamma1: k_rho = i t, -b <= t <= 0; Gamma2:
    k_rho = t - i b, t >= 0), with its own Gauss-Legendre layout: an
    independent rule for the brute-force comparison."""
    x, w = np.polynomial.legendre.leggauss(n1)
    s = 0.5 * b * (1 + x)
    k1 = -1j * s
    w1 = -1j * 0.5 * b * w
    x2, ww2 = np.polynomial.legendre.leggauss(n2)
    m = int(math.ceil(T / panel))
    lo = panel * np.arange(m)
    t = (lo[:, None] + 0.5 * panel * (1 + x2[None, :])).ravel()
    k2 = t - 1j * b
    w2 = np.tile(0.5 * panel * ww2, m).astype(complex)
    kr = np.concatenate([k1, k2])
    wt = np.concatenate([w1, w2])
    return kr, wt, len(kr)          # all nodes complex -> series / jv for J_0


def test_two_independent_quadratures_agree():
    med = Medium([0.8, 1.2, 1.6], [0.0, -1.2], eps=[1, 2, 3])
    rng = np.random.default_rng(4)
    for l, lp in [(0, 0), (1, 0), (1, 1), (2, 1), (0, 2)]:
        tz = {0: 0.35, 1: -0.45, 2: -1.6}[l]
        t = np.array([0.2, -0.1, tz])
        src = rng.uniform(-0.6, 0.6, (4, 3))
        src[:, 2] = {0: rng.uniform(0.1, 1.0, 4), 1: rng.uniform(-1.1, -0.1, 4),
                     2: rng.uniform(-2.2, -1.3, 4)}[lp]
        for a in med.arrows_target(l):
            for b in med.arrows_source(lp):
                v1 = green.reaction_component(med, l, lp, a, b, t, src, green.oracle_rule(med, 0.2, 2.0))
                v2 = green.reaction_component(med, l, lp, a, b, t, src, _gamma12_rule(0.35, 200.0))
                assert np.allclose(v1, v2, rtol=1e-11, atol=0), (l, lp, a, b)


def test_component_and_image_forms_agree_with_full_field():
    # eq. (generalcomponents) summed over (a, b) equals the full spectral field;
    # eq. (generalcomponentsimag) with the image positions of eq.
    # (eqpolarizedsource) equals each component.
    med = Medium([0.8, 1.2, 1.6], [0.0, -1.2], eps=[1, 2, 3])
    rng = np.random.default_rng(5)
    rule = green.oracle_rule(med, 0.2, 3.0)
    for l in range(3):
        for lp in range(3):
            t = np.array([0.1, 0.2, {0: 0.4, 1: -0.6, 2: -1.7}[l]])
            src = rng.uniform(-0.8, 0.8, (5, 3))
            src[:, 2] = {0: rng.uniform(0.1, 1.0, 5), 1: rng.uniform(-1.1, -0.1, 5),
                         2: rng.uniform(-2.2, -1.3, 5)}[lp]
            tot = green.reaction_total_spectral(med, l, lp, t, src, rule)
            comp = 0
            for a in med.arrows_target(l):
                for b in med.arrows_source(lp):
                    c = green.reaction_component(med, l, lp, a, b, t, src, rule)
                    img = src.copy()
                    img[:, 2] = green.image_z(med, l, lp, a, b, src[:, 2])
                    ci = green.reaction_image_kernel(med, l, lp, a, b, t, img, rule)
                    assert np.allclose(c, ci, rtol=1e-13)
                    # images lie across the reference interface from the target
                    dref = med.d[l] if a == UP else med.d[l - 1]
                    assert np.all(np.sign(img[:, 2] - dref) == -np.sign(t[2] - dref))
                    comp = comp + c
            assert np.allclose(comp, tot, rtol=1e-13)


def test_direct_sum_small_brute_force():
    # direct_sum = explicit double loop over pairs of the kernel definitions.
    med = Medium([1.0, 1.5], [0.0], eps=[1, 2])
    rng = np.random.default_rng(6)
    src = rng.uniform(-1, 1, (8, 3))
    src[:4, 2] = rng.uniform(0.1, 1.1, 4)
    src[4:, 2] = rng.uniform(-1.1, -0.1, 4)
    q = rng.uniform(0, 1, 8) + 0j
    got = green.direct_sum(med, src, q, src)
    rule = green.oracle_rule(med, 0.2, 3.0)
    ls = med.layer_of(src[:, 2])
    for i in range(8):
        acc = 0
        for j in range(8):
            if ls[i] == ls[j] and i != j:
                acc += q[j] * green.free_kernel(med.k[ls[i]], src[i], src[j])
            acc += q[j] * green.reaction_total_spectral(med, ls[i], ls[j], src[i], src[j][None], rule)[0]
        assert abs(got[i] - acc) <= 1e-11 * abs(acc)

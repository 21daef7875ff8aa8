"""Pins for oracle.media (reaction densities, Sec. 3.1)."""
import json
import math
import os

import numpy as np

from oracle import green
from oracle.media import Medium, UP, DOWN

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _printed_three_layer(k0, k1, k2, d1, kz):
    """The explicit three-layer densities printed in Sec. 3.1 (source in layer 1)."""
    k0z, k1z, k2z = kz
    E2 = np.exp(-2j * d1 * k1z)
    E1 = np.exp(-1j * d1 * k1z)
    kap11 = (k1 * k1z - k2 * k2z) / 2 * E2 + (k1 * k1z + k2 * k2z) / 2
    kap12 = 1j * ((k2 * k2z - k1 * k1z) / 2 * E2 + (k1 * k1z + k2 * k2z) / 2)
    den = k0 * k0z * kap11 - 1j * k1 * k1z * kap12
    return {
        (0, UP, UP): k1 * k0z * (k1 * k1z - k2 * k2z) * E1 / den,
        (0, UP, DOWN): k1 * k0z * (k1 * k1z + k2 * k2z) / den,
        (1, UP, UP): (k1 * k1z - k2 * k2z) * (k1 * k1z + k0 * k0z) / (2 * den),
        (1, DOWN, DOWN): (k1 * k1z - k0 * k0z) * (k1 * k1z + k2 * k2z) / (2 * den),
        (1, UP, DOWN): (k1 * k1z - k2 * k2z) / den * (k1 * k1z - k0 * k0z) / 2 * E1,
        (1, DOWN, UP): (k1 * k1z - k0 * k0z) / den * (k1 * k1z - k2 * k2z) / 2 * E1,
        (2, DOWN, UP): k1 * k2z * (k1 * k1z + k0 * k0z) / den,
        (2, DOWN, DOWN): k1 * k2z * (k1 * k1z - k0 * k0z) * E1 / den,
    }


def test_printed_three_layer_densities():
    meta = json.load(open(os.path.join(GOLD, "three_layer_densities.json")))
    k0, k1, k2 = meta["test_medium"]["k"]
    d1 = meta["test_medium"]["d"][1]
    for kk, dd in (((k0, k1, k2), d1), ((0.8, 1.2, 1.6), -1.2)):
        med = Medium(kk, [0.0, dd], eps=kk)
        kr = np.array([0.3 - 0.1j, 1.0 - 0.2j, 2.5 - 0.3j, 5.0 - 0.5j, -0.2j, 12.0 - 0.4j])
        kz = med.kz(kr)
        ref = _printed_three_layer(*kk, dd, kz)
        for (l, a, b), v in ref.items():
            s = med.sigma(kr, l, 1)[(a, b)]
            assert np.allclose(s, v, rtol=1e-12, atol=1e-15), (l, a, b)


def test_identical_layers_give_free_space():
    # All layers equal: no reflection; the only reaction component that
    # survives is the transmitted wave, equal to the free-space wave
    # (Sec. 3.1 eq. domaingreenfn).
    med = Medium([1.1, 1.1, 1.1], [0.0, -1.0], eps=[2.0, 2.0, 2.0])
    kr = np.array([0.2 - 0.3j, 1.5 - 0.3j, 4.0 - 0.3j])
    for lp in range(3):
        for l in range(3):
            sig = med.sigma(kr, l, lp)
            for (a, b), s in sig.items():
                # the surviving pair is the direct wave continuing past the
                # interface: target above the source layer carries
                # e^{ikz(z - d_l)} e^{ikz(d_{l'-1} - z')} -> (a, b) = (up, down)
                expect_one = (l < lp and (a, b) == (UP, DOWN)) or (l > lp and (a, b) == (DOWN, UP))
                if expect_one:
                    # the phase e^{ikz(d_l - d_{l'-1})} across intermediate layers
                    dl = (med.d[l] - med.d[lp - 1]) if l < lp else (med.d[lp] - med.d[l - 1])
                    expected = np.exp(1j * med.kz(kr)[0] * dl)
                    assert np.allclose(s, expected, atol=1e-14)
                else:
                    assert np.allclose(s, 0.0, atol=1e-14)


def test_equal_k_two_layer_images():
    # Equal k, unequal eps: sigma is constant; the reflected field is
    # R e^{ik|r - r*|}/(4 pi |r - r*|) with r* mirrored in z = 0 and
    # R = (eps0 - eps1)/(eps0 + eps1); the transmitted field is (1 + R) times
    # the free field (closed form by images).
    k, e0, e1 = 1.3, 1.0, 2.0
    med = Medium([k, k], [0.0], eps=[e0, e1])
    R = (e0 - e1) / (e0 + e1)
    rng = np.random.default_rng(0)
    s = rng.uniform(-1, 1, (6, 3))
    s[:, 2] = rng.uniform(0.1, 1.0, 6)
    t = np.array([0.2, -0.1, 0.35])
    rule = green.oracle_rule(med, 0.2, 3.0)
    v = green.reaction_total_spectral(med, 0, 0, t, s, rule)
    img = s.copy()
    img[:, 2] = -s[:, 2]
    assert np.allclose(v, R * green.free_kernel(k, t, img), rtol=1e-12)
    t2 = np.array([0.2, -0.1, -0.45])
    v = green.reaction_total_spectral(med, 1, 0, t2, s, green.oracle_rule(med, 0.5, 3.0))
    assert np.allclose(v, (1 + R) * green.free_kernel(k, t2, s), rtol=1e-12)


def test_equal_k_three_layer_image_series():
    # Equal k, three layers (slab of thickness D): the reflected field in the
    # top layer from a source in the top layer is the image series
    # R01 e^{..}(r - r_0) + sum_n T01 T10 R12 (R10 R12)^{n} ... (closed form by
    # images, summed to convergence).
    k, eps = 0.9, (1.0, 3.0, 1.5)
    D = 0.8
    med = Medium([k, k, k], [0.0, -D], eps=eps)

    def refl(ea, eb):        # wave in medium a hitting medium b
        return (ea - eb) / (ea + eb)
    R01, R10, R12 = refl(eps[0], eps[1]), refl(eps[1], eps[0]), refl(eps[1], eps[2])
    T01, T10 = 1 + R01, 1 + R10
    src = np.array([[0.3, -0.2, 0.4]])
    t = np.array([-0.1, 0.25, 0.7])
    zs = src[0, 2]
    val = R01 * green.free_kernel(k, t, [src[0, 0], src[0, 1], -zs])
    for n in range(0, 80):
        zimg = -zs - 2 * D * (n + 1)
        val += T01 * T10 * R12 * (R10 * R12) ** n * green.free_kernel(k, t, [src[0, 0], src[0, 1], zimg])
    got = green.reaction_total_spectral(med, 0, 0, t, src, green.oracle_rule(med, 1.0, 1.0))[0]
    assert abs(got - val) <= 1e-11 * abs(val)


def test_transmission_conditions():
    # [G] = 0 and [eps dG/dz] = 0 across every interface (reading c1), for
    # unequal k where no closed form exists.
    med = Medium([0.8, 1.2, 1.6], [0.0, -1.2], eps=[1, 2, 3])
    for lp, src in [(1, [[0.1, 0.2, -0.5]]), (0, [[0.1, 0.2, 0.3]]), (2, [[0.1, 0.2, -1.5]])]:
        src = np.array(src)
        for dj, (lu, ll) in [(0.0, (0, 1)), (-1.2, (1, 2))]:
            t = np.array([0.4, -0.3, dj])
            rule = green.oracle_rule(med, 0.1, 3.0)

            def G(l, dz):
                val = green.reaction_total_spectral(med, l, lp, t, src, rule, dz=dz)[0]
                if l == lp:
                    val += (green.free_kernel_dz if dz else green.free_kernel)(med.k[l], t, src[0])
                return val
            assert abs(G(lu, False) - G(ll, False)) <= 1e-12 * abs(G(lu, False))
            fu, fl = med.eps[lu] * G(lu, True), med.eps[ll] * G(ll, True)
            assert abs(fu - fl) <= 1e-12 * abs(fu)


def test_reciprocity():
    # eps_l G(r, r') = eps_l' G(r', r) (symmetry of div(eps grad) + eps k^2).
    med = Medium([0.8, 1.2, 1.6], [0.0, -1.2], eps=[1, 2, 3])
    pts = {0: np.array([0.3, 0.1, 0.5]), 1: np.array([-0.2, 0.4, -0.7]), 2: np.array([0.1, -0.3, -1.7])}
    rule = green.oracle_rule(med, 0.5, 3.0)
    for l in range(3):
        for lp in range(3):
            ra, rb = pts[l], pts[lp]
            if l == lp:
                rb = rb + np.array([0.2, 0.1, 0.05])
            g_ab = green.reaction_total_spectral(med, l, lp, ra, rb[None], rule)[0]
            g_ba = green.reaction_total_spectral(med, lp, l, rb, ra[None], rule)[0]
            assert abs(med.eps[l] * g_ab - med.eps[lp] * g_ba) <= 1e-12 * abs(g_ab)


def test_layer_classification_rejects_interface():
    med = Medium([1.0, 2.0], [0.0])
    assert list(med.layer_of(np.array([0.5, -0.5]))) == [0, 1]
    try:
        med.layer_of(np.array([0.0]))
    except ValueError:
        return
    raise AssertionError("point on the interface accepted")

"""Pins for oracle.specfun (Sec. 2.1-2.2)."""
import math

import numpy as np
from scipy import special as sp

from oracle import specfun as sf
from oracle.green import j0_complex
from oracle.media import Medium
from oracle.green import oracle_rule


def test_phat_real_matches_lpmv():
    # Y_n^m = (-1)^m sqrt((2n+1)/4pi (n-m)!/(n+m)!) P_n^m, P_n^m with the
    # Condon-Shortley phase as scipy defines it (Sec. 2.1).
    p = 12
    x = np.linspace(-0.999, 0.999, 37)
    P = sf.phat_all(p, x)
    for n in range(p + 1):
        for m in range(0, n + 1):
            c = math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - m) / math.factorial(n + m))
            ref = (-1) ** m * c * sp.lpmv(m, n, x)
            assert np.allclose(P[:, sf.nm(n, m)], ref, rtol=1e-12, atol=1e-13)
            assert np.allclose(P[:, sf.nm(n, -m)], (-1) ** m * ref, rtol=1e-12, atol=1e-13)


def test_ylm_orthonormal():
    p = 6
    xg, wg = np.polynomial.legendre.leggauss(20)
    th = np.arccos(xg)
    ph = 2 * math.pi * np.arange(24) / 24
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    Y = sf.ylm_all(p, TH, PH)                      # (20, 24, P)
    W = (wg[:, None] * np.full(24, 2 * math.pi / 24)[None, :])
    G = np.einsum("ab,abi,abj->ij", W, np.conj(Y), Y)
    assert np.allclose(G, np.eye(sf.ncoef(p)), atol=1e-13)


def test_branch_limits():
    # eq. (branch): +sqrt(1-x^2) from above the cut, -sqrt(1-x^2) from below.
    x = np.linspace(-0.9, 0.9, 7)
    assert np.allclose(sf.sqrt1mz2(x + 1e-14j), np.sqrt(1 - x * x), atol=1e-12)
    assert np.allclose(sf.sqrt1mz2(x - 1e-14j), -np.sqrt(1 - x * x), atol=1e-12)


def test_phat_complex_parity_and_symmetry():
    # P^_n^{-m} = (-1)^m P^_n^m and P^_n^m(-z) = (-1)^{n+m} P^_n^m(z) (Sec. 2.2)
    # hold for the continuation off the cut (z not on [-1, 1]).
    p = 10
    z = np.array([1.0 + 1.0j, 0.3 + 2.0j, 2.0 + 0.5j, 0.5 + 0.1j])
    P = sf.phat_all(p, z)
    Pm = sf.phat_all(p, -z)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            assert np.allclose(P[:, sf.nm(n, -m)], (-1) ** (m % 2) * P[:, sf.nm(n, m)])
    # for odd m the branch changes sign with z -> -z on the upper half plane:
    # the polynomial part carries (-1)^{n-m}, the root (-1), so the total is
    # (-1)^{n+m} only up to that root; check the even-m identity exactly
    for n in range(p + 1):
        for m in range(0, n + 1, 2):
            assert np.allclose(Pm[:, sf.nm(n, m)], (-1) ** ((n + m) % 2) * P[:, sf.nm(n, m)])


def _funk_hecke_rhs(p, k, kz, r, alpha):
    """sum_{n<=p} sum_m A_n^m(r) i^n P^_n^m(kz/k) e^{-i m alpha} (eq. extfunkhecke)."""
    rr, th, ph = sf.cart2sph(r)
    A = 4 * math.pi * sf.expand_n(sf.sph_jn_all(p, k * rr), p) * sf.ylm_all(p, th, ph)
    ns, ms = sf.nm_table(p)
    P = sf.phat_all(p, np.array(kz / k))
    return np.sum(A * (1j ** (ns % 4)) * P * np.exp(-1j * ms * alpha))


def test_extended_funk_hecke():
    # Prop. 2.3: the expansion holds for every complex k_z with the branch of
    # eq. (branch); the three families of Fig. FunkHeckeApperr (r = (0.3, 0.4, z),
    # alpha = pi/4).
    alpha = math.pi / 4
    cases = []
    for k in (1.0, 1.8, 3.0):
        cases.append((k, 1 + 1j, 0.5))                 # (a) z = 0.5, k_z = 1 + i
    for z in (0.2, 0.5, 1.0):
        cases.append((1.8, 1 - 1.3j, z))               # (b) k = 1.8, k_z = 1 - 1.3 i
    for kz in (0.5, 2.0j, 1 + 1j, 1 - 1.3j, 2.5 + 0.2j):
        cases.append((1.8, kz, 0.5))                   # (c) z = 0.5, k = 1.8
    for k, kz, z in cases:
        r = np.array([0.3, 0.4, z])
        krho = k * sf.sqrt1mz2(np.array(kz / k))
        lhs = np.exp(1j * (krho * (r[0] * math.cos(alpha) + r[1] * math.sin(alpha)) + kz * r[2]))
        rhs = _funk_hecke_rhs(40, k, kz, r, alpha)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (k, kz, z, abs(lhs - rhs) / abs(lhs))


def test_branch_gives_krho_on_contours():
    # The Sommerfeld integrals use P^_n^m(k_z/k) with k_rho the integration
    # variable; the branch must give k * sqrt(1 - (k_z/k)^2) = k_rho on both
    # the oracle contour and the Gamma1 u Gamma2 contour of Sec. 3.5.
    med = Medium([0.8, 1.2, 1.6], [0.0, -1.2])
    kr, _, _ = oracle_rule(med, 0.3, 2.0)
    b = 0.4
    g1 = -1j * np.linspace(1e-3, b, 9)
    g2 = np.linspace(0.0, 40.0, 101) - 1j * b
    for nodes in (kr[:len(kr) // 3], g1, g2):
        kz = med.kz(nodes)
        for j, k in enumerate(med.k):
            s = k * sf.sqrt1mz2(kz[j] / k)
            assert np.allclose(s, nodes, rtol=1e-12, atol=1e-12)


def test_j0_series_matches_scipy():
    z = (np.random.default_rng(0).uniform(0, 12, 400) * np.exp(-1j * np.random.default_rng(1).uniform(0, 0.6, 400)))
    assert np.allclose(j0_complex(z), sp.jv(0, z), rtol=1e-11, atol=1e-12)

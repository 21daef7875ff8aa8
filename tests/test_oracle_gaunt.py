"""Pins for oracle.gaunt (Sec. 2.1)."""
import math

import numpy as np

from oracle import specfun as sf
from oracle.gaunt import gaunt, wigner3j


def test_wigner3j_textbook_values():
    assert abs(wigner3j(1, 1, 0, 0, 0, 0) + 1 / math.sqrt(3)) < 1e-15
    assert abs(wigner3j(1, 1, 2, 0, 0, 0) - math.sqrt(2 / 15)) < 1e-15
    assert abs(wigner3j(2, 2, 2, 0, 0, 0) + math.sqrt(2 / 35)) < 1e-15
    assert abs(wigner3j(1, 1, 1, 1, -1, 0) - 1 / math.sqrt(6)) < 1e-15
    assert wigner3j(1, 1, 1, 0, 0, 0) == 0.0
    assert wigner3j(2, 1, 0, 0, 0, 0) == 0.0


def test_wigner3j_orthogonality():
    # sum_{m1,m2} (j1 j2 j3; m1 m2 m3)(j1 j2 j3'; m1 m2 m3) = delta / (2 j3 + 1)
    j1, j2 = 3, 2
    for j3 in range(1, 6):
        for m3 in range(-j3, j3 + 1):
            s = sum(wigner3j(j1, j2, j3, m1, -m1 - m3, m3) ** 2
                    for m1 in range(-j1, j1 + 1) if abs(-m1 - m3) <= j2)
            assert abs(s - 1 / (2 * j3 + 1)) < 1e-14


def test_gaunt_is_triple_harmonic_integral():
    # G(n,m; nu,mu; q) = int Y_n^m Y_nu^mu conj(Y_q^{m+mu}) dOmega, by exact
    # Gauss-Legendre x trapezoid quadrature on the sphere.
    p = 5
    xg, wg = np.polynomial.legendre.leggauss(3 * p + 2)
    nph = 6 * p + 4
    th = np.arccos(xg)
    ph = 2 * math.pi * np.arange(nph) / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    Y = sf.ylm_all(2 * p, TH, PH)
    W = wg[:, None] * (2 * math.pi / nph)
    for n in range(p + 1):
        for nu in range(p + 1):
            for q in range(abs(n - nu), n + nu + 1):
                for m in range(-n, n + 1):
                    for mu in range(-nu, nu + 1):
                        if abs(m + mu) > q:
                            continue
                        integ = np.sum(W * Y[..., sf.nm(n, m)] * Y[..., sf.nm(nu, mu)]
                                       * np.conj(Y[..., sf.nm(q, m + mu)]))
                        assert abs(integ - gaunt(n, m, nu, mu, q)) < 1e-13, (n, m, nu, mu, q)

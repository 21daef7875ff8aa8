"""Wigner 3-j symbols and Gaunt coefficients (Sec. 2.1).

G(n,m; nu,mu; q) = (-1)^{m+mu} S (n nu q; 0 0 0)(n nu q; m mu -m-mu),
S = sqrt((2n+1)(2nu+1)(2q+1) / (4 pi)).

The 3-j symbol is Racah's closed formula evaluated with exact integers
(fractions.Fraction); only the final square root and product are rounded.

Pins: tests/test_oracle_gaunt.py (textbook 3-j values; the Gaunt coefficient
as the integral of three spherical harmonics computed by exact quadrature on
the sphere; selection rules).
"""
import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

from .specfun import nm, ncoef


@lru_cache(maxsize=None)
def wigner3j(j1, j2, j3, m1, m2, m3):
    """(j1 j2 j3; m1 m2 m3) for integer arguments by Racah's formula."""
    if m1 + m2 + m3 != 0:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    f = math.factorial
    tri = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pref2 = tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    s = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (f(k) * f(j3 - j2 + k + m1) * f(j3 - j1 + k - m2) * f(j1 + j2 - j3 - k)
               * f(j1 - k - m1) * f(j2 - k + m2))
        s += Fraction((-1) ** k, den)
    sign = -1 if (j1 - j2 - m3) % 2 else 1
    if s == 0:
        return 0.0
    val2 = pref2 * s * s                 # exact square of |value|
    mag = math.sqrt(val2.numerator) / math.sqrt(val2.denominator) \
        if val2.numerator < 2 ** 1000 else math.sqrt(float(val2))
    return float(sign * (1 if s > 0 else -1) * mag)


@lru_cache(maxsize=None)
def gaunt(n, m, nu, mu, q):
    """Gaunt coefficient G(n,m; nu,mu; q) as defined in Sec. 2.1."""
    if (n + nu + q) % 2:
        return 0.0
    S = math.sqrt((2 * n + 1) * (2 * nu + 1) * (2 * q + 1) / (4.0 * math.pi))
    w0 = wigner3j(n, nu, q, 0, 0, 0)
    if w0 == 0.0:
        return 0.0
    w1 = wigner3j(n, nu, q, m, mu, -m - mu)
    return (-1) ** ((m + mu) % 2) * S * w0 * w1


@lru_cache(maxsize=None)
def gaunt_table(p):
    """Dense table G[(n,m), (nu,mu), q] = G(n,m; nu,-mu; q) for n, nu <= p,
    q <= 2p (the combination appearing in eqs. spmhat3d / singularseparation)."""
    P = ncoef(p)
    T = np.zeros((P, P, 2 * p + 1))
    for n in range(p + 1):
        for m in range(-n, n + 1):
            for nu in range(p + 1):
                for mu in range(-nu, nu + 1):
                    for q in range(abs(n - nu), n + nu + 1):
                        if abs(mu - m) <= q:
                            T[nm(n, m), nm(nu, mu), q] = gaunt(n, m, nu, -mu, q)
    return T

"""Special functions for the oracle (FP64).

Coefficient layout used throughout the oracle: degree n = 0..p, order
m = -n..n, flat index ``n*n + n + m``; (p+1)**2 entries.

Pins: tests/test_oracle_specfun.py (scipy's lpmv for real arguments, the
extended Funk-Hecke identity of Prop. 2.3 for complex k_z, the relation
between the branch of eq. (branch) and k_rho on both contours, parity and
reflection identities).
"""
import math

import numpy as np
from scipy import special as sp


def nm(n, m):
    """Flat index of (n, m)."""
    return n * n + n + m


def ncoef(p):
    return (p + 1) * (p + 1)


def nm_table(p):
    """Arrays n[i], m[i] for the flat layout."""
    ns, ms = [], []
    for n in range(p + 1):
        for m in range(-n, n + 1):
            ns.append(n)
            ms.append(m)
    return np.array(ns), np.array(ms)


def sqrt1mz2(z):
    """Branch of sqrt(1 - z^2) chosen in Sec. 2.2, eq. (branch).

    With z+1 = r1 e^{i t1}, z-1 = r2 e^{i t2} (principal arguments) the branch
    is -i sqrt(r1 r2) e^{i (t1+t2)/2}, i.e. -i * sqrt(z+1) * sqrt(z-1) with
    principal square roots.  It is cut along [-1, 1] and tends to
    +sqrt(1-x^2) from above the cut.
    """
    z = np.asarray(z, dtype=complex)
    return -1j * np.sqrt(z + 1.0) * np.sqrt(z - 1.0)


def _ab(n, m):
    """Recurrence coefficients a_n^m, b_n^m of Sec. 2.2."""
    a = math.sqrt((2 * n - 1) * (2 * n + 1) / ((n - m) * (n + m)))
    if n - m - 1 <= 0:
        b = 0.0
    else:
        b = math.sqrt((2 * n + 1) * (n - m - 1) * (n + m - 1)
                      / ((2 * n - 3) * (n + m) * (n - m)))
    return a, b


def phat_all(p, z, s=None):
    """Normalized associated Legendre functions P^_n^m(z), all n <= p, |m| <= n.

    Follows the recurrences of Sec. 2.2 (after Prop. 2.3's branch):
      P^_0^0 = 1/sqrt(4 pi)   (the printed "1/(4 pi)" is read as 1/sqrt(4 pi):
                              Y_0^0 = P^_0^0 must be 1/sqrt(4 pi)),
      P^_n^n = sqrt((2n+1)/(2n)) * s * P^_{n-1}^{n-1},  s = sqrt(1-z^2) (branch),
      P^_n^m = a_n^m z P^_{n-1}^m - b_n^m P^_{n-2}^m,
      P^_n^{-m} = (-1)^m P^_n^m.
    ``z`` may be real (then s = +sqrt(1-z^2), z in [-1,1]) or complex (then
    s follows eq. (branch)); ``s`` may be passed explicitly.
    Returns an array of shape z.shape + ((p+1)^2,).
    """
    z = np.asarray(z)
    if s is None:
        if np.iscomplexobj(z):
            s = sqrt1mz2(z)
        else:
            s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    dtype = complex if (np.iscomplexobj(z) or np.iscomplexobj(s)) else float
    out = np.zeros(z.shape + (ncoef(p),), dtype=dtype)
    diag = np.full(z.shape, 1.0 / math.sqrt(4.0 * math.pi), dtype=dtype)
    for m in range(p + 1):
        if m > 0:
            diag = math.sqrt((2 * m + 1) / (2 * m)) * s * diag
        out[..., nm(m, m)] = diag
        prev2 = np.zeros_like(diag)
        prev1 = diag
        for n in range(m + 1, p + 1):
            a, b = _ab(n, m)
            cur = a * z * prev1 - b * prev2
            out[..., nm(n, m)] = cur
            prev2, prev1 = prev1, cur
    for n in range(1, p + 1):
        for m in range(1, n + 1):
            out[..., nm(n, -m)] = (-1) ** m * out[..., nm(n, m)]
    return out


def ylm_all(p, theta, phi):
    """Spherical harmonics Y_n^m(theta, phi) = P^_n^m(cos theta) e^{i m phi} (Sec. 2.1)."""
    theta = np.asarray(theta, dtype=float)
    phi = np.asarray(phi, dtype=float)
    P = phat_all(p, np.cos(theta), s=np.abs(np.sin(theta)))
    _, ms = nm_table(p)
    return P * np.exp(1j * ms * phi[..., None])


def cart2sph(v):
    """(r, theta, phi) of vectors v[..., 3]; theta = phi = 0 at the origin."""
    v = np.asarray(v, dtype=float)
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    r = np.sqrt(x * x + y * y + z * z)
    with np.errstate(invalid="ignore", divide="ignore"):
        ct = np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0)
    theta = np.arccos(np.clip(ct, -1.0, 1.0))
    phi = np.arctan2(y, x)
    return r, theta, phi


def sph_jn_all(p, x):
    """Spherical Bessel j_n(x), n = 0..p, real x (scipy).  Shape x.shape + (p+1,)."""
    x = np.asarray(x, dtype=float)
    return np.stack([sp.spherical_jn(n, x) for n in range(p + 1)], axis=-1)


def sph_hn_all(p, x):
    """Spherical Hankel h_n^(1)(x) = j_n + i y_n, n = 0..p, real x > 0 (scipy)."""
    x = np.asarray(x, dtype=float)
    return np.stack([sp.spherical_jn(n, x) + 1j * sp.spherical_yn(n, x)
                     for n in range(p + 1)], axis=-1)


def expand_n(arr_n, p):
    """Repeat a per-degree array [..., p+1] onto the flat (n, m) layout."""
    ns, _ = nm_table(p)
    return arr_n[..., ns]


def besselj(n, z):
    """Cylindrical Bessel J_n(z), integer n, real or complex z (scipy)."""
    return sp.jv(n, z)

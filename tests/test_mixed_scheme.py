"""The number scheme of the mixed-precision M2L, emulated on the CPU with the
oracle's operators and multipole expansions: per-degree power-of-two scaling
by s_n = (k rho)^n / (2n+1)!!, one power-of-two shift per operator and per
column, real split [Ar -Ai; Ai Ar], FP16 hi/lo parts and three products
(hi*hi + hi*lo + lo*hi) accumulated in FP32.  The translated coefficients,
weighted by s_n as they enter the potential, keep a relative error of a few
1e-7 -- far inside the 1e-5 bound of the mixed form -- while a single FP16
product (no lo parts) does not."""
import math

import numpy as np
import pytest

from oracle import fmm
from oracle import specfun as sf


def _exp2_floor(x):
    return math.frexp(x)[1] - 1


def _emulate(A, Y, En, three_products=True):
    As = A * 2.0 ** (En[:, None] + En[None, :])
    mx = max(np.abs(As.real).max(), np.abs(As.imag).max())
    sh = math.frexp(mx)[1] - 15
    As = As * 2.0 ** (-sh)
    Ys = Y * 2.0 ** (-En[:, None])
    ek = np.array([math.frexp(max(np.abs(c.real).max(), np.abs(c.imag).max()))[1] for c in Ys.T])
    Ys = Ys * 2.0 ** (-ek[None, :])

    def split(x):
        h = x.astype(np.float32).astype(np.float16)
        lo = (x.astype(np.float32) - h.astype(np.float32)).astype(np.float16)
        return h, lo

    B = np.block([[As.real, -As.imag], [As.imag, As.real]])
    yv = np.vstack([Ys.real, Ys.imag])
    Bh, Bl = split(B)
    yh, yl = split(yv)
    f = lambda a, b: a.astype(np.float32) @ b.astype(np.float32)
    D = f(Bh, yh) + (f(Bh, yl) + f(Bl, yh) if three_products else 0)
    P = A.shape[0]
    return (D[:P] + 1j * D[P:]).astype(np.complex128) * 2.0 ** (sh - En[:, None]) * 2.0 ** ek[None, :]


@pytest.mark.parametrize("p,lev", [(8, 3), (10, 5)])
def test_scaled_split_product(p, lev):
    k, w = 1.6, 3.4 / 2 ** lev
    P = (p + 1) ** 2
    A = fmm.free_m2l_matrix(p, k, np.array([2 * w, w, -2 * w]), np.zeros(3))
    rng = np.random.default_rng(lev)
    Y = np.array([fmm.p2m(p, k, np.zeros(3), rng.uniform(-w / 2, w / 2, (40, 3)), rng.uniform(0, 1, 40))
                  for _ in range(48)]).T
    deg = np.array([math.isqrt(i) for i in range(P)])
    s = np.array([(k * math.sqrt(3) / 2 * w) ** n / math.prod(range(1, 2 * n + 2, 2)) for n in deg])
    En = np.array([_exp2_floor(v) for v in s], dtype=float)
    ref = A @ Y
    weighted = lambda Z: np.linalg.norm((Z - ref) * s[:, None]) / np.linalg.norm(ref * s[:, None])
    err3 = weighted(_emulate(A, Y, En))
    err1 = weighted(_emulate(A, Y, En, three_products=False))
    assert err3 < 1e-6, err3
    assert err1 > 20 * err3, (err1, err3)

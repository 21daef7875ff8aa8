"""The identity behind the rotation form of the translations (CPU, oracle
functions only): for a rotation Q taking the offset b to |b| z and W the
block-diagonal matrix of Y_n^m(Q x) = sum_m' W[m, m'] Y_n^m'(x), every
translation of the method factors as
    op(b) = W^T op(|b| z) conj(W),
and op(|b| z) couples only equal orders m -- for the free-space M2L
(Thm. 2.3) and for the M2M / L2L shifts (eq. metome).  W is computed by an
exact product quadrature on the sphere."""
import math

import numpy as np
import pytest

from oracle import fmm
from oracle import specfun as sf

P_ORDER, K = 6, 1.3


def _rot_to_z(bhat):
    th = math.acos(max(-1.0, min(1.0, bhat[2])))
    ph = math.atan2(bhat[1], bhat[0])
    rz = np.array([[math.cos(ph), math.sin(ph), 0], [-math.sin(ph), math.cos(ph), 0], [0, 0, 1]])
    ry = np.array([[math.cos(th), 0, -math.sin(th)], [0, 1, 0], [math.sin(th), 0, math.cos(th)]])
    return ry @ rz


def _w_matrix(p, Q):
    xg, wg = np.polynomial.legendre.leggauss(p + 2)
    nphi = 2 * p + 2
    pts, wts = [], []
    for ct, wc in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            pts.append([st * math.cos(ph), st * math.sin(ph), ct])
            wts.append(wc * 2 * math.pi / nphi)
    pts, wts = np.array(pts), np.array(wts)

    def Y(v):
        _, th, ph = sf.cart2sph(v)
        return sf.ylm_all(p, th, ph)

    Yx, Yq = Y(pts), Y(pts @ Q.T)
    P = (p + 1) ** 2
    W = np.zeros((P, P), complex)
    for n in range(p + 1):
        idx = np.arange(n * n, n * n + 2 * n + 1)
        W[np.ix_(idx, idx)] = (Yq[:, idx] * wts[:, None]).T @ np.conj(Yx[:, idx])
    return W


@pytest.mark.parametrize("d", [(2, 1, -1), (-3, 2, 0), (0, 0, -2), (3, 3, 3)])
def test_free_space_m2l_factors(d):
    w = 0.15
    b = np.array(d, float) * w
    Q = _rot_to_z(b / np.linalg.norm(b))
    W = _w_matrix(P_ORDER, Q)
    assert np.abs(W @ W.conj().T - np.eye(len(W))).max() < 1e-13         # unitary
    A = fmm.free_m2l_matrix(P_ORDER, K, b, np.zeros(3))
    Az = fmm.free_m2l_matrix(P_ORDER, K, np.array([0.0, 0.0, np.linalg.norm(b)]), np.zeros(3))
    _, ms = sf.nm_table(P_ORDER)
    assert np.abs(Az[ms[:, None] != ms[None, :]]).max() == 0.0
    assert np.abs(W.T @ Az @ np.conj(W) - A).max() < 1e-13 * np.abs(A).max()


@pytest.mark.parametrize("signs", [(1, -1, 1), (-1, -1, -1), (1, 1, 1)])
def test_shifts_factor(signs):
    w = 0.2
    b = 0.5 * w * np.array(signs, float)
    Q = _rot_to_z(b / np.linalg.norm(b))
    W = _w_matrix(P_ORDER, Q)
    bz = np.array([0.0, 0.0, np.linalg.norm(b)])
    for op in (lambda v: np.conj(fmm.sep_matrix(P_ORDER, K, v, True)),      # M2M
               lambda v: fmm.sep_matrix(P_ORDER, K, v, True).T):            # L2L
        A, Az = op(b), op(bz)
        assert np.abs(W.T @ Az @ np.conj(W) - A).max() < 1e-13 * np.abs(A).max()

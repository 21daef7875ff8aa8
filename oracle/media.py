"""Layered medium and reaction densities (Sec. 3.1).

Layers l = 0..L from top to bottom; interfaces d_0 > d_1 > ... > d_{L-1};
layer l is d_l < z < d_{l-1} with d_{-1} = +inf, d_L = -inf.

The paper defers the interface conditions to its reference [wang2018]; the
oracle takes [u] = 0 and [eps * du/dz] = 0 at every interface, with eps the
per-layer material coefficient (reading c1).  The paper's printed three-layer
densities correspond to eps_l = k_l; the test of those formulas uses that.

Reaction densities are obtained from first principles, as Sec. 3.1 describes
("solve a linear system"): in the Fourier (k_x, k_y) domain the field in layer
j is A_j e^{i k_jz (z - d_j)} + B_j e^{i k_jz (d_{j-1} - z)} plus, in the
source layer l', the free wave (i / 2k_l'z) e^{i k_l'z |z - z'|}.  No wave
enters from z = +-inf (B_0 = A_L = 0).  Imposing the two transmission
conditions at the L interfaces gives a 2L x 2L system, solved here directly
(numpy.linalg.solve) for two unit excitations: the source wave arriving at the
bottom interface d_l' ("dn", carries e^{i k_l'z (z' - d_l')}) and at the top
interface d_{l'-1} ("up", carries e^{i k_l'z (d_{l'-1} - z')}).  Matching the
result to eqs. (greenfuncomponent)-(totaldensity) gives

  sigma^{a b}_{l l'} = (k_lz / k_l'z) * X,   X = A_l (a = up) or B_l (a = down)
                                              for excitation dn (b = up) or up (b = down).

Pins: tests/test_oracle_media.py (printed three-layer formulas, equal-k
closed form, identical layers, transmission conditions of the full Green's
function, reciprocity).
"""
import numpy as np

UP, DOWN = 0, 1          # arrow values for a (target side) and b (source side)
ARROW = {UP: "u", DOWN: "d"}


class Medium:
    def __init__(self, k, d=(), eps=None):
        self.k = np.asarray(k, dtype=float)
        self.d = np.asarray(d, dtype=float)
        self.L = len(self.k) - 1
        if self.L < 0:
            raise ValueError("need at least one layer")
        if len(self.d) != self.L:
            raise ValueError("need L interfaces for L+1 layers")
        if np.any(self.k <= 0):
            raise ValueError("wave numbers must be positive")
        if self.L > 1 and np.any(np.diff(self.d) >= 0):
            raise ValueError("interfaces must be strictly decreasing")
        self.eps = np.ones(self.L + 1) if eps is None else np.asarray(eps, dtype=float)
        if len(self.eps) != self.L + 1 or np.any(self.eps <= 0):
            raise ValueError("need L+1 positive material coefficients")

    # -- geometry ---------------------------------------------------------
    def layer_of(self, z):
        """Layer index of each z; raises on a point exactly on an interface."""
        z = np.asarray(z, dtype=float)
        if np.any(np.isin(z, self.d)):
            raise ValueError("point on an interface")
        # layer l: d_l < z < d_{l-1}  <=>  number of interfaces above z
        return np.sum(z[..., None] < self.d[None, :], axis=-1).astype(int)

    def top(self, l):
        """d_{l-1} (the interface above layer l)."""
        return self.d[l - 1]

    def bottom(self, l):
        """d_l (the interface below layer l)."""
        return self.d[l]

    def arrows_target(self, l):
        """Allowed a for targets in layer l (eq. generalreact)."""
        out = []
        if l < self.L:
            out.append(UP)
        if l > 0:
            out.append(DOWN)
        return out

    def arrows_source(self, lp):
        """Allowed b for sources in layer l' (eq. totaldensity)."""
        return self.arrows_target(lp)

    def delta_t(self, a, l, z):
        """Target distance to the reference interface: z - d_l (a=up), d_{l-1} - z (a=down)."""
        return (z - self.d[l]) if a == UP else (self.d[l - 1] - z)

    def delta_s(self, b, lp, zp):
        """Source distance: z' - d_l' (b=up), d_{l'-1} - z' (b=down)."""
        return (zp - self.d[lp]) if b == UP else (self.d[lp - 1] - zp)

    # -- spectral quantities --------------------------------------------
    def kz(self, kr):
        """k_jz = sqrt(k_j^2 - k_rho^2), principal branch (Re >= 0, Im >= 0 on
        the contours used), shape (L+1,) + kr.shape."""
        kr = np.asarray(kr, dtype=complex)
        arg = self.k[:, None] ** 2 - (kr ** 2)[None, ...] if kr.ndim else self.k ** 2 - kr ** 2
        out = np.sqrt(arg)
        # On the real axis beyond k_j the argument is negative real; the limit
        # from the fourth quadrant is +i sqrt(k_rho^2 - k_j^2).
        return np.where((out.imag < 0), -out, out)

    def unit_responses(self, kr, lp):
        """Reaction amplitudes (A_j, B_j) for the unit excitations of a source
        in layer l'.  Returns dict exc -> (A[L+1, Q], B[L+1, Q]) with exc in
        {'dn', 'up'} (only those that exist)."""
        L = self.L
        kr = np.atleast_1d(np.asarray(kr, dtype=complex))
        Q = kr.shape[0]
        kz = self.kz(kr)                                    # (L+1, Q)
        # thickness phase of finite layers 1..L-1
        e = np.zeros((L + 1, Q), dtype=complex)
        for j in range(1, L):
            e[j] = np.exp(1j * kz[j] * (self.d[j - 1] - self.d[j]))
        # unknown ordering: A_0..A_{L-1}, then B_1..B_L
        def ia(j):
            return j

        def ib(j):
            return L + j - 1

        n = 2 * L
        M = np.zeros((Q, n, n), dtype=complex)
        for j in range(L):                 # interface d_j between layers j and j+1
            rc, rf = 2 * j, 2 * j + 1
            up, lo = j, j + 1
            M[:, rc, ia(up)] += 1.0
            M[:, rf, ia(up)] += self.eps[up] * 1j * kz[up]
            if up >= 1:
                M[:, rc, ib(up)] += e[up]
                M[:, rf, ib(up)] += -self.eps[up] * 1j * kz[up] * e[up]
            if lo <= L - 1:
                M[:, rc, ia(lo)] += -e[lo]
                M[:, rf, ia(lo)] += -self.eps[lo] * 1j * kz[lo] * e[lo]
            M[:, rc, ib(lo)] += -1.0
            M[:, rf, ib(lo)] += self.eps[lo] * 1j * kz[lo]
        out = {}
        excs = []
        if lp <= L - 1:
            # source wave of unit value at z = d_l' (from above), derivative -i k z
            rhs = np.zeros((Q, n), dtype=complex)
            rhs[:, 2 * lp] = -1.0
            rhs[:, 2 * lp + 1] = self.eps[lp] * 1j * kz[lp]
            excs.append(("dn", rhs))
        if lp >= 1:
            # source wave of unit value at z = d_{l'-1} (from below), derivative +i k z
            rhs = np.zeros((Q, n), dtype=complex)
            rhs[:, 2 * (lp - 1)] = 1.0
            rhs[:, 2 * (lp - 1) + 1] = self.eps[lp] * 1j * kz[lp]
            excs.append(("up", rhs))
        for name, rhs in excs:
            x = np.linalg.solve(M, rhs[..., None])[..., 0]   # (Q, n)
            A = np.zeros((L + 1, Q), dtype=complex)
            B = np.zeros((L + 1, Q), dtype=complex)
            for j in range(L):
                A[j] = x[:, ia(j)]
            for j in range(1, L + 1):
                B[j] = x[:, ib(j)]
            out[name] = (A, B)
        return out

    def sigma(self, kr, l, lp):
        """Reaction densities sigma^{ab}_{l l'}(k_rho) (eq. totaldensity).
        Returns dict (a, b) -> complex array over kr."""
        if self.L == 0:
            return {}
        kr = np.atleast_1d(np.asarray(kr, dtype=complex))
        kz = self.kz(kr)
        resp = self.unit_responses(kr, lp)
        ratio = kz[l] / kz[lp]
        out = {}
        for a in self.arrows_target(l):
            for b in self.arrows_source(lp):
                exc = "dn" if b == UP else "up"
                A, B = resp[exc]
                X = A[l] if a == UP else B[l]
                out[(a, b)] = ratio * X
        return out

"""Seeded synthetic workloads shaped like the paper's experiments.

This module holds no arithmetic of the method: it only describes media and
draws particle positions and charges from a seeded generator.  It is shared
by the tests, the benchmark and the oracle-side checks.

Each workload returns a dict with keys
  k, d, eps      -- wave numbers (top to bottom), interfaces, material coefficients
  p, leaf        -- expansion order and leaf size
  src, q, tgt    -- float64 [N,3] sources, complex128 [N] charges, targets
"""
import numpy as np


def _cube(rng, n, zlo, zhi):
    x = rng.uniform(-1.0, 1.0, n)
    y = rng.uniform(-1.0, 1.0, n)
    z = rng.uniform(zlo, zhi, n)
    return np.stack([x, y, z], axis=1)


def _split(n, parts):
    base = n // parts
    out = [base] * parts
    for i in range(n - base * parts):
        out[i] += 1
    return out


def two_layer(n=1000, seed=0, p=5, leaf=40):
    """Two layers, interface z = 0, k = (1.0, 1.5), eps = (1, 2); half the
    points uniform in [-1,1]^2 x [0.1,1.1], half in [-1,1]^2 x [-1.1,-0.1];
    real charges U[0,1]; targets = sources."""
    rng = np.random.default_rng(seed)
    n0, n1 = _split(n, 2)
    src = np.concatenate([_cube(rng, n0, 0.1, 1.1), _cube(rng, n1, -1.1, -0.1)])
    q = rng.uniform(0.0, 1.0, n).astype(complex)
    return dict(k=[1.0, 1.5], d=[0.0], eps=[1.0, 2.0], p=p, leaf=leaf,
                src=src, q=q, tgt=src.copy(), name=f"two-layer N={n} p={p} leaf={leaf}")


THREE_LAYER_CUBES = ((0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3))


def three_layer(n=32768, seed=0, p=8, leaf=64, complex_charges=False):
    """Three layers, interfaces z = 0 and -1.2, k = (0.8, 1.2, 1.6),
    eps = (1, 2, 3); n points split evenly over the cubes [-1,1]^2 x
    {[0.1,1.1], [-1.1,-0.1], [-2.3,-1.3]}; charges U[0,1] (or complex with
    Re, Im ~ U[-1,1]); targets = sources."""
    rng = np.random.default_rng(seed)
    parts = _split(n, 3)
    src = np.concatenate([_cube(rng, m, lo, hi) for m, (lo, hi) in zip(parts, THREE_LAYER_CUBES)])
    if complex_charges:
        q = rng.uniform(-1.0, 1.0, n) + 1j * rng.uniform(-1.0, 1.0, n)
    else:
        q = rng.uniform(0.0, 1.0, n).astype(complex)
    return dict(k=[0.8, 1.2, 1.6], d=[0.0, -1.2], eps=[1.0, 2.0, 3.0], p=p, leaf=leaf,
                src=src, q=q, tgt=src.copy(), name=f"three-layer N={n} p={p} leaf={leaf}")


def sample_targets(n, count, seed=1):
    """Seeded sample of target indices (sorted, distinct)."""
    rng = np.random.default_rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False))


def batched(n_problems=64, seed=0, n_min=10_000, n_max=200_000, p=10, leaf=64):
    """Independent problems of uneven size: N log-uniform in [n_min, n_max],
    2-5 layers, interior layer thickness U[0.8, 1.5] (first interface at
    z = 0), k_l ~ U[0.5, 3.0], eps_l = 1 + l, real charges U[0,1], targets =
    sources.  Points lie in [-1,1]^2 x slabs kept 0.1 away from the
    interfaces: the interior of each interior layer, and a slab of thickness
    1 on the far side of the top and bottom interfaces; a layer receives
    points in proportion to its slab thickness."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        L1 = int(rng.integers(2, 6))
        d = [0.0]
        for _ in range(L1 - 2):
            d.append(d[-1] - rng.uniform(0.8, 1.5))
        k = list(rng.uniform(0.5, 3.0, L1))
        eps = [1.0 + l for l in range(L1)]
        slabs = [(d[0] + 0.1, d[0] + 1.1)]
        for j in range(1, L1 - 1):
            slabs.append((d[j] + 0.1, d[j - 1] - 0.1))
        slabs.append((d[-1] - 1.1, d[-1] - 0.1))
        th = np.array([hi - lo for lo, hi in slabs])
        counts = np.floor(n * th / th.sum()).astype(int)
        counts[: n - counts.sum()] += 1
        src = np.concatenate([_cube(rng, m, lo, hi) for m, (lo, hi) in zip(counts, slabs)])
        q = rng.uniform(0.0, 1.0, n).astype(complex)
        out.append(dict(k=k, d=d, eps=eps, p=p, leaf=leaf, src=src, q=q, tgt=src.copy(),
                        name=f"batched problem {i}: N={n}, {L1} layers"))
    return out


PAPER_DOMAINS = (((0.0, 0.0, 0.6), 0.10), ((0.0, 0.0, -0.6), 0.15), ((0.0, 0.0, -1.8), 0.05))


def _in_domain(rng, n, center, a):
    """n points uniform inside r(theta) = 0.5 - a + a P_4(cos theta) about
    `center` (rejection from the enclosing ball of radius 0.5)."""
    out = []
    while len(out) < n:
        p = rng.uniform(-0.5, 0.5, (4 * n, 3))
        r = np.linalg.norm(p, axis=1)
        c = np.divide(p[:, 2], r, out=np.zeros_like(r), where=r > 0)
        p4 = (35 * c ** 4 - 30 * c ** 2 + 3) / 8
        keep = p[r < 0.5 - a + a * p4]
        out.extend(keep[: n - len(out)])
    return np.asarray(out) + np.asarray(center)


def paper_domains(counts=(912, 640, 1296), seed=0, p=6, leaf=40):
    """The paper's shaped test: three layers with interfaces z = 0 and -1.2,
    k = (1.2, 1.5, 1.8), eps = (1, 2, 3); particles uniform inside the
    irregular domains r = 0.5 - a + a P_4(cos theta), a = 0.1, 0.15, 0.05,
    centred at (0, 0, 0.6), (0, 0, -0.6), (0, 0, -1.8) (one per layer);
    real charges U[0,1]; targets = sources."""
    rng = np.random.default_rng(seed)
    src = np.concatenate([_in_domain(rng, m, c, a) for m, (c, a) in zip(counts, PAPER_DOMAINS)])
    q = rng.uniform(0.0, 1.0, len(src)).astype(complex)
    n = len(src)
    return dict(k=[1.2, 1.5, 1.8], d=[0.0, -1.2], eps=[1.0, 2.0, 3.0], p=p, leaf=leaf,
                src=src, q=q, tgt=src.copy(), name=f"paper domains N={n} p={p} leaf={leaf}")

"""Host-side checks of the seeded workload generators (no method arithmetic)."""
import numpy as np

from paper_1902_05132_gb300 import workloads


def test_paper_domains_inside_their_shapes_and_layers():
    w = workloads.paper_domains()
    src = w["src"]
    assert len(src) == 912 + 640 + 1296
    starts = np.cumsum([0, 912, 640, 1296])
    for i, (c, a) in enumerate(workloads.PAPER_DOMAINS):
        p = src[starts[i]:starts[i + 1]] - np.asarray(c)
        r = np.linalg.norm(p, axis=1)
        ct = p[:, 2] / r
        assert (r < 0.5 - a + a * (35 * ct ** 4 - 30 * ct ** 2 + 3) / 8).all()
    z = src[:, 2]
    assert (z[:912] > 0).all() and ((z[912:1552] < 0) & (z[912:1552] > -1.2)).all() and (z[1552:] < -1.2).all()
    again = workloads.paper_domains()
    assert np.array_equal(again["src"], src) and np.array_equal(again["q"], w["q"])


def test_batched_recipe():
    ws = workloads.batched(8, seed=3, n_min=1000, n_max=5000)
    for w in ws:
        L1 = len(w["k"])
        assert 2 <= L1 <= 5 and len(w["d"]) == L1 - 1
        assert 1000 <= len(w["src"]) <= 5000
        assert all(0.5 <= k <= 3.0 for k in w["k"])
        d = np.asarray(w["d"])
        z = w["src"][:, 2]
        gap = np.min(np.abs(z[:, None] - d[None, :]), axis=1)
        assert (gap >= 0.1 - 1e-12).all()          # kept 0.1 away from every interface

"""Learned surrogate of the reaction components (mixed + surrogate form).

The quadrature of the library (pinned to the oracle's direct sum by
test_gpu_direct) generates the training data and judges the surrogate: a cell
of the input box is used only if its held-out error is within the bound.
Checked here: the report is complete, a strict bound leaves the direct sum
identical to the quadrature wherever no cell passed, and under a loose bound
the surrogate's direct sum stays within that bound of the quadrature's."""
import numpy as np
import pytest

from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu

BOX = dict(rho_max=2.9, z_min=0.09, z_max=1.11)     # the two-layer point slabs, 0.1..1.1 from the interface


def _solvers(pkg, w):
    plain = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    surr = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], surrogate=True)
    return plain, surr


def test_surrogate_report_and_strict_bound():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer(n=400)
    plain, surr = _solvers(pkg, w)
    err, ok = surr.train_surrogate(**BOX, samples=131072, steps=1500, bound=1e-5, seed=1)
    # two layers: components (0,0,up,up), (0,1,up,down), (1,0,down,up), (1,1,down,down)
    L1 = 2
    slots = [((l * L1 + lp) * 2 + a) * 2 + b for l in range(2) for lp in range(2) for a in range(2) for b in range(2)
             if (a == 0 and l < 1 or a == 1 and l > 0) and (b == 0 and lp < 1 or b == 1 and lp > 0)]
    judged = err[slots]
    assert (judged >= 0).all(), judged            # every cell of every component judged
    others = np.delete(err, slots, axis=0)
    assert (others < 0).all()
    print("held-out relative RMS error per cell: median %.2e, max %.2e, cells within 1e-5: %d of %d"
          % (np.median(judged), judged.max(), ok.sum(), judged.size))
    src, q, tgt = to_dev(torch, w)
    a = plain.direct(src, q, tgt).cpu().numpy()
    b = surr.direct(src, q, tgt).cpu().numpy()
    if ok.sum() == 0:
        assert np.array_equal(a, b)
    else:
        assert rel_l2(b, a) < 1e-5


def test_surrogate_loose_bound_error_within_bound():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer(n=400)
    plain, surr = _solvers(pkg, w)
    bound = 3e-2
    err, ok = surr.train_surrogate(**BOX, samples=131072, steps=1500, bound=bound, seed=2)
    assert ok.sum() > 0
    assert (err[ok] <= bound).all()
    src, q, tgt = to_dev(torch, w)
    a = plain.direct(src, q, tgt).cpu().numpy()
    b = surr.direct(src, q, tgt).cpu().numpy()
    e = rel_l2(b, a)
    print("loose bound %.0e: %d cells used, direct-sum error vs quadrature %.2e" % (bound, ok.sum(), e))
    assert 0 < e < bound
    # the FMM near field takes the same path: results stay within the bound
    fa = plain.eval(src, q, tgt).cpu().numpy()
    fb = surr.eval(src, q, tgt).cpu().numpy()
    assert rel_l2(fb, fa) < bound
    # re-judged against a bound no cell meets: the quadrature everywhere again
    _, ok2 = surr.surrogate_set_bound(1e-9)
    assert ok2.sum() == 0
    assert np.array_equal(surr.direct(src, q, tgt).cpu().numpy(), a)

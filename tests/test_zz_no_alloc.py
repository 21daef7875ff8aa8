"""The allocation-free direct sum (for callers that cannot allocate device
memory, e.g. inside another framework's memory manager or an allocation-free
solver loop) gives the same potentials as the regular direct sum, call after
call, although its scratch is one fixed array that keeps the previous call's
contents.  Named to be collected last."""
import numpy as np
import pytest

from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_matches_direct_two_calls():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.three_layer(n=330, leaf=16, p=4)
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    ref = s.direct(src, q, tgt).cpu().numpy()
    out = torch.empty(len(w["tgt"]), dtype=torch.complex128, device=tgt.device)
    for _ in range(2):
        out.fill_(complex(np.nan, np.nan))
        got = s.direct_noalloc(src, q, tgt, out=out).cpu().numpy()
        assert rel_l2(got, ref) < 1e-12, rel_l2(got, ref)
    # a different problem right after: stale scratch contents must not leak
    w2 = workloads.two_layer(n=200, seed=5)
    s2 = pkg.LayeredFMM(w2["k"], w2["d"], w2["eps"], p=4, leaf=16)
    src2, q2, tgt2 = to_dev(torch, w2)
    ref2 = s2.direct(src2, q2, tgt2).cpu().numpy()
    for _ in range(2):
        got2 = s2.direct_noalloc(src2, q2, tgt2).cpu().numpy()
        assert rel_l2(got2, ref2) < 1e-12


def test_noalloc_rejects_table_beyond_scratch():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    # eight layers: 64 * 8^2 * Q bytes exceed the fixed scratch once the rule
    # grows past 1024 nodes, which points 0.004 from an interface force
    d = [0.0, -0.5, -1.0, -1.5, -2.0, -2.5, -3.0]
    s = pkg.LayeredFMM([1.0 + 0.1 * i for i in range(8)], d, p=3, leaf=8)
    dev = torch.device("cuda:0")
    pts = torch.tensor([[0.0, 0.0, 0.002], [0.1, 0.0, -0.002], [0.2, 0.1, 0.3]], dtype=torch.float64, device=dev)
    q = torch.ones(3, dtype=torch.complex128, device=dev)
    s.direct(pts, q, pts)
    with pytest.raises(pkg.FmmError) as ei:
        s.direct_noalloc(pts, q, pts)
    assert ei.value.code == -7 and "fixed scratch" in str(ei.value)

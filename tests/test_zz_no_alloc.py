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


def test_noalloc_uses_the_trained_surrogate_like_direct():
    # with FMM_SURROGATE and a trained network, both entry points take the
    # reaction components from the surrogate in the same cells
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer(n=200, seed=6)
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=4, leaf=16, surrogate=True)
    s.train_surrogate(rho_max=2.9, z_min=0.09, z_max=1.11, samples=65536, steps=300, bound=1e-5)
    _, ok = s.surrogate_set_bound(10.0)          # every judged cell uses the network
    assert ok.sum() > 0
    plain = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=4, leaf=16)
    src, q, tgt = to_dev(torch, w)
    quad = plain.direct(src, q, tgt).cpu().numpy()
    ref = s.direct(src, q, tgt).cpu().numpy()
    assert rel_l2(ref, quad) > 1e-12              # the surrogate did run
    for _ in range(2):
        got = s.direct_noalloc(src, q, tgt).cpu().numpy()
        assert rel_l2(got, ref) < 1e-12, rel_l2(got, ref)


def test_noalloc_fresh_handle_allocates_nothing():
    # first call on a handle that never ran anything else: device memory in
    # use and torch's reserved pool are the same before and after the call
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    rng = np.random.default_rng(12)
    pts = rng.uniform(-1, 1, (240, 3))
    pts[:120, 2] = rng.uniform(0.2, 1.2, 120)        # 0.2 from the interface: the rule
    pts[120:, 2] = rng.uniform(-1.2, -0.2, 120)      # built at create reaches far enough
    dev = torch.device("cuda:0")
    src = torch.tensor(pts, device=dev)
    q = torch.tensor(rng.uniform(0, 1, 240) + 0j, device=dev)
    warm = pkg.LayeredFMM([1.0, 1.5], [0.0], [1.0, 2.0], p=4, leaf=16)
    warm.direct_noalloc(src, q, src)                 # the library's code is loaded on the device
    fresh = pkg.LayeredFMM([1.0, 1.5], [0.0], [1.0, 2.0], p=4, leaf=16)
    out = torch.empty(240, dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_reserved(dev)
    fresh.direct_noalloc(src, q, src, out=out)
    torch.cuda.synchronize()
    free1, reserved1 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_reserved(dev)
    assert free1 == free0 and reserved1 == reserved0, (free0 - free1, reserved1 - reserved0)
    ref = fresh.direct(src, q, src).cpu().numpy()
    assert rel_l2(out.cpu().numpy(), ref) < 1e-12


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

"""GPU results at the workloads' stated sizes vs stored oracle values
(tests/golden/oracle_values.npz, written by tests/golden/make_golden.py from
the oracle alone)."""
import os

import numpy as np
import pytest

from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu
GOLD = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_values.npz"))


def test_three_layer_full_size_fmm_matches_oracle_fmm():
    # three-layer N = 32,768, p = 8, leaf 64 (the bench workload, same launch
    # configuration): GPU FMM vs the oracle FMM at 24 sampled targets.
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.three_layer()
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    got = s.eval(src, q, tgt).cpu().numpy()
    sel = GOLD["three_layer_sel"]
    err_fmm = rel_l2(got[sel], GOLD["three_layer_fmm"])
    err_dir = rel_l2(got[sel], GOLD["three_layer_direct"])
    print(f"three-layer N=32768: rel L2 vs oracle FMM {err_fmm:.2e}, vs direct sum {err_dir:.2e}")
    assert err_fmm < 1e-9, err_fmm            # parity: same method, FP64
    assert err_dir < 1e-4, err_dir            # truncation of the method at p = 8
    # the GPU direct sum agrees with the oracle direct sum at the same targets
    d = s.direct(src, q, tgt[torch.as_tensor(sel, device=tgt.device)]).cpu().numpy()
    assert rel_l2(d, GOLD["three_layer_direct"]) < 1e-10


def test_two_layer_full_size_all_targets_vs_direct():
    # two-layer N = 1000, p = 5, leaf 40: all potentials vs the oracle direct sum
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer()
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    got = s.eval(src, q, tgt).cpu().numpy()
    ref = GOLD["two_layer_direct"]
    err = rel_l2(got, ref)
    print(f"two-layer N=1000 p=5: rel L2 vs direct sum {err:.2e}")
    assert err < 1e-4, err
    d = s.direct(src, q, tgt).cpu().numpy()
    assert rel_l2(d, ref) < 1e-10


def test_accuracy_improves_with_p():
    # the FMM error against the direct sum decays geometrically in p (Sec. 3.3)
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer()
    src, q, tgt = to_dev(torch, w)
    ref = GOLD["two_layer_direct"]
    errs = []
    for p in (4, 6, 8, 10, 12):
        s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=p, leaf=w["leaf"])
        errs.append(rel_l2(s.eval(src, q, tgt).cpu().numpy(), ref))
        s.close()
    print("two-layer errors vs p:", ["%.2e" % e for e in errs])
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs
    # orders whose operators no longer fit in shared memory whole run as
    # row blocks (p = 10..12) or streamed contraction chunks (p >= 13)
    for p in (13, 16):
        s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=p, leaf=w["leaf"])
        e = rel_l2(s.eval(src, q, tgt).cpu().numpy(), ref)
        s.close()
        print("p=%d: %.2e" % (p, e))
        assert e < 1e-7, (p, e)

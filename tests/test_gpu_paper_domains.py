"""The paper's shaped test (three irregular domains, one per layer, N = 912 +
640 + 1296): the FMM error against the direct sum decays with the expansion
order (Sec. 4, accuracy study), and the GPU direct sum agrees with the oracle
direct sum on sampled targets."""
import numpy as np
import pytest

from oracle import green
from oracle.media import Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def test_paper_domains_accuracy_vs_p():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.paper_domains()
    src, q, tgt = to_dev(torch, w)
    ref = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=4, leaf=w["leaf"]).direct(src, q, tgt).cpu().numpy()
    sel = workloads.sample_targets(len(w["tgt"]), 6, seed=5)
    orc = green.direct_sum(Medium(w["k"], w["d"], w["eps"]), w["src"], w["q"], w["tgt"][sel])
    assert rel_l2(ref[sel], orc) < 1e-10
    errs = []
    for p in (4, 6, 8, 10):
        s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=p, leaf=w["leaf"])
        errs.append(rel_l2(s.eval(src, q, tgt).cpu().numpy(), ref))
        m = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=p, leaf=w["leaf"], mixed=True)
        assert rel_l2(m.eval(src, q, tgt).cpu().numpy(), ref) < errs[-1] + 1e-5
    print("paper domains N=2848: FMM error vs p=4,6,8,10:", ["%.2e" % e for e in errs])
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6

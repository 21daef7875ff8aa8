"""Mixed-precision form: M2L translations on the tensor cores (FP16 hi/lo
operands with power-of-two scaling, FP32 accumulation).  Its potentials must
stay within 1e-5 (relative L2) of the FP64 oracle FMM and of the FP64 GPU
path on the same trees."""
import os

import numpy as np
import pytest

from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu

GOLD = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_values.npz"))


def _pair(torch, w, p=None):
    import paper_1902_05132_gb300 as pkg
    p = w["p"] if p is None else p
    src, q, tgt = to_dev(torch, w)
    plain = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=p, leaf=w["leaf"])
    mixed = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=p, leaf=w["leaf"], mixed=True)
    a = plain.eval(src, q, tgt).cpu().numpy()
    b = mixed.eval(src, q, tgt).cpu().numpy()
    b2 = mixed.eval(src, q, tgt).cpu().numpy()
    return a, b, b2, mixed


def test_mixed_two_layer_matches_fp64():
    torch = cuda_or_skip()
    w = workloads.two_layer()
    a, b, b2, _ = _pair(torch, w)
    err = rel_l2(b, a)
    print("two-layer N=1000 p=5: mixed vs FP64 path %.2e" % err)
    assert err < 1e-5
    assert np.array_equal(b, b2)        # cached operators, deterministic


def test_mixed_three_layer_matches_oracle():
    torch = cuda_or_skip()
    w = workloads.three_layer()
    a, b, _, s = _pair(torch, w)
    sel = GOLD["three_layer_sel"]
    e_fp64 = rel_l2(b, a)
    e_orc = rel_l2(b[sel], GOLD["three_layer_fmm"])
    st = s.stats()
    print("three-layer N=32768 p=8: mixed vs FP64 path %.2e, vs oracle FMM %.2e, M2L products %.3f ms"
          % (e_fp64, e_orc, st["gpu_ms_m2l_gemm"]))
    assert e_fp64 < 1e-5 and e_orc < 1e-5


@pytest.mark.parametrize("p", [10, 12])
def test_mixed_large_orders(p):
    # p = 12: operators of 169 rows run as two row blocks (128 + 41)
    torch = cuda_or_skip()
    w = workloads.two_layer(n=600, seed=3)
    a, b, _, _ = _pair(torch, w, p=p)
    err = rel_l2(b, a)
    print("two-layer N=600 p=%d: mixed vs FP64 path %.2e" % (p, err))
    assert err < 1e-5


def test_tensor_core_wait_expiry_is_reported():
    # A test-only flag makes every pipeline stage of the tensor-core M2L wait
    # for bytes that never come: its bounded waits run out, the kernel frees
    # its tensor memory and returns, and the evaluation reports a timeout.
    # The context stays usable: a normal evaluation right after is correct.
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer(n=300, leaf=20, p=5)
    src, q, tgt = to_dev(torch, w)
    stalled = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], mixed=True,
                             extra_flags=pkg.FMM_TEST_STALL_TC)
    with pytest.raises(pkg.FmmError) as ei:
        stalled.eval(src, q, tgt)
    assert ei.value.code == -6 and "bounded wait" in str(ei.value)
    stalled.close()
    a, b, _, _ = _pair(torch, w)
    assert rel_l2(b, a) < 1e-5

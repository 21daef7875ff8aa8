"""GPU FMM vs the oracle FMM (same tree, same p) and vs the direct sum."""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import green
from oracle.media import Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _run(w, sel):
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    got = s.eval(src, q, tgt).cpu().numpy()
    med = Medium(w["k"], w["d"], w["eps"])
    ref = ofmm.FMM(med, w["p"], w["leaf"]).evaluate(w["src"], w["q"], w["tgt"], targets=sel)
    return got, ref, s


def test_fmm_two_layer_small_matches_oracle_fmm():
    w = workloads.two_layer(n=400, leaf=20, p=5)
    sel = np.arange(400)
    got, ref, _ = _run(w, sel)
    assert rel_l2(got[sel], ref) < 1e-10, rel_l2(got[sel], ref)


def test_fmm_three_layer_small_matches_oracle_fmm():
    w = workloads.three_layer(n=900, leaf=16, p=6)
    sel = workloads.sample_targets(900, 90)
    got, ref, _ = _run(w, sel)
    assert rel_l2(got[sel], ref) < 1e-10, rel_l2(got[sel], ref)


def test_fmm_two_layer_config_all_targets_vs_direct():
    # two-layer workload at its stated size: all N potentials vs the direct sum
    w = workloads.two_layer()
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    got = s.eval(src, q, tgt).cpu().numpy()
    dgpu = s.direct(src, q, tgt).cpu().numpy()
    med = Medium(w["k"], w["d"], w["eps"])
    sel = workloads.sample_targets(len(w["src"]), 60)
    ref = green.direct_sum(med, w["src"], w["q"], w["tgt"], targets=sel)
    assert rel_l2(dgpu[sel], ref) < 1e-10
    # p = 5: truncation error of the method (Sec. 3.3), not a parity bound
    assert rel_l2(got, dgpu) < 1e-4, rel_l2(got, dgpu)


def test_m2l_autotuner_choice_and_identical_results():
    # the first evaluation times every candidate tile of the rotation-form
    # M2L (p >= 5) and keeps the fastest; each candidate computes the same
    # columns, so every later evaluation is bit-identical to the first
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.three_layer(n=4000, leaf=32, p=8)
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    a = s.eval(src, q, tgt).cpu().numpy()
    st = s.stats()
    assert st["tune_zrot_candidates"] >= 2
    assert st["tune_zrot_kc"] >= 1 and st["tune_zrot_threads"] in (128, 256)
    assert 0 < st["tune_zrot_ms"] <= st["tune_zrot_rule_ms"]
    b = s.eval(src, q, tgt).cpu().numpy()
    assert np.array_equal(a, b)
    s.close()

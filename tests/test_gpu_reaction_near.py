"""The reaction near field inside the FMM (Algorithm 1, last step: direct
interactions of the reaction components, eq. generalcomponentsimag) against
the oracle FMM.  With count-only reaction trees (FMM_TREE_COUNTS) target
leaves next to an interface meet image leaves in their U, W and X lists;
both sides then evaluate those pairs by Sommerfeld quadrature on their own
contours and rules."""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle.media import Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _clustered(n=900, leaf=16, p=6, n_cluster=150):
    # three-layer workload with a cluster 0.1-0.2 above the top interface:
    # uneven refinement there gives the reaction trees W and X lists
    w = workloads.three_layer(n=n, leaf=leaf, p=p)
    rng = np.random.default_rng(9)
    w["src"][:n_cluster] = np.array([0.3, -0.2, 0.15]) + 0.03 * rng.standard_normal((n_cluster, 3))
    w["src"][:n_cluster, 2] = np.abs(w["src"][:n_cluster, 2] - 0.15) + 0.1
    w["tgt"] = w["src"].copy()
    return w


def test_reaction_near_field_fmm_matches_oracle_fmm():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = _clustered()
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True)
    src, q, tgt = to_dev(torch, w)
    got = s.eval(src, q, tgt).cpu().numpy()
    st = s.stats()
    assert st["n_reac_pairs"] > 0, st["n_reac_pairs"]
    reac = [g for g in s.trees() if g["kind"] == 1]
    n_wx = sum(len(g["lists"]["W"]) + len(g["lists"]["X"]) for g in reac)
    assert n_wx > 0
    sel = workloads.sample_targets(len(w["tgt"]), 300, seed=4)
    med = Medium(w["k"], w["d"], w["eps"])
    ref = ofmm.FMM(med, w["p"], w["leaf"], split_interface=False).evaluate(w["src"], w["q"], w["tgt"], targets=sel)
    err = rel_l2(got[sel], ref)
    emax = float(np.max(np.abs(got[sel] - ref)) / np.max(np.abs(ref)))
    print(f"count-only trees: {st['n_reac_pairs']} reaction near pairs, {n_wx} reaction W/X entries; "
          f"rel L2 vs oracle FMM {err:.2e}, max {emax:.2e}")
    assert err < 1e-9 and emax < 1e-9, (err, emax)
    # same sum as the default tree (reaction through M2L only): the two FMMs
    # differ by their truncation error alone
    s0 = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    got0 = s0.eval(src, q, tgt).cpu().numpy()
    assert s0.stats()["n_reac_pairs"] == 0
    d = s.direct(src, q, tgt).cpu().numpy()
    e_c, e_0 = rel_l2(got, d), rel_l2(got0, d)
    print(f"vs direct sum: count-only {e_c:.2e}, interface rule {e_0:.2e}")
    assert e_c < 1e-4 and e_0 < 1e-4
    # mixed form on the count-only trees (reaction near field stays FP64)
    m = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True, mixed=True)
    gm = m.eval(src, q, tgt).cpu().numpy()
    assert m.stats()["n_reac_pairs"] == st["n_reac_pairs"]
    em = rel_l2(gm[sel], ref)
    print(f"mixed form, count-only trees: rel L2 vs oracle FMM {em:.2e}")
    assert em < 1e-5, em


def test_surrogate_in_the_fmm_near_field():
    # the same count-only FMM with the learned surrogate (FMM_SURROGATE):
    # reaction near-field pairs whose cell passed the held-out check at 1e-5
    # take the network, the others the quadrature.  Checked: the surrogate
    # serves pairs, the potentials stay within the bound of the oracle FMM,
    # and the reaction near field takes less device time than by quadrature.
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = _clustered()
    src, q, tgt = to_dev(torch, w)
    plain = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True)
    surr = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True, surrogate=True)
    got_q = plain.eval(src, q, tgt).cpu().numpy()
    plain.eval(src, q, tgt)
    st_q = plain.stats()
    # train on the box of (rho, zt, zs) this geometry's near field needs
    box = dict(rho_max=1.001 * st_q["reac_near_rho_max"], z_min=0.999 * st_q["reac_near_z_min"],
               z_max=1.001 * st_q["reac_near_z_max"])
    assert 0 < box["z_min"] < box["z_max"] and box["rho_max"] > 0, box
    err, ok = surr.train_surrogate(**box, samples=262144, steps=4000, bound=1e-5, seed=3)
    judged = err[err >= 0]
    got_s = surr.eval(src, q, tgt).cpu().numpy()
    surr.eval(src, q, tgt)
    st_s = surr.stats()
    frac = st_s["n_reac_surr_pairs"] / st_s["n_reac_pairs"]
    sel = workloads.sample_targets(len(w["tgt"]), 300, seed=4)
    med = Medium(w["k"], w["d"], w["eps"])
    ref = ofmm.FMM(med, w["p"], w["leaf"], split_interface=False).evaluate(w["src"], w["q"], w["tgt"], targets=sel)
    e_s, e_q = rel_l2(got_s[sel], ref), rel_l2(got_q[sel], ref)
    print(f"near-field box rho <= {box['rho_max']:.3f}, z in [{box['z_min']:.3f}, {box['z_max']:.3f}]; "
          f"held-out error per cell: median {np.median(judged):.2e}, max {judged.max():.2e}, "
          f"{int(ok.sum())} of {judged.size} cells within 1e-5; surrogate pairs {st_s['n_reac_surr_pairs']} of "
          f"{st_s['n_reac_pairs']} ({100 * frac:.1f} %); reaction near field {st_s['gpu_ms_near_reac']:.3f} ms "
          f"(quadrature {st_q['gpu_ms_near_reac']:.3f} ms); evaluation {st_s['gpu_ms_total']:.2f} ms "
          f"(quadrature {st_q['gpu_ms_total']:.2f} ms); rel L2 vs oracle FMM {e_s:.2e} (quadrature {e_q:.2e})")
    assert st_s["n_reac_surr_pairs"] > 0
    assert e_s < 1e-5, e_s
    if frac > 0.9:
        assert st_s["gpu_ms_near_reac"] < st_q["gpu_ms_near_reac"]

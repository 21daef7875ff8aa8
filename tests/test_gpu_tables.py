"""Tabulated reaction M2L integrals (FMM_TABLES; Sec. 3.5, eqs. M2Ltable,
metoletableform) on the GPU against the oracle.

  * single operators interpolated by the library against the oracle's
    interpolated tables (oracle/tables.py, its own quadrature of the same
    integrals) and against the oracle's direct radial operator of eq.
    me2lesimplified, errors weighted by the size of the expansion
    coefficients each entry multiplies;
  * whole FMM evaluations with tables against the oracle FMM (quadrature
    operators) at the same tree and p, and a second geometry whose operators
    all come from the tables (no quadrature node is summed for them).
"""
import math

import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import tables as otab
from oracle.media import DOWN, UP, Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu

MED_ARGS = ([0.8, 1.2, 1.6], [0.0, -1.2], [1.0, 2.0, 3.0])


@pytest.fixture(scope="module")
def solver8():
    cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    s = pkg.LayeredFMM(*MED_ARGS, p=8, leaf=64, tables=True)
    yield s
    s.close()


def _direct_T(med, comp, p, w, jt, js, r):
    l, lp, a, b = comp
    rh, zt, zs = otab.ray(jt, js, r)
    d = med.d[l] if a == UP else med.d[l - 1]
    zt_abs = d + zt * w if a == UP else d - zt * w
    zs_abs = d - zs * w if a == UP else d + zs * w
    rule = ofmm.t_rule(med, (zt + zs) * w, max(rh * w, 1e-3), p)
    return ofmm.reaction_T_radial(med, l, lp, a, b, p, rh * w, zt_abs, zs_abs, rule)


@pytest.mark.parametrize("comp,u,jt,js,r", [
    ((0, 1, UP, DOWN), -3.6, 0, 1, 3),     # whole-octave panel
    ((2, 1, DOWN, DOWN), -1.7, 1, 0, 9),   # half-octave panel
    ((1, 1, DOWN, UP), 0.6, 0, 0, 9),      # quarter-octave panel, widest class
    ((0, 0, UP, UP), 1.3, 1, 1, 4),
    ((1, 2, UP, DOWN), -0.4, 1, 1, 0),     # rho = 0
])
def test_table_operator_matches_oracle(solver8, comp, u, jt, js, r):
    med = Medium(*MED_ARGS)
    p = 8
    w = 2.0 ** u / max(MED_ARGS[0])
    got = solver8.table_operator(*comp, w, jt, js, r)
    want_tab = otab.table_T(med, comp, p, w, jt, js, r)
    want_dir = _direct_T(med, comp, p, w, jt, js, r)
    W = otab.degree_weights(med, comp, p, w)
    e_tab = np.abs((got - want_tab) * W).max() / np.abs(want_tab * W).max()
    e_dir = np.abs((got - want_dir) * W).max() / np.abs(want_dir * W).max()
    assert e_tab < 1e-11, e_tab
    assert e_dir < 1e-11, e_dir


def test_table_operator_rejects_outside_range(solver8):
    import paper_1902_05132_gb300 as pkg
    with pytest.raises(pkg.FmmError):
        solver8.table_operator(0, 1, UP, DOWN, 2.0 ** 2 / 1.6, 0, 0, 4)
    with pytest.raises(pkg.FmmError):
        solver8.table_operator(0, 0, DOWN, UP, 0.1, 0, 0, 4)       # layer 0 has no arrow down


def _fmm(torch, w, tables, scale=1.0):
    import paper_1902_05132_gb300 as pkg
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tables=tables)
    wd = dict(w)
    src, q, tgt = to_dev(torch, wd)
    src = src * scale
    tgt = tgt * scale
    return s, s.eval(src, q, tgt).cpu().numpy()


def test_fmm_with_tables_matches_oracle_fmm():
    torch = cuda_or_skip()
    w = workloads.three_layer(n=900, leaf=16, p=6)
    sel = workloads.sample_targets(900, 90)
    s, got = _fmm(torch, w, tables=True)
    st = s.stats()
    assert st["n_reac_table_classes"] > 0
    assert st["n_reac_T_nodes"] == 0          # every reaction class came from the tables
    med = Medium(w["k"], w["d"], w["eps"])
    ref = ofmm.FMM(med, w["p"], w["leaf"]).evaluate(w["src"], w["q"], w["tgt"], targets=sel)
    assert rel_l2(got[sel], ref) < 1e-10, rel_l2(got[sel], ref)
    s.close()


def test_new_geometry_uses_tables_and_agrees_with_quadrature():
    torch = cuda_or_skip()
    w = workloads.three_layer(n=6000, leaf=32, p=8)
    for scale in (1.0, 0.83):
        # x, y and z scaled about the origin: new box widths; the interface
        # at z = 0 stays, the one at -1.2 moves, so scale the medium too
        ws = dict(w)
        ws["d"] = [d * scale for d in w["d"]]
        sq, gq = _fmm(torch, ws, tables=False, scale=scale)
        stq = sq.stats()
        sq.close()
        st_, gt = _fmm(torch, ws, tables=True, scale=scale)
        stt = st_.stats()
        assert stt["n_reac_table_classes"] == stq["n_reac_classes"] > 0
        assert stt["n_reac_T_nodes"] == 0
        assert rel_l2(gt, gq) < 1e-11, rel_l2(gt, gq)
        st_.close()


def test_tables_limit_on_order():
    cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    with pytest.raises(pkg.FmmError):
        pkg.LayeredFMM(*MED_ARGS, p=13, leaf=64, tables=True)


def test_reaction_near_field_from_table_matches_oracle_fmm():
    # count-only trees: target leaves next to an interface meet image leaves;
    # their pairs take the kernel from the near-field table
    from tests.test_gpu_reaction_near import _clustered
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = _clustered()
    src, q, tgt = to_dev(torch, w)
    st_ = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True, tables=True)
    got = st_.eval(src, q, tgt).cpu().numpy()
    st = st_.stats()
    assert st["n_reac_pairs"] > 0
    assert st["n_reac_table_pairs"] > 0.9 * st["n_reac_pairs"], (st["n_reac_table_pairs"], st["n_reac_pairs"])
    sq = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"], tree_counts=True)
    gq = sq.eval(src, q, tgt).cpu().numpy()
    assert sq.stats()["n_reac_table_pairs"] == 0
    assert rel_l2(got, gq) < 1e-10, rel_l2(got, gq)
    sel = workloads.sample_targets(len(w["tgt"]), 150, seed=4)
    med = Medium(w["k"], w["d"], w["eps"])
    ref = ofmm.FMM(med, w["p"], w["leaf"], split_interface=False).evaluate(w["src"], w["q"], w["tgt"], targets=sel)
    err = rel_l2(got[sel], ref)
    emax = float(np.max(np.abs(got[sel] - ref)) / np.max(np.abs(ref)))
    assert err < 1e-9 and emax < 1e-9, (err, emax)
    st_.close()
    sq.close()

"""GPU octrees and interaction lists are bit-identical to the oracle's."""
import numpy as np
import pytest

from oracle import fmm as ofmm
from oracle import green
from oracle.media import Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


def _oracle_trees(w, split=True):
    med = Medium(w["k"], w["d"], w["eps"])
    src, tgt = w["src"], w["tgt"]
    ls, lt = med.layer_of(src[:, 2]), med.layer_of(tgt[:, 2])
    ns_l = [int(np.sum(ls == l)) for l in range(med.L + 1)]
    nt_l = [int(np.sum(lt == l)) for l in range(med.L + 1)]
    out = []
    for comp in ofmm.components(med, ns_l, nt_l):
        sl = comp.l if comp.kind == "free" else comp.lp
        spos = src[ls == sl].copy()
        if comp.kind == "reac":
            spos[:, 2] = green.image_z(med, comp.l, comp.lp, comp.a, comp.b, spos[:, 2])
        tree = ofmm.component_tree(med, comp, spos, tgt[lt == comp.l], w["leaf"], split_interface=split)
        out.append((comp, tree, ofmm.build_lists(tree)))
    return out


def _check(w, tree_counts=False):
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=3, leaf=w["leaf"], tree_counts=tree_counts)
    src, q, tgt = to_dev(torch, w)
    s.eval(src, q, tgt)
    gpu = s.trees()
    ora = _oracle_trees(w, split=not tree_counts)
    assert len(gpu) == len(ora)
    for g, (comp, tree, (U, V, W, X)) in zip(gpu, ora):
        kind = 0 if comp.kind == "free" else 1
        assert (g["kind"], g["l"]) == (kind, comp.l)
        if kind:
            assert (g["lp"], g["a"], g["b"]) == (comp.lp, comp.a, comp.b)
        assert np.array_equal(g["root"][:3], tree.c) and g["root"][3] == tree.h, (g["root"], tree.c, tree.h)
        assert np.array_equal(g["level"], tree.level)
        assert np.array_equal(g["prefix"], tree.prefix)
        assert np.array_equal(g["src_begin"], tree.src_begin) and np.array_equal(g["src_end"], tree.src_end)
        assert np.array_equal(g["tgt_begin"], tree.tgt_begin) and np.array_equal(g["tgt_end"], tree.tgt_end)
        assert np.array_equal(g["parent"], tree.parent)
        assert np.array_equal(g["sperm"], tree.sperm) and np.array_equal(g["tperm"], tree.tperm)
        for name, lst in zip("VUWX", (V, U, W, X)):
            assert g["lists"][name] == {b: list(v) for b, v in lst.items()}, name
    return gpu


def test_trees_two_layer():
    _check(workloads.two_layer(n=1000, leaf=40))


def test_trees_three_layer_adaptive():
    w = workloads.three_layer(n=3000, leaf=12)
    # a cluster forces uneven refinement (coarse leaves next to fine ones)
    rng = np.random.default_rng(9)
    w["src"][:400] = np.array([0.3, -0.2, 0.15]) + 0.03 * rng.standard_normal((400, 3))
    w["src"][:400, 2] = np.abs(w["src"][:400, 2]) + 0.1
    w["tgt"] = w["src"].copy()
    _check(w)


def test_trees_three_layer_count_only():
    # count-only refinement of the reaction trees (FMM_TREE_COUNTS): still
    # bit-identical, and the reaction trees now carry U, W and X lists
    w = workloads.three_layer(n=3000, leaf=12)
    rng = np.random.default_rng(9)
    w["src"][:400] = np.array([0.3, -0.2, 0.15]) + 0.03 * rng.standard_normal((400, 3))
    w["src"][:400, 2] = np.abs(w["src"][:400, 2] - 0.15) + 0.1
    w["tgt"] = w["src"].copy()
    gpu = _check(w, tree_counts=True)
    reac = [g for g in gpu if g["kind"] == 1]
    assert sum(len(g["lists"]["U"]) for g in reac) > 0
    assert sum(len(g["lists"]["W"]) + len(g["lists"]["X"]) for g in reac) > 0

"""One problem's components split into ranges (the multi-GPU protocol of
paper_1902_05132_gb300.distributed, run here rank after rank on one GPU):
each range is evaluated by its own handle, the running sum is passed along
and every later range adds its components in order; the total is
bit-identical to one evaluation of all components."""
import numpy as np
import pytest

from paper_1902_05132_gb300 import distributed, workloads
from tests.gpu_common import cuda_or_skip, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_ranks", [2, 3, 5])
def test_component_ranges_chain_to_the_full_result(n_ranks):
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.three_layer(n=3000, leaf=32, p=6)
    src, q, tgt = to_dev(torch, w)
    full = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    ref = full.eval(src, q, tgt)
    work = full.component_work()
    assert len(work) == full.stats()["n_components"] == 19 and (work > 0).all()
    ranges = distributed.partition(work, n_ranks)
    outs, handles = [], []
    for first, count in ranges:
        h = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
        h.set_components(first, count)
        outs.append(h.eval(src, q, tgt))
        assert h.stats()["n_components"] == count
        handles.append(h)
    running = outs[0].clone()
    for h in handles[1:]:
        h.add_components(running)
    assert torch.equal(running, ref)
    # the plain sum of the partial results agrees to rounding
    tot = sum(outs[1:], outs[0].clone())
    assert float(torch.linalg.vector_norm(tot - ref) / torch.linalg.vector_norm(ref)) < 1e-14


def test_empty_component_range_gives_zero():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = workloads.two_layer(n=200, leaf=16, p=4)
    src, q, tgt = to_dev(torch, w)
    h = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    h.set_components(50, 3)
    out = h.eval(src, q, tgt)
    assert h.stats()["n_components"] == 0 and not torch.any(out != 0)
    h.set_components(0, -1)
    full = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    assert torch.equal(h.eval(src, q, tgt), full.eval(src, q, tgt))

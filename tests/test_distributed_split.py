"""The component split over ranks (paper_1902_05132_gb300.distributed) on
CPU: the contiguous partition is optimal, and the chain sum over gloo ranks
reproduces the one-process potentials bit for bit.  The component potentials
come from the oracle FMM (one FMM per component, summed in component order,
as in eq. totalinteraction); the GPU library follows the same protocol
(tests/test_gpu_components.py)."""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_1902_05132_gb300 import distributed, workloads

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _brute(work, k):
    n = len(work)
    best = None
    for cuts in itertools.combinations_with_replacement(range(n + 1), k - 1):
        b = (0,) + cuts + (n,)
        load = max(sum(work[b[r]:b[r + 1]]) for r in range(k))
        if best is None or load < best:
            best = load
    return best


def test_partition_is_contiguous_and_optimal():
    rng = np.random.default_rng(0)
    for n, k in ((6, 2), (7, 3), (19, 4), (5, 8), (1, 3)):
        work = list(rng.uniform(0.1, 10.0, n))
        parts = distributed.partition(work, k)
        assert len(parts) == k
        pos = 0
        for first, count in parts:
            assert first == pos and count >= 0
            pos += count
        assert pos == n
        load = max(sum(work[f:f + c]) for f, c in parts)
        if n <= 8:
            assert load == pytest.approx(_brute(work, k))


def _oracle_components(w, first=0, count=None):
    """Potentials of components [first, first + count) of the oracle FMM, in
    component order (all by default)."""
    from oracle import fmm as ofmm
    from oracle.green import image_z
    from oracle.media import Medium
    med = Medium(w["k"], w["d"], w["eps"])
    src, q, tgt = w["src"], w["q"], w["tgt"]
    ls, lt = med.layer_of(src[:, 2]), med.layer_of(tgt[:, 2])
    F = ofmm.FMM(med, w["p"], w["leaf"])
    comps = ofmm.components(med, [int(np.sum(ls == l)) for l in range(med.L + 1)],
                            [int(np.sum(lt == l)) for l in range(med.L + 1)])
    out = []
    want = np.ones(len(tgt), bool)
    for comp in comps[first:None if count is None else first + count]:
        js = np.nonzero(ls == (comp.l if comp.kind == "free" else comp.lp))[0]
        it = np.nonzero(lt == comp.l)[0]
        spos = src[js].copy()
        if comp.kind == "reac":
            spos[:, 2] = image_z(med, comp.l, comp.lp, comp.a, comp.b, src[js, 2])
        out.append((it, F._component(comp, spos, q[js], tgt[it], want[it], None)))
    return F, out


def _worker(rank, ws, port, w, ranges, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    first, count = ranges[rank]
    _, comps = _oracle_components(w, first, count)

    def add_own(buf):
        for it, vals in comps:
            idx = torch.as_tensor(it)
            buf[idx] += torch.from_numpy(vals)
    buf = torch.zeros(len(w["tgt"]), dtype=torch.complex128)
    distributed.chain_sum(buf, add_own, rank, ws, dist)
    out[rank] = buf.numpy().copy()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_chain_sum_over_gloo_ranks_is_bit_identical(ws):
    w = workloads.two_layer(n=80, leaf=12, p=3)
    F, comps = _oracle_components(w)
    ref = F.evaluate(w["src"], w["q"], w["tgt"])
    work = [len(it) for it, _ in comps]
    ranges = distributed.partition(work, ws)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, w, ranges, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        assert np.array_equal(res[r], ref), r

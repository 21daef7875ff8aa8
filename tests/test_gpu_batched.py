"""Batched evaluation of independent problems (fmm_layered_eval_batched).

Each problem of a batch is the same computation as a single evaluation with
its handle, so the batched results must equal the separate results bit for
bit; media with up to five layers are checked against the oracle direct sum
through the GPU direct sum."""
import numpy as np
import pytest

from oracle import green
from oracle.media import Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _problems(torch, n_problems, seed):
    import paper_1902_05132_gb300 as pkg
    ws = workloads.batched(n_problems, seed=seed, n_min=300, n_max=3000, p=5, leaf=32)
    solvers = [pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"]) for w in ws]
    return ws, solvers, [to_dev(torch, w) for w in ws]


def test_batched_equals_separate_evaluations():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    ws, solvers, probs = _problems(torch, 6, seed=4)
    assert {len(w["k"]) for w in ws} >= {2, 3}
    sep = [s.eval(*pr).cpu().numpy() for s, pr in zip(solvers, probs)]
    for _ in range(2):                  # cold and cached operators
        got = [o.cpu().numpy() for o in pkg.eval_batched(solvers, probs)]
        for a, b in zip(got, sep):
            assert np.array_equal(a, b)


def test_batched_with_shared_workspaces_equals_separate_evaluations():
    # ten problems over three workspaces: the problems of a workspace run one
    # after the other, groups run concurrently; results bit for bit as alone
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    ws, solvers, probs = _problems(torch, 10, seed=5)
    sep = [s.eval(*pr).cpu().numpy() for s, pr in zip(solvers, probs)]
    for i in range(3, 10):
        solvers[i].share_workspace(solvers[i % 3])
    for _ in range(2):
        got = [o.cpu().numpy() for o in pkg.eval_batched(solvers, probs)]
        for a, b in zip(got, sep):
            assert np.array_equal(a, b)
    # a handle sharing a workspace still evaluates alone, and closing the
    # owner first leaves the workspace to the others
    solvers[0].close()
    alone = solvers[3].eval(*probs[3]).cpu().numpy()
    assert np.array_equal(alone, sep[3])
    for s in solvers[1:]:
        s.close()


def test_batched_many_layers_against_direct_and_oracle():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    ws, solvers, probs = _problems(torch, 12, seed=7)
    got = [o.cpu().numpy() for o in pkg.eval_batched(solvers, probs)]
    layers_seen = set()
    for w, s, pr, g in zip(ws, solvers, probs, got):
        ref = s.direct(*pr).cpu().numpy()
        # p = 5: the truncation error of the expansions (Sec. 3.3)
        assert rel_l2(g, ref) < 5e-4, (w["name"], rel_l2(g, ref))
        L1 = len(w["k"])
        if L1 not in layers_seen:
            layers_seen.add(L1)
            med = Medium(w["k"], w["d"], w["eps"])
            sel = workloads.sample_targets(len(w["tgt"]), 4, seed=L1)
            orc = green.direct_sum(med, w["src"], w["q"], w["tgt"][sel])
            assert rel_l2(ref[sel], orc) < 1e-9, (w["name"], rel_l2(ref[sel], orc))
    assert max(layers_seen) >= 4, layers_seen


def _raw_batched(pkg, handles, args, outs):
    import ctypes
    n = len(handles)
    P = ctypes.c_void_p * n
    L = ctypes.c_long * n
    c = lambda arr: ctypes.cast(arr, ctypes.c_void_p)
    return pkg.lib().fmm_layered_eval_batched(
        n, c(P(*handles)), c(L(*[a[0].shape[0] for a in args])), c(P(*[a[0].data_ptr() for a in args])),
        c(P(*[a[1].data_ptr() for a in args])), c(L(*[a[2].shape[0] for a in args])),
        c(P(*[a[2].data_ptr() for a in args])), c(P(*[o.data_ptr() for o in outs])), None)


def test_batched_errors():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    ws, solvers, probs = _problems(torch, 3, seed=9)
    # a repeated handle is rejected before anything runs
    args = [pkg.LayeredFMM._dev_args(*probs[0])] * 2
    outs = [torch.view_as_real(torch.empty(probs[0][2].shape[0], dtype=torch.complex128, device=probs[0][2].device))
            for _ in range(2)]
    assert _raw_batched(pkg, [solvers[0].h, solvers[0].h], args, outs) == -1
    with pytest.raises(ValueError):
        pkg.eval_batched([solvers[0], solvers[0]], [probs[0], probs[0]])
    # a point exactly on an interface fails its own problem only
    bad = probs[1][0].clone()
    bad[0, 2] = ws[1]["d"][0]
    outs = [torch.full((pr[2].shape[0],), complex(np.nan, np.nan), dtype=torch.complex128, device=pr[2].device)
            for pr in probs]
    with pytest.raises(pkg.FmmError) as ei:
        pkg.eval_batched(solvers, [probs[0], (bad, probs[1][1], bad), probs[2]], outs=outs)
    assert ei.value.code == -2 and "problem 1" in str(ei.value)
    for i in (0, 2):
        assert np.array_equal(outs[i].cpu().numpy(), solvers[i].eval(*probs[i]).cpu().numpy())

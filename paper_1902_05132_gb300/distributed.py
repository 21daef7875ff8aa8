"""One problem's components split over several GPUs (one process per GPU).

The free-space and reaction components of a layered-media problem are
independent FMMs whose potentials are only summed at the end (eq.
totalinteraction; the paper's Sec. 4 notes that they can run in parallel).
Each rank evaluates a contiguous range of the component order
(``LayeredFMM.set_components``); the ranges are chosen from the work
estimate of an all-component evaluation (``LayeredFMM.component_work``) so
that the largest load is as small as possible.  The potentials are then
summed along the ranks in order: rank 0 starts from its own result, every
later rank receives the running sum, adds its components one after the
other (``LayeredFMM.add_components``) and passes it on; the last rank
broadcasts the total.  The additions are the ones a single evaluation of
all components makes, in the same order, so the result is bit-identical to
the one-GPU result.  The exchange is one vector of N complex potentials per
hop (16 N bytes) and one broadcast.

Host logic only: the arithmetic runs in the library's kernels; the
collectives are torch.distributed point-to-point sends and a broadcast (NCCL
between GPUs, gloo on the CPU).
"""
import numpy as np


def partition(work, n_ranks):
    """Contiguous ranges [(first, count)] of the components, one per rank,
    that minimize the largest summed work (exact, by dynamic programming over
    the cut positions; ties go to the earliest cut).  Ranks beyond the number
    of components get empty ranges."""
    w = [float(x) for x in work]
    n = len(w)
    k = max(1, int(n_ranks))
    pre = np.concatenate([[0.0], np.cumsum(w)])
    INF = float("inf")
    # best[j][i]: smallest possible maximum load of the first i components on j ranks
    best = [[INF] * (n + 1) for _ in range(k + 1)]
    cut = [[0] * (n + 1) for _ in range(k + 1)]
    best[0][0] = 0.0
    for j in range(1, k + 1):
        for i in range(n + 1):
            for m in range(i + 1):                 # ranks 1..j-1 take the first m components
                v = max(best[j - 1][m], pre[i] - pre[m])
                if v < best[j][i]:
                    best[j][i] = v
                    cut[j][i] = m
    bounds = [n]
    i = n
    for j in range(k, 0, -1):
        i = cut[j][i]
        bounds.append(i)
    bounds = bounds[::-1]
    return [(bounds[r], bounds[r + 1] - bounds[r]) for r in range(k)]


def chain_sum(buf, add_own, rank, world, dist, own_result=None):
    """Sum the ranks' component potentials in component order.

    buf: complex tensor of the N potentials (device or CPU); add_own(buf)
    adds this rank's components to it in their order.  Rank 0 may pass its
    own evaluation result as ``own_result`` (the sum of its components
    starting from zero, the same additions) instead of adding them again.
    Returns buf holding the total on every rank."""
    import torch
    view = torch.view_as_real(buf)
    if rank == 0:
        if own_result is not None:
            buf.copy_(own_result)
        else:
            buf.zero_()
            add_own(buf)
    else:
        dist.recv(view, src=rank - 1)
        add_own(buf)
    if rank < world - 1:
        dist.send(view, dst=rank + 1)
    dist.broadcast(view, src=world - 1)
    return buf

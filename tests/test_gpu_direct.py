"""GPU all-pairs direct sum vs the oracle direct sum (element by element)."""
import numpy as np
import pytest

from oracle import green
from oracle.media import Medium
from paper_1902_05132_gb300 import workloads
from tests.gpu_common import cuda_or_skip, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker,n", [(workloads.two_layer, 240), (workloads.three_layer, 270)])
def test_direct_matches_oracle(maker, n):
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    w = maker(n=n)
    med = Medium(w["k"], w["d"], w["eps"])
    ref = green.direct_sum(med, w["src"], w["q"], w["tgt"])
    s = pkg.LayeredFMM(w["k"], w["d"], w["eps"], p=w["p"], leaf=w["leaf"])
    src, q, tgt = to_dev(torch, w)
    got = s.direct(src, q, tgt).cpu().numpy()
    err = np.abs(got - ref) / np.max(np.abs(ref))
    assert rel_l2(got, ref) < 1e-10 and err.max() < 1e-10, (rel_l2(got, ref), err.max())


def test_direct_single_layer_is_free_space():
    torch = cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    rng = np.random.default_rng(3)
    src = rng.uniform(-1, 1, (150, 3))
    q = rng.uniform(-1, 1, 150) + 1j * rng.uniform(-1, 1, 150)
    k = 1.7
    s = pkg.LayeredFMM([k], [], p=4, leaf=16)
    dev = torch.device("cuda:0")
    got = s.direct(torch.tensor(src, device=dev), torch.tensor(q, device=dev), torch.tensor(src, device=dev)).cpu().numpy()
    R = np.linalg.norm(src[:, None] - src[None], axis=-1)
    np.fill_diagonal(R, 1.0)
    G = np.exp(1j * k * R) / (4 * np.pi * R)
    np.fill_diagonal(G, 0.0)
    assert rel_l2(got, G @ q) < 1e-13

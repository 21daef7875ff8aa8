"""Helpers shared by the GPU tests (no oracle arithmetic here)."""
import numpy as np
import pytest


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1902_05132_gb300 as pkg
    pkg.lib()          # fails loudly when the library is missing
    return torch


def to_dev(torch, w):
    dev = torch.device("cuda:0")
    return (torch.tensor(w["src"], device=dev), torch.tensor(w["q"], device=dev),
            torch.tensor(w["tgt"], device=dev))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))

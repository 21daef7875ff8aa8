"""The surrogate's training kernels compute the gradient of the loss.

A plain FP64 re-implementation of the network's forward and backward pass
(written here from the definition of the network: 3 -> 64 -> 64 -> 64 -> 2,
GELU, mean squared error over the minibatch) is compared with the gradient
the library's training kernels produce for one fixed minibatch
(fmm_layered_surrogate_grad).  The reference is itself pinned against
central finite differences of its own loss.

Tolerances.  The kernels round every weight and every layer input to BF16
(relative spacing 2^-8, rounding error <= 2^-9) and accumulate in FP32.
  * Against the reference with the same BF16 roundings emulated, the only
    differences are FP32 accumulation (~1e-6 relative) and the rare BF16
    rounding that flips by one unit because the FP32 and FP64 pre-activations
    differ (a handful per minibatch, each moving one activation by 2^-8 and
    the summed gradient by ~1e-5 of its size): rel L2 < 1e-4.
  * Against the exact FP64 gradient (no rounding), the BF16 operand error of
    2^-9 enters every product of the forward and backward chains (a few
    layers deep): rel L2 < 2e-2."""
import numpy as np
import pytest

from tests.gpu_common import cuda_or_skip
from tests.mlp_reference import SHAPES, batch, bf16, loss_and_grad

pytestmark = pytest.mark.gpu


def test_training_kernel_gradient_matches_cpu_backprop():
    cuda_or_skip()
    import paper_1902_05132_gb300 as pkg
    theta, x, y = batch(0)
    g_gpu = pkg.surrogate_grad(theta, x, y).astype(np.float64)
    _, g_bf = loss_and_grad(theta, x.astype(np.float64), y.astype(np.float64), bf16)
    _, g_ex = loss_and_grad(theta, x.astype(np.float64), y.astype(np.float64), lambda a: np.asarray(a, np.float64))
    e_bf = np.linalg.norm(g_gpu - g_bf) / np.linalg.norm(g_bf)
    e_ex = np.linalg.norm(g_gpu - g_ex) / np.linalg.norm(g_ex)
    print(f"training-kernel gradient vs FP64 backprop: {e_bf:.2e} (BF16 roundings emulated), {e_ex:.2e} (exact)")
    assert e_bf < 1e-4, e_bf
    assert e_ex < 2e-2, e_ex
    # every parameter block is checked, not only the large ones
    o = 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        blk = slice(o, o + n)
        eb = np.linalg.norm(g_gpu[blk] - g_bf[blk]) / max(np.linalg.norm(g_bf[blk]), 1e-30)
        assert eb < 1e-3, (name, eb)
        o += n

"""Pin of the FP64 reference backprop of the surrogate network
(tests/mlp_reference.py): its gradient equals central finite differences
of its own loss."""
import numpy as np

from tests.mlp_reference import batch, loss_and_grad


def test_reference_backward_matches_finite_differences():
    # pins the reference itself (CPU only: no rounding, central differences)
    theta, x, y = batch(1)
    theta = theta.astype(np.float64)
    x, y = x[:64].astype(np.float64), y[:64].astype(np.float64)
    def ident(a):
        return np.asarray(a, np.float64)
    _, g = loss_and_grad(theta, x, y, ident)
    rng = np.random.default_rng(3)
    for i in rng.choice(len(theta), 40, replace=False):
        e = np.zeros_like(theta)
        e[i] = 1e-6
        fd = (loss_and_grad(theta + e, x, y, ident)[0] - loss_and_grad(theta - e, x, y, ident)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])



"""Plain FP64 forward and backward pass of the surrogate network
(3 -> 64 -> 64 -> 64 -> 2, GELU, mean squared error over the minibatch),
written from the network's definition for checking the library's training
kernels; optional BF16 rounding of weights and layer inputs emulates theirs.
Test infrastructure: no code of the library is used."""
import math

import numpy as np

H = 64
SHAPES = [("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (2, H)), ("b4", (2,))]


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    assert o == len(theta)
    return out


def bf16(a):
    """Round float32 values to bfloat16 (round to nearest, ties to even)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_d(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def loss_and_grad(theta, x, y, rnd):
    """Loss (1/B) sum |net(x) - y|^2 and its gradient; rnd rounds weights and
    layer inputs (identity for the exact gradient)."""
    p = {k: rnd(v) for k, v in unpack(np.asarray(theta, np.float64)).items()}
    B = len(x)
    a0 = rnd(x)
    h1 = a0 @ p["W1"].T + p["b1"]
    a1 = rnd(gelu(h1))
    h2 = a1 @ p["W2"].T + p["b2"]
    a2 = rnd(gelu(h2))
    h3 = a2 @ p["W3"].T + p["b3"]
    a3 = rnd(gelu(h3))
    out = a3 @ p["W4"].T + p["b4"]
    r = out - y
    loss = float(np.sum(r * r) / B)
    g_out = 2.0 * r / B
    g = {"W4": g_out.T @ a3, "b4": g_out.sum(0)}
    d3 = (g_out @ p["W4"]) * gelu_d(h3)
    g["W3"], g["b3"] = d3.T @ a2, d3.sum(0)
    d2 = (d3 @ p["W3"]) * gelu_d(h2)
    g["W2"], g["b2"] = d2.T @ a1, d2.sum(0)
    d1 = (d2 @ p["W2"]) * gelu_d(h1)
    g["W1"], g["b1"] = d1.T @ a0, d1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SHAPES])


def batch(seed=0):
    rng = np.random.default_rng(seed)
    theta = np.concatenate([rng.uniform(-1, 1, int(np.prod(s))) * (math.sqrt(6.0 / (s[0] + s[1])) if len(s) == 2
                                                                     else 0.05) for _, s in SHAPES])
    x = rng.uniform(-1, 1, (1024, 3))
    # a smooth target of the kind the surrogate fits
    y = np.stack([np.cos(2 * x[:, 0] + x[:, 1]) * np.exp(-0.5 * x[:, 2]), np.sin(x[:, 0] - x[:, 2])], 1)
    return theta.astype(np.float32), x.astype(np.float32), y.astype(np.float32)



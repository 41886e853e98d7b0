"""Float64 reference of the learned schedule network (8 -> 64 -> 64 -> 2,
ReLU, linear outputs) and of its squared-error gradient.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the tests use it to
check the CUDA training and inference kernels.  Weights are taken from a
float32 master vector in the order W1 [64][8], W2 [64][64], W3 [2][64],
b1 [64], b2 [64], b3 [2]; the matrices are rounded to bfloat16 (round to
nearest even) first, as the kernels store them.
"""
from __future__ import annotations

import numpy as np

SIZES = [("W1", (64, 8)), ("W2", (64, 64)), ("W3", (2, 64)), ("b1", (64,)), ("b2", (64,)), ("b3", (2,))]
N_PARAMS = 4866


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(master: np.ndarray, round_weights: bool = True):
    p = {}
    o = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        v = np.asarray(master[o:o + n], dtype=np.float32).reshape(shape)
        p[name] = bf16_round(v) if (round_weights and name.startswith("W")) else v.astype(np.float64)
        o += n
    return p


def forward(master: np.ndarray, x: np.ndarray):
    p = unpack(master)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (x, z1, h1, z2, h2)


def loss_and_grad(master: np.ndarray, x: np.ndarray, t: np.ndarray, n_total: int | None = None):
    """sum_s ||net(x_s) - t_s||^2 / n_total and its gradient (master order)
    with respect to the (rounded) weights and the biases."""
    p = unpack(master)
    out, (x, z1, h1, z2, h2) = forward(master, x)
    n_total = n_total or x.shape[0]
    e = out - np.asarray(t, dtype=np.float64)
    loss = float((e * e).sum() / n_total)
    d_out = 2.0 * e / n_total
    g = {"W3": d_out.T @ h2, "b3": d_out.sum(0)}
    d2 = (d_out @ p["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, flat


def adam_step(master, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), float64."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return master - lr * mh / (np.sqrt(vh) + eps), m, v

"""TEST INFRASTRUCTURE ONLY: plain FP64 restatement of the learned cost model.

Only tests, `__graft_entry__.smoke()` and bench.py's reference leg may use it;
the engine's network (CUDA kernels in the library) shares no code with it.

The network: 8 -> 64 -> 64 -> 64 -> 1, ReLU on the hidden layers, linear
output; loss = mean over the batch of (y - t)^2; Adam with beta1 0.9, beta2
0.999, eps 1e-8 (Kingma & Ba, 2015).  The engine computes with the FP32 master
weights rounded to bf16 (round to nearest, ties to even) and FP32 sums; this
oracle takes the same bf16-valued weights as float64 and computes in float64.
Parameter vector layout (row-major W[out][in]):
W1[64][8], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 8, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_H, N_H)), ("b3", (N_H,)), ("W4", (N_H,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = p[o:o + n].reshape(shp)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x) -> np.ndarray:
    """FP32 -> bf16 (kept as float32 values), round to nearest, ties to even:
    add 0x7FFF plus the lowest kept bit to the 32-bit pattern, then clear the
    16 dropped bits (finite inputs)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def init_params(seed: int) -> np.ndarray:
    """He-uniform initial weights (FP32), zero biases."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[-1] if len(shp) == 2 else N_H
            lim = np.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-lim, lim, shp)
        else:
            d[name] = np.zeros(shp)
    return pack(d).astype(np.float32)


def forward(p64: np.ndarray, x: np.ndarray):
    """Network output for the rows of x, and the activations backward needs."""
    w = unpack(p64)
    z1 = x @ w["W1"].T + w["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ w["W2"].T + w["b2"]
    a2 = np.maximum(z2, 0.0)
    z3 = a2 @ w["W3"].T + w["b3"]
    a3 = np.maximum(z3, 0.0)
    y = a3 @ w["W4"] + w["b4"][0]
    return y, (x, z1, a1, z2, a2, z3, a3)


def loss(p64: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(p64, x)
    return float(np.mean((y - t) ** 2))


def gradient(p64: np.ndarray, x: np.ndarray, t: np.ndarray):
    """Backpropagation through the layers in reverse order; returns (loss,
    gradient vector in the parameter layout)."""
    w = unpack(p64)
    y, (x, z1, a1, z2, a2, z3, a3) = forward(p64, x)
    n = x.shape[0]
    dy = 2.0 * (y - t) / n                       # dL/dy
    g = {"W4": a3.T @ dy, "b4": np.array([dy.sum()])}
    d3 = np.outer(dy, w["W4"]) * (z3 > 0)        # dL/dz3
    g["W3"], g["b3"] = d3.T @ a2, d3.sum(0)
    d2 = (d3 @ w["W3"]) * (z2 > 0)
    g["W2"], g["b2"] = d2.T @ a1, d2.sum(0)
    d1 = (d2 @ w["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = d1.T @ x, d1.sum(0)
    return float(np.mean((y - t) ** 2)), pack(g)


def effective(master32: np.ndarray) -> np.ndarray:
    """The weights the engine computes with: bf16-rounded master, as float64."""
    return bf16_round(master32).astype(np.float64)


def adam_step(master: np.ndarray, m: np.ndarray, v: np.ndarray, g: np.ndarray, step: int,
              lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step = 1, 2, ...); returns new (master, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return master - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(master32: np.ndarray, x: np.ndarray, t: np.ndarray, steps: int, lr: float = 1e-3):
    """Full-batch Adam on the bf16-rounded weights; returns (master, losses)."""
    master = master32.astype(np.float64)
    m = np.zeros_like(master)
    v = np.zeros_like(master)
    losses = []
    for s in range(1, steps + 1):
        l, g = gradient(effective(master.astype(np.float32)), x, t)
        losses.append(l)
        master, m, v = adam_step(master, m, v, g, s, lr)
    return master, losses

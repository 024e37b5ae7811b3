"""CPU oracle of the planner network -- TEST INFRASTRUCTURE ONLY.

The same function as the library's MLP (24 -> 128 -> 128 -> 3, ReLU) in
float64 numpy: weights, inputs and hidden activations rounded to BF16 (round
to nearest, ties to even, written out from the IEEE-754 bit layout),
products and sums in float64.  Loss: sum M (Y - T)^2 / count(M != 0).
"""
from __future__ import annotations

import numpy as np

NIN, NH, NOUT = 24, 128, 3
SIZES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NOUT)),
         ("b3", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def bf16(x):
    """Round float values to the nearest BF16 value (ties to even), as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    nan = np.isnan(a)
    out = np.where(nan, a, out)
    return out.astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def forward(p, X, round_bf16=True):
    W = unpack(bf16(p) if round_bf16 else p)
    r = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    x = r(X)
    h1 = r(np.maximum(x @ W["W1"] + W["b1"], 0.0))
    h2 = r(np.maximum(h1 @ W["W2"] + W["b2"], 0.0))
    y = h2 @ W["W3"] + W["b3"]
    return x, h1, h2, y


def loss_and_grad(p, X, T, M, round_bf16=True):
    """Loss and its gradient with respect to the (rounded) parameters."""
    W = unpack(bf16(p) if round_bf16 else p)
    x, h1, h2, y = forward(p, X, round_bf16)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(1.0, float((M != 0).sum()))
    e = y - np.asarray(T, dtype=np.float64)
    loss = float((M * e * e).sum() / cnt)
    dy = 2.0 * M * e / cnt
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dh2 = (dy @ W["W3"].T) * (h2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ W["W2"].T) * (h1 > 0)
    g["W1"] = x.T @ dh1
    g["b1"] = dh1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SIZES])


def init_params(seed: int):
    """He-uniform weights, zero biases."""
    g = np.random.default_rng(seed)
    parts = []
    for name, shape in SIZES:
        if name.startswith("W"):
            lim = np.sqrt(6.0 / shape[0])
            parts.append(g.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(shape).ravel())
    return np.concatenate(parts).astype(np.float32)

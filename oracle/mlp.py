"""Plain numpy reference of the subset-proposal network (FP64).

TEST INFRASTRUCTURE ONLY: the gradient checks of the GPU network compare against it; the
library never imports it.  Parity of this module itself is pinned by central finite
differences (tests/test_oracle_mlp.py).

The network maps 20 inputs to one output: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
y = w3 . h2 + b3, with W1 256 x 20, W2 256 x 256.  The loss of a batch is the mean of
(y - t)^2.  Parameters are one flat vector: W1 (row-major, output x input), b1, W2, b2,
w3, b3.

With ``bf16=True`` values are rounded to bfloat16 (round to nearest even) exactly where
the GPU stores them in 16 bits: the inputs, W1 and W2, the hidden activations h1 and h2,
and the back-propagated pre-activation gradients of both hidden layers; every product is
otherwise exact (FP64 here, FP32 accumulation on the GPU).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 20, 256
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) and back to float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X, bf16_points: bool = False):
    """Network outputs and the cached activations."""
    P = unpack(p)
    r = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    x = r(np.asarray(X, dtype=np.float64))
    W1, W2 = r(P["W1"]), r(P["W2"])
    h1 = r(np.maximum(x @ W1.T + P["b1"], 0.0))
    h2 = r(np.maximum(h1 @ W2.T + P["b2"], 0.0))
    y = h2 @ P["w3"] + P["b3"][0]
    return y, (x, W1, W2, h1, h2)


def loss_and_grad(p, X, t, bf16_points: bool = False):
    """Mean squared error of the batch and its gradient (flat, parameter layout)."""
    P = unpack(p)
    r = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    t = np.asarray(t, dtype=np.float64)
    B = t.size
    y, (x, W1, W2, h1, h2) = forward(p, X, bf16_points)
    e = y - t
    loss = float(np.mean(e * e))
    d = 2.0 * e / B                                  # dL/dy
    g = {"w3": h2.T @ d, "b3": np.array([d.sum()])}
    dz2 = r(np.where(h2 > 0, d[:, None] * P["w3"][None, :], 0.0))
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = r(np.where(h1 > 0, dh1, 0.0))
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def numeric_grad(p, X, t, idx, h: float = 1e-6):
    """Central differences of the (unrounded) loss for the parameters idx."""
    out = np.zeros(len(idx))
    for k, i in enumerate(idx):
        q = np.array(p, dtype=np.float64)
        q[i] += h
        lp, _ = loss_and_grad(q, X, t)
        q[i] -= 2 * h
        lm, _ = loss_and_grad(q, X, t)
        out[k] = (lp - lm) / (2 * h)
    return out

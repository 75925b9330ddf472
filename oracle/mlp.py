"""Plain fp64 numpy reference of the learned estimator's network -- TEST INFRASTRUCTURE ONLY.

The learned estimator is not part of the paper (which estimates with Thm. 2
alone); this module is the reference its GPU kernels are checked against:
x (16) -> ReLU(W1 x + b1) (64) -> ReLU(W2 h1 + b2) (64) -> W3 h2 + b3, with
the flat parameter order W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3.
Weights are taken exactly as the kernels see them (BF16 values widened to
fp64); everything else is fp64.
"""
from __future__ import annotations

import numpy as np

IN, HID = 16, 64
SIZES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].astype(np.float64).reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SIZES])


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    """uint16 BF16 bit patterns -> fp64 values (exact)."""
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def forward(flat: np.ndarray, X: np.ndarray):
    p = unpack(flat)
    X = X.astype(np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (X, a1, h1, a2, h2)


def loss_and_grad(flat: np.ndarray, X: np.ndarray, t: np.ndarray, scale: float):
    """(sum of squared errors, gradient of scale * sum (y - t)^2) by backpropagation."""
    p = unpack(flat)
    y, (X, a1, h1, a2, h2) = forward(flat, X)
    r = y - t.astype(np.float64)
    d3 = 2.0 * r * scale                      # dL/dy
    g = {"W3": h2.T @ d3, "b3": np.array([d3.sum()])}
    d2 = np.outer(d3, p["W3"]) * (a2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (a1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return float((r * r).sum()), pack(g)

"""Plain float64 reference of the surrogate network (TEST INFRASTRUCTURE ONLY: imported by
tests/ and nothing else).  It shares no code with the CUDA kernels.

Network: x[7] -> 256 -> 256 -> 192, GELU in its tanh form
    g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
linear output, loss = mean over batch and outputs of (y - t)^2.  Parameters in the flat
layout W1[256][7], b1[256], W2[256][256], b2[256], W3[192][256], b3[192].

`bf16=True` rounds to bfloat16 (round to nearest, ties to even) at the points where the
GPU kernels keep BF16 values: the inputs, the weights, the hidden activations, and the
output and hidden gradients that feed the next matrix product.  All arithmetic is float64.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 7, 256, 192
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
C_GELU = np.sqrt(2.0 / np.pi)


def unflatten(p: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[off:off + n], dtype=np.float64).reshape(shp)
        off += n
    return out


def flatten(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(C_GELU * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU * (1.0 + 3.0 * 0.044715 * z * z)


def forward(p: np.ndarray, x: np.ndarray, bf16_points: bool = False) -> tuple[np.ndarray, dict]:
    q = unflatten(p)
    r = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    X = r(x)
    W1, W2, W3 = r(q["W1"]), r(q["W2"]), r(q["W3"])
    Z1 = X @ W1.T + q["b1"]
    H1 = r(gelu(Z1))
    Z2 = H1 @ W2.T + q["b2"]
    H2 = r(gelu(Z2))
    Y = H2 @ W3.T + q["b3"]
    return Y, dict(X=X, W1=W1, W2=W2, W3=W3, Z1=Z1, H1=H1, Z2=Z2, H2=H2)


def loss(p, x, t, bf16_points: bool = False) -> float:
    y, _ = forward(p, x, bf16_points)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(p: np.ndarray, x: np.ndarray, t: np.ndarray, bf16_points: bool = False):
    """(flat gradient of the loss, loss), by the chain rule layer by layer."""
    r = bf16 if bf16_points else (lambda a: np.asarray(a, dtype=np.float64))
    y, c = forward(p, x, bf16_points)
    B = y.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    L = float(np.mean(d ** 2))
    dY = 2.0 * d / (B * N_OUT)
    dYr = r(dY)
    g = {"W3": dYr.T @ c["H2"], "b3": dY.sum(axis=0)}
    dH2 = dYr @ c["W3"]
    dZ2 = dH2 * gelu_grad(c["Z2"])
    dZ2r = r(dZ2)
    g["W2"] = dZ2r.T @ c["H1"]
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2r @ c["W2"]
    dZ1 = dH1 * gelu_grad(c["Z1"])
    g["W1"] = r(dZ1).T @ c["X"]
    g["b1"] = dZ1.sum(axis=0)
    return flatten(g), L

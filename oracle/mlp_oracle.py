"""FP64 CPU oracle of the learned-kernel network.

TEST INFRASTRUCTURE ONLY: imported by tests/ (never by the product package).

The network is this project's extension of the method, not part of the paper:
it maps a visibility's w and sub-grid offset to its w-kernel (Section 3.1) on a
fixed 32 x 32 window of grid cells plus a support mask (Section 3.2's kept set).
This module is its plain definition in float64 NumPy, written out layer by
layer, and its gradient by the chain rule; the pins in tests/ check the
gradient against central finite differences of the loss.

    h1 = GELU(W1 x0 + b1), h2 = GELU(W2 h1 + b2), h3 = GELU(W3 h2 + b3)
    y  = W4 h3 + b4                                   (2048 values, 1024 logits)
    loss = mean_values (y - t)^2 + mask_weight * mean_mask BCE(logit, t_mask)
    GELU(z) = z Phi(z), Phi the standard normal CDF (erf form).

Parameters are one flat vector: W1 (256x3), b1, W2 (256x256), b2, W3 (256x256),
b3, W4 (3072x256), b4, matrices stored row-major [out][in].
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

N_IN, N_HID, N_VAL, N_MASK = 3, 256, 2048, 1024
N_OUT = N_VAL + N_MASK
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    return z * 0.5 * (1.0 + scipy.special.erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    """d/dz z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + scipy.special.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(flat: np.ndarray, x0: np.ndarray) -> dict:
    P = unpack(flat)
    x0 = np.asarray(x0, dtype=np.float64)
    z1 = x0 @ P["W1"].T + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    z3 = h2 @ P["W3"].T + P["b3"]
    h3 = gelu(z3)
    y = h3 @ P["W4"].T + P["b4"]
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3, "h3": h3, "y": y}


def loss(y: np.ndarray, tv: np.ndarray, tm: np.ndarray, mask_weight: float) -> float:
    yv, ym = y[:, :N_VAL], y[:, N_VAL:]
    mse = np.mean((yv - tv) ** 2)
    # binary cross-entropy with logits, written in the overflow-safe form
    bce = np.mean(np.maximum(ym, 0.0) - tm * ym + np.log1p(np.exp(-np.abs(ym))))
    return float(mse + mask_weight * bce)


def gradients(flat: np.ndarray, x0: np.ndarray, tv: np.ndarray, tm: np.ndarray, mask_weight: float):
    """(loss, flat gradient) by the chain rule."""
    P = unpack(flat)
    f = forward(flat, x0)
    B = x0.shape[0]
    y = f["y"]
    dy = np.empty_like(y)
    dy[:, :N_VAL] = 2.0 * (y[:, :N_VAL] - tv) / (B * N_VAL)
    dy[:, N_VAL:] = mask_weight * (scipy.special.expit(y[:, N_VAL:]) - tm) / (B * N_MASK)
    g = {}
    g["W4"] = dy.T @ f["h3"]
    g["b4"] = dy.sum(axis=0)
    dh3 = dy @ P["W4"]
    dz3 = dh3 * gelu_prime(f["z3"])
    g["W3"] = dz3.T @ f["h2"]
    g["b3"] = dz3.sum(axis=0)
    dh2 = dz3 @ P["W3"]
    dz2 = dh2 * gelu_prime(f["z2"])
    g["W2"] = dz2.T @ f["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * gelu_prime(f["z1"])
    g["W1"] = dz1.T @ np.asarray(x0, dtype=np.float64)
    g["b1"] = dz1.sum(axis=0)
    return loss(y, tv, tm, mask_weight), pack(g)


def round_bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)

"""Bicubic upscaling oracle (FP64, numpy). TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 2 initialises each scale after the first by upscaling the previous result by 2; the
paper does not name the interpolation. Reading used: bicubic convolution (Keys kernel with
a = -0.75), half-pixel sample centres (source coordinate (i + 0.5) * h / H - 0.5), and
edge-clamped source indices. Output size H x W is given (normally 2h x 2w).
"""
from __future__ import annotations

import numpy as np

A = -0.75


def keys(t):
    """Keys cubic convolution kernel with parameter A."""
    t = np.abs(t)
    return np.where(t <= 1, ((A + 2) * t - (A + 3)) * t * t + 1,
                    np.where(t < 2, ((A * t - 5 * A) * t + 8 * A) * t - 4 * A, 0.0))


def _weights(n_out, n_in):
    """(n_out, 4) source indices (clamped) and weights along one axis."""
    scale = n_in / n_out
    src = (np.arange(n_out) + 0.5) * scale - 0.5
    i0 = np.floor(src).astype(np.int64)
    t = src - i0
    idx = np.stack([i0 - 1, i0, i0 + 1, i0 + 2], axis=1)
    w = np.stack([keys(1 + t), keys(t), keys(1 - t), keys(2 - t)], axis=1)
    return np.clip(idx, 0, n_in - 1), w


def upsample(x, H, W):
    """x: C x h x w -> C x H x W, separable bicubic (rows then columns), float64."""
    x = np.asarray(x, np.float64)
    C, h, w = x.shape
    iy, wy = _weights(H, h)
    ix, wx = _weights(W, w)
    out = np.empty((C, H, W))
    for c in range(C):
        rows = (x[c][iy] * wy[:, :, None]).sum(axis=1)          # H x w
        out[c] = (rows[:, ix] * wx[None, :, :]).sum(axis=2)      # H x W
    return out

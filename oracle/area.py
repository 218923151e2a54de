"""Area-average downscaling oracle (FP64, numpy). TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 2 downscales the content and style images by 2^(n_scales - s) at scale s; the paper
does not name the filter. Reading used: area averaging (adaptive average pooling): output pixel
i along an axis averages the input indices [floor(i h / H), ceil((i + 1) h / H)), uniformly,
separately along rows and columns; for an integer factor f = h / H this is the f x f box mean.
"""
from __future__ import annotations

import numpy as np


def _ranges(n_out, n_in):
    return [((i * n_in) // n_out, -((-(i + 1) * n_in) // n_out)) for i in range(n_out)]


def downscale(x, H, W):
    """x: C x h x w -> C x H x W (H <= h, W <= w), float64."""
    x = np.asarray(x, np.float64)
    C, h, w = x.shape
    ry, rx = _ranges(H, h), _ranges(W, w)
    tmp = np.stack([x[:, a:b, :].mean(axis=1) for a, b in ry], axis=1)      # C x H x w
    return np.stack([tmp[:, :, a:b].mean(axis=2) for a, b in rx], axis=2)   # C x H x W

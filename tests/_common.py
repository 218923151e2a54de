"""Helpers shared by the tests: seeded problem set-up through the oracle (FP64)."""
import numpy as np

import oracle
from paper_2212_13459_gb300 import synth

# equal style weights (beta = 1 split over the five layers) and alpha/beta = 1e-3
W_STYLE = np.full(5, 0.2)
LAMBDA_C = 1e-3


def problem(H, W, seed=0, Hv=None, Wv=None, bias_std=0.0, style="noise"):
    """Seeded (params, packed params, u, v) for an H x W content and an Hv x Wv style image."""
    params = synth.vgg19_params(seed, bias_std=bias_std)
    P = oracle.pack_params(params)
    u = synth.content_image(H, W, seed)
    Hv = Hv or H
    Wv = Wv or W
    v = synth.noise_style(Hv, Wv, seed) if style == "noise" else synth.stroke_style(Hv, Wv, seed)
    return params, P, u, v


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

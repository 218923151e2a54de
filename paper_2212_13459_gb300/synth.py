"""Seeded synthetic inputs: images shaped like the paper's and random-init VGG-19 weights.

This module serves both the library's callers (bench, tests) and the FP64 oracle's tests. It holds
none of the method's arithmetic: it only draws numbers. The paper's photographs, paintings and
pretrained VGG-19 weights are not available, so these stand in for them:

* ``content_image``: smooth seeded colour ramps plus random axis-aligned rectangles (a stand-in
  for a photograph: large smooth regions with sharp edges).
* ``noise_style``: multi-octave value noise mapped through a six-colour palette.
* ``stroke_style``: a painting-like texture: anisotropic Gaussian brush strokes over a palette,
  one-pixel crack lines (random walks, darkened) and a canvas-weave sinusoid.
* ``vgg19_params``: He-normal weights N(0, 2/(9 Cin)), layout [Cout][Cin][3][3], conv1_1..conv5_1,
  zero biases by default.

All images are float32, C x H x W (RGB), values in [0, 1].
"""
from __future__ import annotations

import numpy as np

# (Cin, Cout) of the 13 convolutions conv1_1 ... conv5_1 of VGG-19
VGG19_CONVS = [(3, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256), (256, 256),
               (256, 256), (256, 512), (512, 512), (512, 512), (512, 512), (512, 512)]
CONV_NAMES = ["conv1_1", "conv1_2", "conv2_1", "conv2_2", "conv3_1", "conv3_2", "conv3_3",
              "conv3_4", "conv4_1", "conv4_2", "conv4_3", "conv4_4", "conv5_1"]


def vgg19_params(seed: int = 0, bias_std: float = 0.0):
    """List of 13 (W [Cout,Cin,3,3] float32, b [Cout] float32), He-normal, seeded."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout in VGG19_CONVS:
        w = rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2.0 / (9.0 * cin))
        if bias_std > 0:
            b = rng.standard_normal(cout) * bias_std
        else:
            b = np.zeros(cout)
        out.append((w.astype(np.float32), b.astype(np.float32)))
    return out


def flat_params(params) -> np.ndarray:
    """Concatenate [W_0, b_0, W_1, b_1, ...] into one float32 vector (the library's input format)."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params]).astype(
        np.float32)


def _palette(rng, n=6):
    return rng.uniform(0.05, 0.95, size=(n, 3))


def content_image(H: int, W: int, seed: int = 0) -> np.ndarray:
    """Three random linear ramps per channel plus 12 random axis-aligned rectangles."""
    rng = np.random.default_rng(seed)
    yy = np.linspace(0.0, 1.0, H, dtype=np.float64)[:, None]
    xx = np.linspace(0.0, 1.0, W, dtype=np.float64)[None, :]
    img = np.zeros((3, H, W))
    for c in range(3):
        acc = np.zeros((H, W))
        for _ in range(3):
            a, b = rng.uniform(-1, 1, size=2)
            acc += a * yy + b * xx
        acc -= acc.min()
        acc /= max(acc.max(), 1e-9)
        img[c] = 0.2 + 0.6 * acc
    for _ in range(12):
        h = int(rng.integers(max(1, H // 16), max(2, H // 3)))
        w = int(rng.integers(max(1, W // 16), max(2, W // 3)))
        y0 = int(rng.integers(0, max(1, H - h)))
        x0 = int(rng.integers(0, max(1, W - w)))
        col = rng.uniform(0, 1, size=3)
        img[:, y0:y0 + h, x0:x0 + w] = col[:, None, None]
    return np.ascontiguousarray(np.clip(img, 0, 1), dtype=np.float32)


def _value_noise(H, W, rng, octaves=5, persistence=0.5, base=4):
    out = np.zeros((H, W))
    amp, tot = 1.0, 0.0
    for o in range(octaves):
        cells = base * (2 ** o)
        gh, gw = cells + 2, int(np.ceil(cells * W / max(H, 1))) + 2
        grid = rng.uniform(0, 1, size=(gh, gw))
        ys = np.linspace(0, cells, H, endpoint=False)
        xs = np.linspace(0, gw - 2, W, endpoint=False)
        y0 = np.floor(ys).astype(int)
        x0 = np.floor(xs).astype(int)
        ty = ys - y0
        tx = xs - x0
        ty = ty * ty * (3 - 2 * ty)
        tx = tx * tx * (3 - 2 * tx)
        g00 = grid[y0][:, x0]
        g01 = grid[y0][:, x0 + 1]
        g10 = grid[y0 + 1][:, x0]
        g11 = grid[y0 + 1][:, x0 + 1]
        top = g00 * (1 - tx)[None, :] + g01 * tx[None, :]
        bot = g10 * (1 - tx)[None, :] + g11 * tx[None, :]
        out += amp * (top * (1 - ty)[:, None] + bot * ty[:, None])
        tot += amp
        amp *= persistence
    return out / tot


def noise_style(H: int, W: int, seed: int = 0) -> np.ndarray:
    """Five-octave value noise (persistence 0.5) mapped through a seeded six-colour palette."""
    rng = np.random.default_rng(seed + 1000)
    pal = _palette(rng)
    n = _value_noise(H, W, rng)
    n = (n - n.min()) / max(n.max() - n.min(), 1e-9) * (len(pal) - 1)
    i0 = np.clip(np.floor(n).astype(int), 0, len(pal) - 2)
    t = (n - i0)[..., None]
    img = pal[i0] * (1 - t) + pal[i0 + 1] * t
    return np.ascontiguousarray(np.clip(img.transpose(2, 0, 1), 0, 1), dtype=np.float32)


def stroke_style(H: int, W: int, seed: int = 0, n_strokes: int = 2000) -> np.ndarray:
    """Painting-like texture: anisotropic Gaussian strokes, crack lines and canvas weave."""
    rng = np.random.default_rng(seed + 2000)
    pal = _palette(rng)
    img = np.empty((H, W, 3))
    img[:] = pal[0] * 0.8 + 0.1
    short = min(H, W)
    for _ in range(n_strokes):
        length = rng.uniform(0.005, 0.04) * short
        aspect = rng.uniform(3.0, 10.0)
        width = max(length / aspect, 0.5)
        ang = rng.uniform(0, np.pi)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        col = pal[int(rng.integers(0, len(pal)))] * rng.uniform(0.85, 1.15)
        alpha = rng.uniform(0.6, 0.9)
        r = int(np.ceil(3 * length))
        y0, y1 = max(0, int(cy) - r), min(H, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(W, int(cx) + r + 1)
        if y1 <= y0 or x1 <= x0:
            continue
        ys = np.arange(y0, y1)[:, None] - cy
        xs = np.arange(x0, x1)[None, :] - cx
        u = xs * np.cos(ang) + ys * np.sin(ang)
        v = -xs * np.sin(ang) + ys * np.cos(ang)
        a = alpha * np.exp(-0.5 * ((u / length) ** 2 + (v / width) ** 2))
        img[y0:y1, x0:x1] = img[y0:y1, x0:x1] * (1 - a[..., None]) + col * a[..., None]
    # crack lines: 1-px random walks that darken the paint
    n_cracks = max(4, int(40 * (H * W) / (1024 * 1024)))
    for _ in range(n_cracks):
        y, x = rng.uniform(0, H), rng.uniform(0, W)
        ang = rng.uniform(0, 2 * np.pi)
        steps = int(rng.integers(short // 8, short // 2 + 2))
        turns = rng.normal(0, 0.3, size=steps)
        for k in range(steps):
            ang += turns[k]
            y += np.sin(ang)
            x += np.cos(ang)
            iy, ix = int(y), int(x)
            if 0 <= iy < H and 0 <= ix < W:
                img[iy, ix] *= 0.7
            else:
                break
    # canvas weave
    yy = np.arange(H)[:, None]
    xx = np.arange(W)[None, :]
    img += (0.05 * np.sin(2 * np.pi * xx / 8) * np.sin(2 * np.pi * yy / 8))[..., None]
    return np.ascontiguousarray(np.clip(img.transpose(2, 0, 1), 0, 1), dtype=np.float32)


def scale2_result(H: int, W: int, seed: int = 0) -> np.ndarray:
    """A stand-in for the output of the previous scale: content generator with a stroke overlay."""
    base = content_image(H, W, seed)
    strokes = stroke_style(H, W, seed + 7, n_strokes=max(200, (H * W) // 4000))
    return np.ascontiguousarray(np.clip(0.6 * base + 0.4 * strokes, 0, 1), dtype=np.float32)

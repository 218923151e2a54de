"""Multiscale driver oracle (Algorithm 2). TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Composed only of the pinned oracle parts: area downscaling (oracle/area.py), bicubic upscaling
(oracle/bicubic.py), the L-BFGS two-loop recursion (oracle/lbfgs.py) and the untiled loss and
gradient of the C oracle. Algorithm 2 as read here:

  for s = 1 .. n:
      f = 2^(n - s); u_s, v_s = u, v downscaled by f (area averaging; sizes n / f rounded half
      up, at least 16: 4226 / 4 -> 1057, reading 18)
      x = u_s at s = 1 (or a given x0: texture synthesis starts from white noise at the coarsest
      scale, Section 6.2), else the previous x upscaled to the size of u_s (bicubic)
      `iters[s - 1]` L-BFGS iterations on E with the targets of (u_s, v_s): history 100 at
      the first scale, 10 afterwards (Section 5.1)

Each iteration is one evaluation of E and dE/dx followed by one L-BFGS step, as in the library's
driver.
"""
from __future__ import annotations

import numpy as np

from . import area, bicubic, content_target, loss_grad, storage, style_grams
from .lbfgs import LBFGS


def scaled(n, f):
    """n / f rounded half up, at least 16 px."""
    return max(16, int(n / f + 0.5))


def multiscale(P, u, v, n_scales, iters, w_style, lambda_c, x0=None, storage_mode="f64"):
    """Returns (x at the finest scale, [(scale, iteration, E)] for every evaluation)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    w_style = np.asarray(w_style, np.float64)
    x = None
    losses = []
    for s in range(1, n_scales + 1):
        f = 2 ** (n_scales - s)
        Hs, Ws = scaled(u.shape[1], f), scaled(u.shape[2], f)
        Hv, Wv = scaled(v.shape[1], f), scaled(v.shape[2], f)
        us = u if f == 1 else area.downscale(u, Hs, Ws)
        vs = v if f == 1 else area.downscale(v, Hv, Wv)
        if x is None:
            x = np.array(us if x0 is None else x0, np.float64)
            assert x.shape == us.shape
        else:
            x = bicubic.upsample(x, Hs, Ws)
        with storage(storage_mode):
            ct = content_target(P, us)
            Gv = style_grams(P, vs)
        opt = LBFGS(x.size, 100 if s == 1 else 10)
        xf = x.reshape(-1)
        for k in range(iters[s - 1]):
            with storage(storage_mode):
                E, g, _, _ = loss_grad(P, xf.reshape(x.shape), ct, Gv, w_style, lambda_c)
            losses.append((s, k, E))
            opt.step(xf, g.reshape(-1))
        x = xf.reshape(x.shape)
    return x, losses

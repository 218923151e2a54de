"""FP64 CPU oracle for the localized style-transfer loss and gradient.

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg
may import this package. The library under test (``paper_2212_13459_gb300``) never imports it and
shares no code with it; the only shared module is the seeded input generator ``synth``.

Contents:
* ``nst_oracle.c`` (compiled with gcc, OpenMP): VGG-19 to ReLU5_1, Gram/content losses, Table 1
  feature gradients, the hand-written reverse pass, and Algorithm 1 (blocks with margins).
* ``lbfgs.py``: L-BFGS two-loop recursion and the dense inverse-BFGS matrix it must equal.
* ``bicubic.py``: x2 bicubic upscaling (the initialisation step of Algorithm 2).

Pins of this oracle against things other than itself live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nst_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

NSTYLE = 5
STYLE_CONVS = [0, 2, 4, 8, 12]
STYLE_CHANNELS = [64, 128, 256, 512, 512]
STYLE_STRIDES = [1, 2, 4, 8, 16]
CONTENT_CONV = 9
CONV_COUT = [64, 64, 128, 128, 256, 256, 256, 256, 512, 512, 512, 512, 512]
CONV_STRIDE = [1, 1, 2, 2, 4, 4, 4, 4, 8, 8, 8, 8, 16]


def build(force: bool = False) -> str:
    """Compile nst_oracle.c into _build/liboracle.so (plain gcc, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_param_count.restype = ctypes.c_long
            L.orc_features.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            L.orc_style_grams.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
            L.orc_content_target.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
            L.orc_loss_grad.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                        ctypes.c_double, dp, dp, dp, dp]
            L.orc_loss_grad_tiled.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                              ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            L.orc_table1_gram.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                          dp, dp]
            L.orc_table1_mse.argtypes = [dp, dp, ctypes.c_long, ctypes.c_double, dp, dp]
            L.orc_plan_1d.argtypes = [ctypes.c_int, ctypes.c_int, ip]
            L.orc_set_storage.argtypes = [ctypes.c_int]
            L.orc_style_moments.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_loss_grad_aug.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
                                            dp, dp, dp, ctypes.c_double, dp, dp, dp, dp]
            L.orc_loss_grad_tiled_aug.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                                  dp, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                                  dp, dp]
            L.orc_relu11.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp]
            L.orc_block_style_grad.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                               dp, dp]
            L.orc_table1_mean.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                          dp, dp]
            L.orc_table1_std.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_double,
                                         dp, dp]
            _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle error %d" % rc)


STORAGE = {"f64": 0, "f32": 1, "bf16": 2}


class storage:
    """Context manager: evaluate the oracle with values rounded where the evaluated form stores
    them (\"f32\" or \"bf16\"; \"f64\" = the plain definition). See nst_oracle.c."""

    def __init__(self, mode):
        self.mode = STORAGE[mode]

    def __enter__(self):
        lib().orc_set_storage(self.mode)
        return self

    def __exit__(self, *exc):
        lib().orc_set_storage(0)
        return False


def pack_params(params) -> np.ndarray:
    """[(W, b)] * 13 (any float dtype) -> one float64 vector in the oracle's parameter order."""
    v = np.concatenate([np.concatenate([np.asarray(w, np.float64).ravel(),
                                        np.asarray(b, np.float64).ravel()]) for w, b in params])
    assert v.size == lib().orc_param_count()
    return np.ascontiguousarray(v)


def _img(x):
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    assert x.ndim == 3 and x.shape[0] == 3
    return x


def features(P, x, conv):
    x = _img(x)
    H, W = x.shape[1:]
    s = CONV_STRIDE[conv]
    out = np.zeros((CONV_COUT[conv], H // s, W // s))
    _check(lib().orc_features(_p(P), _p(x), H, W, conv, _p(out)))
    return out


def style_grams(P, v):
    """G^L(v) for L in L_s, as a list of 5 square float64 arrays."""
    v = _img(v)
    H, W = v.shape[1:]
    tot = sum(c * c for c in STYLE_CHANNELS)
    out = np.zeros(tot)
    _check(lib().orc_style_grams(_p(P), _p(v), H, W, _p(out)))
    return split_grams(out)


def split_grams(flat):
    res, o = [], 0
    for c in STYLE_CHANNELS:
        res.append(flat[o:o + c * c].reshape(c, c).copy())
        o += c * c
    return res


def join_grams(gs):
    return np.ascontiguousarray(np.concatenate([np.asarray(g, np.float64).ravel() for g in gs]))


def content_target(P, u):
    u = _img(u)
    H, W = u.shape[1:]
    out = np.zeros((512, H // 8, W // 8))
    _check(lib().orc_content_target(_p(P), _p(u), H, W, _p(out)))
    return out


def loss_grad(P, x, content_t, style_G, w_style, lambda_c, want_grad=True):
    """Untiled E(x) and dE/dx. Returns (E, grad or None, parts[6], grams[5])."""
    x = _img(x)
    H, W = x.shape[1:]
    ct = np.ascontiguousarray(content_t, np.float64)
    sg = join_grams(style_G)
    ws = np.ascontiguousarray(w_style, np.float64)
    E = np.zeros(1)
    parts = np.zeros(6)
    grams = np.zeros(sg.size)
    grad = np.zeros((3, H, W)) if want_grad else None
    _check(lib().orc_loss_grad(_p(P), _p(x), H, W, _p(ct), _p(sg), _p(ws), float(lambda_c),
                               _p(E), _p(grad), _p(parts), _p(grams)))
    return float(E[0]), grad, parts, split_grams(grams)


def loss_grad_tiled(P, x, content_t, style_G, w_style, lambda_c, tiles, margins,
                    want_grad=True):
    """Algorithm 1 with a tiles[0] x tiles[1] partition and margins (step 1, step 2)."""
    x = _img(x)
    H, W = x.shape[1:]
    ct = np.ascontiguousarray(content_t, np.float64)
    sg = join_grams(style_G)
    ws = np.ascontiguousarray(w_style, np.float64)
    E = np.zeros(1)
    parts = np.zeros(6)
    grams = np.zeros(sg.size)
    grad = np.zeros((3, H, W)) if want_grad else None
    _check(lib().orc_loss_grad_tiled(_p(P), _p(x), H, W, _p(ct), _p(sg), _p(ws),
                                     float(lambda_c), int(tiles[0]), int(tiles[1]),
                                     int(margins[0]), int(margins[1]), _p(E), _p(grad),
                                     _p(parts), _p(grams)))
    return float(E[0]), grad, parts, split_grams(grams)


def table1_gram(V, Gref, w):
    V = np.ascontiguousarray(V, np.float64)
    npx, nc = V.shape
    Gref = np.ascontiguousarray(Gref, np.float64)
    E = np.zeros(1)
    g = np.zeros_like(V)
    lib().orc_table1_gram(_p(V), npx, nc, _p(Gref), float(w), _p(E), _p(g))
    return float(E[0]), g


def table1_mse(V, Vref, lam):
    V = np.ascontiguousarray(V, np.float64)
    Vref = np.ascontiguousarray(Vref, np.float64)
    E = np.zeros(1)
    g = np.zeros_like(V)
    lib().orc_table1_mse(_p(V), _p(Vref), V.size, float(lam), _p(E), _p(g))
    return float(E[0]), g


def plan_1d(L, k):
    b = (ctypes.c_int * (k + 1))()
    rc = lib().orc_plan_1d(int(L), int(k), b)
    _check(rc)
    return list(b)


STYLE_MOMENTS = sum(STYLE_CHANNELS)   # 1,472


def split_vec(flat):
    res, o = [], 0
    for c in STYLE_CHANNELS:
        res.append(flat[o:o + c].copy())
        o += c
    return res


def style_moments(P, v):
    """(mean, std) of the five style layers of v: lists of per-channel vectors (Eq. 5)."""
    v = _img(v)
    H, W = v.shape[1:]
    m = np.zeros(STYLE_MOMENTS)
    sd = np.zeros(STYLE_MOMENTS)
    _check(lib().orc_style_moments(_p(P), _p(v), H, W, _p(m), _p(sd)))
    return split_vec(m), split_vec(sd)


def loss_grad_aug(P, x, content_t, style_G, style_mean, style_std, w_style, w_mean, w_std,
                  lambda_c, want_grad=True, tiles=None, margins=(80, 160)):
    """E(x) with the augmented style loss of Eq. 5 and dE/dx; untiled, or Algorithm 1 with
    `tiles` blocks. Returns (E, grad or None, parts[6], grams[5])."""
    x = _img(x)
    H, W = x.shape[1:]
    ct = np.ascontiguousarray(content_t, np.float64)
    sg = join_grams(style_G)
    sm = np.ascontiguousarray(np.concatenate(style_mean), np.float64)
    ss = np.ascontiguousarray(np.concatenate(style_std), np.float64)
    ws = np.ascontiguousarray(w_style, np.float64)
    wm = np.ascontiguousarray(w_mean, np.float64)
    wsd = np.ascontiguousarray(w_std, np.float64)
    E = np.zeros(1)
    parts = np.zeros(6)
    grams = np.zeros(sg.size)
    grad = np.zeros((3, H, W)) if want_grad else None
    if tiles is None:
        _check(lib().orc_loss_grad_aug(_p(P), _p(x), H, W, _p(ct), _p(sg), _p(sm), _p(ss),
                                       _p(ws), _p(wm), _p(wsd), float(lambda_c), _p(E), _p(grad),
                                       _p(parts), _p(grams)))
    else:
        _check(lib().orc_loss_grad_tiled_aug(_p(P), _p(x), H, W, _p(ct), _p(sg), _p(sm), _p(ss),
                                             _p(ws), _p(wm), _p(wsd), float(lambda_c),
                                             int(tiles[0]), int(tiles[1]), int(margins[0]),
                                             int(margins[1]), _p(E), _p(grad), _p(parts),
                                             _p(grams)))
    return float(E[0]), grad, parts, split_grams(grams)


def table1_mean(V, mu, w):
    V = np.ascontiguousarray(V, np.float64)
    npx, nc = V.shape
    E = np.zeros(1)
    g = np.zeros_like(V)
    lib().orc_table1_mean(_p(V), npx, nc, _p(np.ascontiguousarray(mu, np.float64)), float(w),
                          _p(E), _p(g))
    return float(E[0]), g


def table1_std(V, sigma, w):
    V = np.ascontiguousarray(V, np.float64)
    npx, nc = V.shape
    E = np.zeros(1)
    g = np.zeros_like(V)
    lib().orc_table1_std(_p(V), npx, nc, _p(np.ascontiguousarray(sigma, np.float64)), float(w),
                         _p(E), _p(g))
    return float(E[0]), g


def relu11_gram(P, x, strip=192):
    """G^{ReLU1_1}(x) = V V^T / n_p of a large image, strip by strip: conv1_1 features of each
    row strip (with a 1-row halo on each side, dropped afterwards) summed with numpy in FP64."""
    x = _img(x)
    _, H, W = x.shape
    S = np.zeros((64, 64))
    for y0 in range(0, H, strip):
        y1 = min(H, y0 + strip)
        a, b = max(0, y0 - 1), min(H, y1 + 1)
        blk = np.ascontiguousarray(x[:, a:b])
        out = np.zeros((64, b - a, W))
        _check(lib().orc_relu11(_p(P), _p(blk), b - a, W, _p(out)))
        V = out[:, y0 - a:y0 - a + (y1 - y0)].reshape(64, -1)
        S += V @ V.T
    return S / (H * W)


def block_style_grad(P, blk, G_glob, G_ref, np_glob, w_style):
    """Algorithm 1, Step 2 for one block with the given global statistics (no content term)."""
    blk = _img(blk)
    _, h, w = blk.shape
    out = np.zeros((3, h, w))
    _check(lib().orc_block_style_grad(_p(P), _p(blk), h, w, _p(join_grams(G_glob)),
                                      _p(join_grams(G_ref)),
                                      _p(np.ascontiguousarray(np_glob, np.float64)),
                                      _p(np.ascontiguousarray(w_style, np.float64)), _p(out)))
    return out

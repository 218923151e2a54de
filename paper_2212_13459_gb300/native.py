"""Thin ctypes binding of libnst (include/nst.h): argument marshalling only.

Every step of the loss/gradient path runs inside libnst's CUDA kernels; this module only turns
torch tensors into device pointers and the current CUDA stream into a handle. There is no CPU or
PyTorch fallback: if libnst.so has not been built, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libnst.so")
_lib = None
_lock = threading.Lock()

NST_OK, NST_ERR_INVALID_ARG, NST_ERR_SHAPE, NST_ERR_CUDA, NST_ERR_OOM = 0, 1, 2, 3, 4
NST_ERR_TIMEOUT, NST_ERR_NONFINITE, NST_ERR_STATE = 5, 6, 7
PREC_FP32, PREC_BF16 = 0, 1
CONV_AUTO, CONV_SIMT, CONV_TC = 0, 1, 2
SCHED_AUTO, SCHED_TWO_PASS = 0, 1
N_PARAMS = 12944960
GRAM_TOTAL = 610304
STYLE_CHANNELS = [64, 128, 256, 512, 512]

_STATUS = {0: "ok", 1: "invalid argument", 2: "shape", 3: "cuda", 4: "out of memory",
           5: "timeout", 6: "non-finite input", 7: "state"}


class NSTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libnst error %d (%s): %s" % (code, _STATUS.get(code, "?"), msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("w_style", ctypes.c_float * 5), ("lambda_c", ctypes.c_float),
                ("tiles_h", ctypes.c_int), ("tiles_w", ctypes.c_int),
                ("margin1", ctypes.c_int), ("margin2", ctypes.c_int),
                ("precision", ctypes.c_int), ("conv_engine", ctypes.c_int),
                ("max_batch_tiles", ctypes.c_int), ("workspace_limit_bytes", ctypes.c_longlong),
                ("w_mean", ctypes.c_float * 5), ("w_std", ctypes.c_float * 5),
                ("schedule", ctypes.c_int)]


def lib():
    """Load libnst.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libnst.so not built: run __graft_entry__.build() or "
                                   "python -m paper_2212_13459_gb300.build")
            L = ctypes.CDLL(LIB_PATH)
            vp, ip, dp, fp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
            ll = ctypes.c_longlong
            sig = {
                "nst_config_default": ([ctypes.POINTER(Config)], ip),
                "nst_create": ([ctypes.POINTER(vp), fp, ll, ctypes.POINTER(Config)], ip),
                "nst_destroy": ([vp], ip),
                "nst_style_targets": ([vp, fp, ip, ip, vp], ip),
                "nst_content_targets": ([vp, fp, ip, ip, vp], ip),
                "nst_loss_grad": ([vp, fp, ip, ip, fp, dp, vp], ip),
                "nst_loss_grad_host": ([vp, fp, ip, ip, fp, dp, vp], ip),
                "nst_get_stats": ([vp, dp, dp, vp], ip),
                "nst_get_style_grams": ([vp, dp, vp], ip),
                "nst_get_style_moments": ([vp, dp, dp, vp], ip),
                "nst_get_timing": ([vp, dp, vp], ip),
                "nst_set_timing": ([vp, ip], ip),
                "nst_sync_status": ([vp, vp], ip),
                "nst_set_schedule": ([vp, ip], ip),
                "nst_check_timeout_path": ([vp, ll, vp], ip),
                "nst_pass_info": ([vp, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)], ip),
                "nst_last_error": ([vp], ctypes.c_char_p),
                "nst_tile_plan": ([ip, ip, ip, ip, ip, vp], ip),
                "nst_lbfgs_create": ([ctypes.POINTER(vp), ll, ip], ip),
                "nst_lbfgs_create_ex": ([ctypes.POINTER(vp), ll, ip, ip], ip),
                "nst_lbfgs_destroy": ([vp], ip),
                "nst_lbfgs_step": ([vp, fp, fp, vp], ip),
                "nst_lbfgs_info": ([vp, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_longlong), vp], ip),
                "nst_upsample_init": ([fp, ip, ip, fp, ip, ip, vp], ip),
                "nst_downscale": ([fp, ip, ip, fp, ip, ip, vp], ip),
                "nst_version": ([], ctypes.c_char_p),
                "nst_conv3x3": ([ip, ip, ip, ip, ip, ip, ip, ip, vp, vp, ip, vp, vp, vp, ip, vp,
                                 vp, vp, vp], ip),
                "nst_gram": ([ip, vp, ll, ip, vp, vp], ip),
                "nst_gram_noalloc": ([ip, vp, ll, ip, vp, vp], ip),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != NST_OK:
        msg = lib().nst_last_error(ctx)
        raise NSTError(rc, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def default_config(**kw) -> Config:
    c = Config()
    _check(lib().nst_config_default(ctypes.byref(c)))
    for k, v in kw.items():
        if k in ("w_style", "w_mean", "w_std"):
            arr = getattr(c, k)
            for i in range(5):
                arr[i] = float(v[i])
        else:
            setattr(c, k, v)
    return c


def tile_plan(H, W, tiles_h, tiles_w, margin):
    out = (ctypes.c_int * (8 * tiles_h * tiles_w))()
    _check(lib().nst_tile_plan(H, W, tiles_h, tiles_w, margin, out))
    return np.array(out, dtype=np.int64).reshape(tiles_h * tiles_w, 8)


class Context:
    """Owns an nst_ctx: VGG-19 weights, style/content targets and the tile workspace."""

    def __init__(self, params_flat: np.ndarray, **cfg):
        p = np.ascontiguousarray(params_flat, dtype=np.float32)
        assert p.size == N_PARAMS, p.size
        self.cfg = default_config(**cfg)
        h = ctypes.c_void_p()
        _check(lib().nst_create(ctypes.byref(h), p.ctypes.data_as(ctypes.c_void_p), p.size,
                                ctypes.byref(self.cfg)))
        self.h = h
        self.H = self.W = None

    def close(self):
        if getattr(self, "h", None):
            lib().nst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def style_targets(self, v, stream=None):
        _check(lib().nst_style_targets(self.h, _ptr(v), v.shape[1], v.shape[2],
                                       _stream(stream)), self.h)

    def content_targets(self, u, stream=None):
        _check(lib().nst_content_targets(self.h, _ptr(u), u.shape[1], u.shape[2],
                                         _stream(stream)), self.h)
        self.H, self.W = u.shape[1], u.shape[2]

    def loss_grad(self, x, grad, loss=None, stream=None):
        _check(lib().nst_loss_grad(self.h, _ptr(x), x.shape[1], x.shape[2], _ptr(grad),
                                   _ptr(loss), _stream(stream)), self.h)

    def loss_grad_host(self, x_host: np.ndarray, grad_host: np.ndarray, stream=None):
        """x_host, grad_host: float32 C-contiguous host arrays (pinned for full speed)."""
        loss = ctypes.c_double(0.0)
        H, W = x_host.shape[1], x_host.shape[2]
        _check(lib().nst_loss_grad_host(self.h, ctypes.c_void_p(x_host.ctypes.data), H, W,
                                        ctypes.c_void_p(grad_host.ctypes.data),
                                        ctypes.cast(ctypes.byref(loss), ctypes.c_void_p),
                                        _stream(stream)), self.h)
        return loss.value

    def stats(self, stream=None, want_grams=True):
        parts = np.zeros(6)
        grams = np.zeros(GRAM_TOTAL) if want_grams else None
        _check(lib().nst_get_stats(self.h, ctypes.c_void_p(parts.ctypes.data),
                                   ctypes.c_void_p(grams.ctypes.data) if want_grams else None,
                                   _stream(stream)), self.h)
        return parts, (split_grams(grams) if want_grams else None)

    def style_grams(self, stream=None):
        g = np.zeros(GRAM_TOTAL)
        _check(lib().nst_get_style_grams(self.h, ctypes.c_void_p(g.ctypes.data),
                                         _stream(stream)), self.h)
        return split_grams(g)

    def style_moments(self, stream=None):
        m = np.zeros(sum(STYLE_CHANNELS))
        sd = np.zeros(sum(STYLE_CHANNELS))
        _check(lib().nst_get_style_moments(self.h, ctypes.c_void_p(m.ctypes.data),
                                           ctypes.c_void_p(sd.ctypes.data), _stream(stream)),
               self.h)
        out_m, out_s, o = [], [], 0
        for c in STYLE_CHANNELS:
            out_m.append(m[o:o + c].copy())
            out_s.append(sd[o:o + c].copy())
            o += c
        return out_m, out_s

    def set_timing(self, on=True):
        _check(lib().nst_set_timing(self.h, 1 if on else 0), self.h)

    def timing(self, stream=None):
        out = np.zeros(6)
        _check(lib().nst_get_timing(self.h, ctypes.c_void_p(out.ctypes.data), _stream(stream)),
               self.h)
        return {"conv_ms": out[0], "conv_flops": out[1], "gram_ms": out[2], "other_ms": out[3],
                "conv_launches": int(out[4]), "launches": int(out[5])}

    def sync_status(self, stream=None):
        return lib().nst_sync_status(self.h, _stream(stream))

    def check_timeout_path(self, limit_cycles=20_000_000, stream=None):
        """Run the bounded-wait failure path once (see nst_check_timeout_path)."""
        _check(lib().nst_check_timeout_path(self.h, int(limit_cycles), _stream(stream)), self.h)

    def set_schedule(self, schedule):
        _check(lib().nst_set_schedule(self.h, int(schedule)), self.h)

    def pass_info(self):
        """(Step-2 batches, resident) of the last loss_grad call."""
        b, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().nst_pass_info(self.h, ctypes.byref(b), ctypes.byref(r)), self.h)
        return b.value, bool(r.value)


def split_grams(flat):
    res, o = [], 0
    for c in STYLE_CHANNELS:
        res.append(flat[o:o + c * c].reshape(c, c).copy())
        o += c * c
    return res


class LBFGS:
    """Device-resident L-BFGS state (nst_lbfgs)."""

    HOST_HISTORY = 1

    def __init__(self, n, m, host_history=False):
        h = ctypes.c_void_p()
        _check(lib().nst_lbfgs_create_ex(ctypes.byref(h), int(n), int(m),
                                         self.HOST_HISTORY if host_history else 0))
        self.h = h
        self.n = n

    def step(self, x, g, stream=None):
        assert x.numel() == self.n and g.numel() == self.n
        _check(lib().nst_lbfgs_step(self.h, _ptr(x), _ptr(g), _stream(stream)))

    def info(self, stream=None):
        pairs = ctypes.c_int(0)
        iters = ctypes.c_longlong(0)
        _check(lib().nst_lbfgs_info(self.h, ctypes.byref(pairs), ctypes.byref(iters),
                                    _stream(stream)))
        return pairs.value, iters.value

    def close(self):
        if getattr(self, "h", None):
            lib().nst_lbfgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def downscale(x, out, stream=None):
    _check(lib().nst_downscale(_ptr(x), x.shape[1], x.shape[2], _ptr(out), out.shape[1],
                               out.shape[2], _stream(stream)))


def upsample_init(x_small, out, stream=None):
    _check(lib().nst_upsample_init(_ptr(x_small), x_small.shape[1], x_small.shape[2], _ptr(out),
                                   out.shape[1], out.shape[2], _stream(stream)))


def conv3x3(dtype, engine, inp, w, out, bias=None, mode=0, mask=None, in2=None, w2=None,
            geom=None, taps=9, stream=None):
    """One convolution layer (unit-test entry). inp [B,H,W,cin], w [cout,taps,cin],
    in2 [B,H,W,k2], w2 [cout,k2], out [B,H,W,cout], geom int32 [B,4] (device)."""
    B, H, W, cout = out.shape
    cin = inp.shape[3] if inp is not None else 0
    k2 = in2.shape[3] if in2 is not None else 0
    _check(lib().nst_conv3x3(dtype, engine, B, H, W, cin, cout, taps, _ptr(inp), _ptr(w), k2,
                             _ptr(in2), _ptr(w2), _ptr(bias), mode, _ptr(mask), _ptr(geom),
                             _ptr(out), _stream(stream)))


def _gram_args(V, G):
    """Marshalling checks shared by gram() and gram_noalloc(): V a contiguous 2-D float32 or
    bfloat16 matrix [npix, C] and G a contiguous C x C float64 matrix on the same device."""
    import torch
    if V.dim() != 2 or not V.is_contiguous() or V.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("V must be a contiguous 2-D float32 or bfloat16 tensor")
    C = V.shape[1]
    if G.dtype != torch.float64 or tuple(G.shape) != (C, C) or not G.is_contiguous():
        raise ValueError("G must be a contiguous %d x %d float64 tensor" % (C, C))
    if V.device != G.device or V.device.type != "cuda":
        raise ValueError("V and G must be on the same CUDA device")
    return PREC_BF16 if V.dtype == torch.bfloat16 else PREC_FP32


def gram(V, G, stream=None):
    """G (C x C float64, device) = V^T V for V [npix, C] (float32 or bfloat16, device)."""
    dtype = _gram_args(V, G)
    _check(lib().nst_gram(dtype, _ptr(V), V.shape[0], V.shape[1], _ptr(G), _stream(stream)))


def gram_noalloc(V, G, stream=None):
    """As gram(), through nst_gram_noalloc: no device allocation by the library (its partial sums
    use a fixed array in the library's device image; calls must not overlap on the GPU)."""
    dtype = _gram_args(V, G)
    _check(lib().nst_gram_noalloc(dtype, _ptr(V), V.shape[0], V.shape[1], _ptr(G),
                                  _stream(stream)))

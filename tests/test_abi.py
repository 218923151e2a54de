"""The C-ABI library loads on a machine without a GPU and exports every entry point that
include/nst.h declares; host-only calls (configuration, block partition, argument checks) work.
No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2212_13459_gb300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(nst_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    build.build()
    return native.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n


def test_config_default(L):
    c = native.default_config()
    assert c.tiles_h == 1 and c.margin1 == 80 and c.margin2 == 160
    assert c.precision == native.PREC_BF16
    assert abs(c.lambda_c - 1e-3) < 1e-9 and all(abs(w - 0.2) < 1e-7 for w in c.w_style)


@pytest.mark.parametrize("H,W,k,m", [(3024, 4032, 8, 160), (3024, 4032, 16, 160), (64, 64, 2, 160),
                                     (757, 1001, 3, 80), (6048, 8064, 16, 160), (128, 128, 4, 160)])
def test_tile_plan_is_a_partition(L, H, W, k, m):
    r = native.tile_plan(H, W, k, k, m)
    cover = np.zeros((H, W), np.int32)
    for iy0, iy1, ix0, ix1, ey0, ey1, ex0, ex1 in r:
        cover[iy0:iy1, ix0:ix1] += 1
        for v in (iy0, ix0):
            assert v % 16 == 0
        assert ey0 == max(0, iy0 - m) and ey1 == min(H, iy1 + m)
        assert ex0 == max(0, ix0 - m) and ex1 == min(W, ix1 + m)
        assert iy1 > iy0 and ix1 > ix0
    assert (cover == 1).all()


def test_tile_plan_balances_extended_blocks(L):
    r = native.tile_plan(3024, 4032, 8, 8, 160)
    eh = r[:, 5] - r[:, 4]
    ew = r[:, 7] - r[:, 6]
    assert eh.max() - eh.min() <= 32 and ew.max() - ew.min() <= 32


def test_argument_errors_without_gpu(L):
    c = native.default_config()
    assert L.nst_tile_plan(10, 10, 2, 2, 160, None) == native.NST_ERR_INVALID_ARG
    buf = (ctypes.c_int * 8 * 64)()
    assert L.nst_tile_plan(64, 64, 64, 64, 0, buf) == native.NST_ERR_SHAPE
    assert L.nst_tile_plan(64, 64, 2, 2, 10, buf) == native.NST_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.nst_create(ctypes.byref(h), None, 0, ctypes.byref(c)) == native.NST_ERR_INVALID_ARG
    p = np.zeros(10, np.float32)
    assert L.nst_create(ctypes.byref(h), p.ctypes.data, 10,
                        ctypes.byref(c)) == native.NST_ERR_INVALID_ARG
    assert L.nst_loss_grad(None, None, 64, 64, None, None, None) == native.NST_ERR_INVALID_ARG
    assert L.nst_lbfgs_create(ctypes.byref(h), 0, 10) == native.NST_ERR_INVALID_ARG
    assert L.nst_upsample_init(None, 1, 1, None, 2, 2, None) == native.NST_ERR_INVALID_ARG
    assert b"sm_103a" in L.nst_version()

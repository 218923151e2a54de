"""Bitwise reproducibility of nst_loss_grad.

Every reduction of the path runs in a fixed order (Gram partial tiles reduced by run index, the
loss parts summed by one thread, each owned pixel of dE/dx written once by one thread), so the
same image must give the same loss, the same Gram matrices and the same dE/dx bit for bit, in
either schedule, from the same context or from a fresh one. An evaluation of a different image
in between leaves other values in the workspace; the result must not depend on them (no read of
memory the evaluation did not write).
"""
import numpy as np
import pytest
import torch

from paper_2212_13459_gb300 import native, synth
from tests._gpu import LAMBDA_C, W_STYLE, seeded

pytestmark = pytest.mark.gpu

FORMS = {"bf16-tc": dict(precision=native.PREC_BF16, conv_engine=native.CONV_TC),
         "fp32": dict(precision=native.PREC_FP32, conv_engine=native.CONV_SIMT)}
SCHEDS = {"resident": native.SCHED_AUTO, "two_pass": native.SCHED_TWO_PASS}


def _ctx(params, u, v, form, sched, tiles):
    ctx = native.Context(synth.flat_params(params), w_style=W_STYLE, lambda_c=LAMBDA_C,
                         tiles_h=tiles[0], tiles_w=tiles[1], schedule=sched, **FORMS[form])
    ctx.style_targets(torch.from_numpy(v).cuda())
    ctx.content_targets(torch.from_numpy(u).cuda())
    return ctx


def _eval(ctx, x):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    g = torch.full_like(xt, 3.0)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.loss_grad(xt, g, loss)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    parts, grams = ctx.stats()
    return loss.item(), g.cpu().numpy(), parts, grams


def _same(a, b):
    assert a[0] == b[0], (a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])
    for s in range(5):
        assert np.array_equal(a[3][s], b[3][s]), s


@pytest.mark.parametrize("sched", list(SCHEDS))
@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("H,W,tiles", [(96, 128, (2, 2)), (208, 176, (3, 2))])
def test_loss_grad_is_bitwise_reproducible(form, sched, H, W, tiles):
    params, u, v, x = seeded(H, W, 6)
    other = np.ascontiguousarray(np.clip(1.0 - x, 0, 1))
    ctx = _ctx(params, u, v, form, SCHEDS[sched], tiles)
    first = _eval(ctx, x)
    _eval(ctx, other)          # different values left in every workspace buffer
    _same(first, _eval(ctx, x))
    ctx.close()
    fresh = _ctx(params, u, v, form, SCHEDS[sched], tiles)
    _same(first, _eval(fresh, x))
    fresh.close()


@pytest.mark.parametrize("form", list(FORMS))
def test_host_entry_matches_device_entry(form):
    """nst_loss_grad_host gives the device call's E and dE/dx bit for bit, with a page-locked
    gradient buffer (written by the last kernel over the host link) and with a pageable one
    (device buffer and copy); a stale value in either buffer must not survive."""
    params, u, v, x = seeded(208, 176, 8)
    ctx = _ctx(params, u, v, form, native.SCHED_TWO_PASS, (3, 2))
    ref = _eval(ctx, x)
    xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    for pinned in (True, False):
        gh = torch.full(x.shape, 7.0, dtype=torch.float32)
        if pinned:
            gh = gh.pin_memory()
        assert gh.is_pinned() == pinned
        E = ctx.loss_grad_host(xh.numpy(), gh.numpy())
        assert E == ref[0], (pinned, E, ref[0])
        assert np.array_equal(gh.numpy(), ref[1]), pinned
    ctx.close()

"""Failure detection without a GPU fault: a device-side wait that can never complete runs out
after its bound, the kernel returns, the host reads NST_ERR_TIMEOUT from the status word, and
the same context then evaluates normally."""
import numpy as np
import pytest
import torch

from paper_2212_13459_gb300 import native, synth
from tests._gpu import seeded

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    params, u, v, x = seeded(64, 64, 0)
    ctx = native.Context(synth.flat_params(params), tiles_h=2, tiles_w=2)
    ctx.style_targets(torch.from_numpy(v).cuda())
    ctx.content_targets(torch.from_numpy(u).cuda())
    ctx.check_timeout_path(20_000_000)          # about 10 ms of SM cycles
    assert ctx.sync_status() == native.NST_ERR_TIMEOUT
    assert ctx.sync_status() == native.NST_OK   # read and cleared
    xt = torch.from_numpy(x).cuda()
    g = torch.empty_like(xt)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.loss_grad(xt, g, loss)
    assert ctx.sync_status() == native.NST_OK
    assert np.isfinite(loss.item()) and torch.isfinite(g).all()
    ctx.close()

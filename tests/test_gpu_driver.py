"""The autograd wrapper, the L-BFGS loop and the multiscale driver on the GPU.

* NSTLossFunction: torch.autograd returns exactly the library's gradient, and the gradient
  matches central finite differences of the loss along smooth random directions (FP32 form):
  tightly for the ReLU1_1 term, within the loss's roughness for the full loss.
* style_transfer: L-BFGS with the localized gradient lowers the loss (SPST-style run, 128 x 128).
* schedules of Section 5.1 (600/300... and SPST-fast 600/200/66/30).
"""
import numpy as np
import pytest
import torch

from paper_2212_13459_gb300 import driver, native, synth
from tests._gpu import seeded

pytestmark = pytest.mark.gpu


def _ctx(H, W, seed, **cfg):
    params, u, v, x = seeded(H, W, seed)
    ctx = native.Context(synth.flat_params(params), **cfg)
    ctx.style_targets(torch.from_numpy(v).cuda())
    ctx.content_targets(torch.from_numpy(u).cuda())
    return ctx, torch.from_numpy(x).cuda()


def test_autograd_function_returns_library_gradient():
    ctx, x = _ctx(64, 64, 0, precision=native.PREC_FP32, tiles_h=2, tiles_w=2)
    xr = x.clone().requires_grad_(True)
    E = driver.nst_loss(xr, ctx)
    (3.0 * E).backward()
    g = torch.empty_like(x)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.loss_grad(x, g, loss)
    assert E.item() == loss.item()
    assert torch.equal(xr.grad, 3.0 * g)


def _directional_fd(ctx, x, h, seed, tol, n_dir=3):
    xr = x.clone().requires_grad_(True)
    driver.nst_loss(xr, ctx).backward()
    g = xr.grad.double()
    gen = torch.Generator(device="cuda").manual_seed(seed)
    H, W = x.shape[1:]
    for _ in range(n_dir):
        # smooth direction: a 12 x 12 random field upsampled by the library's bicubic kernel
        d = driver.resample(torch.randn(3, 12, 12, device="cuda", generator=gen), H, W)
        Ep = driver.nst_loss(x + h * d, ctx).item()
        Em = driver.nst_loss(x - h * d, ctx).item()
        fd = (Ep - Em) / (2 * h)
        gd = g * d.double()
        an = float(gd.sum())
        # relative to the projection's mass sum |g_i d_i| (robust when <g, d> cancels)
        assert abs(fd - an) <= tol * float(gd.abs().sum()), (fd, an)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_directional_fd_relu1_1_term(seed):
    """ReLU1_1 Gram term only: its kinks are those of 64 ReLUs at full resolution, so the
    central difference at h = 1e-3 matches the adjoint to 2e-3."""
    ctx, x = _ctx(96, 96, seed, precision=native.PREC_FP32, tiles_h=2, tiles_w=2,
                  w_style=(0.2, 0, 0, 0, 0), lambda_c=0.0)
    _directional_fd(ctx, x, 1e-3, seed, 2e-3)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_directional_fd_full_loss(seed):
    """Full loss: E is only piecewise smooth (ReLU / max-pool kinks are dense at the 1e-4 scale,
    where the exact gradient already moves by about 3%), so the central difference is the
    directional derivative averaged over [x - h d, x + h d]; 5e-2 bounds that average."""
    ctx, x = _ctx(96, 96, seed, precision=native.PREC_FP32, tiles_h=2, tiles_w=2)
    _directional_fd(ctx, x, 1e-4, seed, 5e-2)


def test_lbfgs_loop_lowers_the_loss():
    ctx, x = _ctx(128, 128, 1, precision=native.PREC_BF16, tiles_h=2, tiles_w=2)
    losses = []
    driver.style_transfer(ctx, x, 40, history=10, callback=lambda k, l: losses.append(l.item()))
    assert losses[-1] < 0.5 * losses[0]
    assert all(np.isfinite(losses))


def test_schedules():
    assert driver.spst_schedule(4) == [600, 300, 300, 300]
    assert driver.spst_fast_schedule(4) == [600, 200, 66, 30]


def test_multiscale_two_scales_runs():
    params, u, v, x = seeded(128, 160, 2)
    out = driver.multiscale(synth.flat_params(params), torch.from_numpy(u).cuda(),
                            torch.from_numpy(v).cuda(), n_scales=2, schedule=[10, 5],
                            precision=native.PREC_BF16)
    assert out.shape == (3, 128, 160) and torch.isfinite(out).all()


def test_scaled_sizes_follow_the_paper_shapes():
    assert driver.scaled(4226, 4) == 1057 and driver.scaled(5319, 4) == 1330
    assert driver.scaled(6048, 8) == 756 and driver.scaled(8064, 8) == 1008


def test_texture_synthesis_runs_and_lowers_style_loss():
    params, u, v, x = seeded(96, 96, 5)
    losses = []
    out = driver.texture_synthesis(synth.flat_params(params), torch.from_numpy(v).cuda(), 96, 96,
                                   n_scales=2, schedule=[15, 10], precision=native.PREC_BF16,
                                   callback=lambda s, k, l: losses.append((s, l.item())))
    assert out.shape == (3, 96, 96) and torch.isfinite(out).all()
    first = [l for s, l in losses if s == 1]
    assert first[-1] < first[0]

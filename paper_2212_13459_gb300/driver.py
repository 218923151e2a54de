"""Driver layer above the C ABI: a torch.autograd.Function for the loss, the L-BFGS loop of one
scale, and the coarse-to-fine multiscale loop of Algorithm 2. Every arithmetic step runs in
libnst's kernels (nst_loss_grad, nst_lbfgs_step, nst_upsample_init); this module only sequences
calls and holds device buffers.
"""
from __future__ import annotations

import torch

from . import native

# iterations per scale (Section 5.1): 600 at the first scale, 300 afterwards; SPST-fast divides
# by 3 from one scale to the next with a floor of 30 (Section 5.1, e.g. 600, 200, 66, 30)
def spst_schedule(n_scales):
    return [600] + [300] * (n_scales - 1)


def spst_fast_schedule(n_scales):
    it = [600]
    for _ in range(n_scales - 1):
        it.append(max(30, it[-1] // 3))
    return it


class NSTLossFunction(torch.autograd.Function):
    """E(x) of Algorithm 1 as a differentiable torch op: forward runs nst_loss_grad (loss and
    gradient together), backward returns grad_output * dE/dx."""

    @staticmethod
    def forward(fctx, x, nst_ctx):
        x = x.detach().contiguous()
        grad = torch.empty_like(x)
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        nst_ctx.loss_grad(x, grad, loss)
        fctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(fctx, grad_out):
        (grad,) = fctx.saved_tensors
        return (grad_out.to(grad.dtype) * grad), None


def nst_loss(x, nst_ctx):
    return NSTLossFunction.apply(x, nst_ctx)


def style_transfer(nst_ctx, x, iters, history=10, callback=None, host_history=False):
    """L-BFGS on E (Section 3.1) from x (updated in place), `iters` evaluations. host_history
    keeps the L-BFGS history in mapped host memory (Section 5.1, last scale)."""
    opt = native.LBFGS(x.numel(), history, host_history=host_history)
    grad = torch.empty_like(x)
    loss = torch.zeros(1, dtype=torch.float64, device=x.device)
    for k in range(iters):
        nst_ctx.loss_grad(x, grad, loss)
        if callback is not None:
            callback(k, loss)
        opt.step(x, grad)
    opt.close()
    return x


def resample(img, H, W):
    """Bicubic resampling of a 3 x h x w device image to 3 x H x W (nst_upsample_init)."""
    out = torch.empty((3, H, W), device=img.device, dtype=torch.float32)
    native.upsample_init(img.contiguous(), out)
    return out


def downscale(img, H, W):
    """Area-average downscaling of a 3 x h x w device image to 3 x H x W (nst_downscale)."""
    out = torch.empty((3, H, W), device=img.device, dtype=torch.float32)
    native.downscale(img.contiguous(), out)
    return out


def scaled(n, f):
    """n / f rounded half up (4226 / 4 -> 1057), at least 16 px."""
    return max(16, int(n / f + 0.5))


def multiscale(params_flat, u, v, n_scales, schedule=None, tiles_for=None, callback=None,
               host_history_last=False, x0=None, **cfg):
    """Algorithm 2: for s = 1..n, downscale (u, v) by 2^(n-s) (area averaging, sizes rounded);
    x = u at the first scale (or x0, a 3 x h x w image of the first scale's size), else the
    previous x upscaled by 2 (bicubic); then L-BFGS with localized gradients (history 100 at the
    first scale, 10 afterwards). tiles_for(H, W) -> (k_h, k_w) picks the block grid of a scale."""
    schedule = schedule or spst_schedule(n_scales)
    x = None
    for s in range(1, n_scales + 1):
        f = 2 ** (n_scales - s)
        Hs, Ws = scaled(u.shape[1], f), scaled(u.shape[2], f)
        Hv, Wv = scaled(v.shape[1], f), scaled(v.shape[2], f)
        us = u if f == 1 else downscale(u, Hs, Ws)
        vs = v if f == 1 else downscale(v, Hv, Wv)
        if x is None:
            x = (us if x0 is None else x0.to(device=us.device, dtype=torch.float32)).clone()
            if tuple(x.shape) != tuple(us.shape):
                raise ValueError("x0 must be 3 x %d x %d (the first scale)" % (Hs, Ws))
        else:
            x = resample(x, Hs, Ws)
        kh, kw = tiles_for(Hs, Ws) if tiles_for else (1, 1)
        ctx = native.Context(params_flat, tiles_h=kh, tiles_w=kw, **cfg)
        ctx.style_targets(vs)
        ctx.content_targets(us)
        style_transfer(ctx, x, schedule[s - 1], history=100 if s == 1 else 10,
                       callback=(lambda k, l, s=s: callback(s, k, l)) if callback else None,
                       host_history=host_history_last and s == n_scales)
        ctx.close()
    return x


def texture_synthesis(params_flat, v, H, W, n_scales, schedule=None, seed=0, tiles_for=None,
                      callback=None, x0=None, **cfg):
    """Texture synthesis (Section 6.2): the multiscale loop with no content term (lambda_c = 0),
    starting from white noise (uniform in [0, 1]) at the coarsest scale, or from the given x0 of
    that size; the output is H x W."""
    f = 2 ** (n_scales - 1)
    if x0 is None:
        g = torch.Generator(device=v.device).manual_seed(seed)
        x0 = torch.rand((3, scaled(H, f), scaled(W, f)), device=v.device, generator=g)
    # the content image only fixes the sizes of the scales (its term has weight 0)
    u = torch.zeros((3, H, W), device=v.device, dtype=torch.float32)
    cfg = dict(cfg)
    cfg["lambda_c"] = 0.0
    return multiscale(params_flat, u, v, n_scales, schedule=schedule, tiles_for=tiles_for,
                      callback=callback, x0=x0, **cfg)

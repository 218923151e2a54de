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


def style_transfer(nst_ctx, x, iters, history=10, callback=None):
    """L-BFGS on E (Section 3.1) from x (updated in place), `iters` evaluations."""
    opt = native.LBFGS(x.numel(), history)
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


def multiscale(params_flat, u, v, n_scales, schedule=None, tiles_for=None, callback=None,
               **cfg):
    """Algorithm 2: for s = 1..n, downscale (u, v) by 2^(n-s); x = u at the first scale, else
    the previous x upscaled by 2; then L-BFGS with localized gradients (history 100 at the first
    scale, 10 afterwards). tiles_for(H, W) -> (k_h, k_w) picks the block grid of a scale."""
    schedule = schedule or spst_schedule(n_scales)
    x = None
    for s in range(1, n_scales + 1):
        f = 2 ** (n_scales - s)
        Hs, Ws = max(16, round(u.shape[1] / f)), max(16, round(u.shape[2] / f))
        Hv, Wv = max(16, round(v.shape[1] / f)), max(16, round(v.shape[2] / f))
        us = u if f == 1 else resample(u, Hs, Ws)
        vs = v if f == 1 else resample(v, Hv, Wv)
        x = us.clone() if x is None else resample(x, Hs, Ws)
        kh, kw = tiles_for(Hs, Ws) if tiles_for else (1, 1)
        ctx = native.Context(params_flat, tiles_h=kh, tiles_w=kw, **cfg)
        ctx.style_targets(vs)
        ctx.content_targets(us)
        style_transfer(ctx, x, schedule[s - 1], history=100 if s == 1 else 10,
                       callback=(lambda k, l, s=s: callback(s, k, l)) if callback else None)
        ctx.close()
    return x

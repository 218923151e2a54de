"""Pin of the oracle's storage-precision mode (decisions taken in the evaluated form's precision).

The oracle in bfloat16 / float32 storage mode is compared with an independent route: PyTorch CPU
float64 autograd of the same network with explicit rounding hooks at the same points (rounded
activations with a straight-through backward, rounded masked gradients, rounded style residual).
Also checks that mode "f64" is the plain definition and that the modes actually differ.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from tests._common import LAMBDA_C, W_STYLE, problem, rel_l2

POOL_AFTER = {1, 3, 7, 11}


def _q(t, mode):
    if mode == "bf16":
        return t.float().bfloat16().double()
    return t.float().double()


class RoundAct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, mode):
        return _q(x, mode)

    @staticmethod
    def backward(ctx, g):
        return g, None


class RoundGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, mode):
        ctx.mode = mode
        return x.clone()

    @staticmethod
    def backward(ctx, g):
        return _q(g, ctx.mode), None


class GramLoss(torch.autograd.Function):
    """w ||V V^T / np - Gref||^2 with dE/dV = V q(4 w (G - Gref) / np)."""

    @staticmethod
    def forward(ctx, V, Gref, w, mode):
        npx = V.shape[1]
        G = V @ V.T / npx
        ctx.save_for_backward(V, _q(4.0 * w * (G - Gref) / npx, mode))
        return w * ((G - Gref) ** 2).sum()

    @staticmethod
    def backward(ctx, g):
        V, R = ctx.saved_tensors
        return g * (R @ V), None, None, None


class RoundPair(torch.autograd.Function):
    """The BF16 form's image: hi = bf16(x), lo = bf16(x - hi); straight-through backward."""

    @staticmethod
    def forward(ctx, x):
        hi = _q(x, "bf16")
        return hi + _q(x - hi, "bf16")

    @staticmethod
    def backward(ctx, g):
        return g


def torch_loss_storage(params, x, ct, grams, ws, lam, mode):
    h = (RoundPair.apply(x) if mode == "bf16" else x)[None]
    feats = {}
    for l, (w, b) in enumerate(params):
        W = torch.as_tensor(w, dtype=torch.float64)
        if mode == "bf16":
            W = _q(W, mode)
        pre = F.conv2d(h, W, torch.as_tensor(b, dtype=torch.float64), padding=1)
        h = RoundAct.apply(F.relu(RoundGrad.apply(pre, mode)), mode)
        feats[l] = h[0]
        if l in POOL_AFTER:
            h = RoundGrad.apply(F.max_pool2d(h, 2, 2), mode)
    E = torch.zeros((), dtype=torch.float64)
    for s, l in enumerate(oracle.STYLE_CONVS):
        V = feats[l].reshape(feats[l].shape[0], -1)
        E = E + GramLoss.apply(V, torch.as_tensor(grams[s]), float(ws[s]), mode)
    E = E + lam * ((feats[oracle.CONTENT_CONV] - torch.as_tensor(ct)) ** 2).sum()
    return E


@pytest.mark.parametrize("mode", ["bf16", "f32"])
def test_storage_mode_matches_torch_route(mode):
    params, P, u, v = problem(48, 64, seed=6)
    rng = np.random.default_rng(3)
    x = np.clip(u + 0.1 * rng.standard_normal(u.shape), 0, 1).astype(np.float32)
    with oracle.storage(mode):
        ct = oracle.content_target(P, u)
        Gv = oracle.style_grams(P, v)
        E, g, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    Et = torch_loss_storage(params, xt, ct, Gv, W_STYLE, LAMBDA_C, mode)
    (gt,) = torch.autograd.grad(Et, xt)
    assert abs(E - Et.item()) <= 1e-12 * abs(E)
    assert rel_l2(g, gt.numpy()) <= 1e-10


def test_storage_modes_differ_and_reset():
    params, P, u, v = problem(48, 64, seed=6)
    x = np.clip(0.5 * (u + v), 0, 1)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    E0, g0, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    with oracle.storage("bf16"):
        E2, g2, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    E1, g1, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    assert E1 == E0 and np.array_equal(g1, g0)          # the context manager restores f64
    assert rel_l2(g2, g0) > 1e-3                          # bf16 decisions move the gradient
    assert abs(E2 - E0) <= 1e-2 * abs(E0)                 # ... while the loss stays close

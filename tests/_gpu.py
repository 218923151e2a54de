"""Helpers for the GPU parity tests: run libnst and the FP64 oracle on the same seeded problem."""
import functools

import numpy as np
import torch

import oracle
from paper_2212_13459_gb300 import native, synth
from tests._common import LAMBDA_C, W_STYLE, rel_l2  # noqa: F401

# tolerances of the two forms of the path (relative L2 error of dE/dx and |dE|/|E|)
TOL_FP32 = 1e-5
TOL_BF16 = 2e-2


@functools.lru_cache(maxsize=None)
def seeded(H, W, seed, Hv=None, Wv=None, noise=0.1, bias_std=0.0):
    params = synth.vgg19_params(seed, bias_std=bias_std)
    u = synth.content_image(H, W, seed)
    v = synth.noise_style(Hv or H, Wv or W, seed)
    rng = np.random.default_rng(seed + 100)
    x = np.clip(u + noise * rng.standard_normal(u.shape), 0, 1).astype(np.float32)
    return params, u, v, x


# BF16 gradient bound of the full loss. The gradient of the VGG trunk is discontinuous at every
# ReLU / max-pool decision, and storing activations in BF16 (8-bit mantissa) perturbs every
# pre-activation by ~1e-3 relative, which flips the decisions that lie that close to a tie.
# Measured with the oracle alone (storage="bf16" against the plain FP64 definition): 0.23 at
# 64x64 and 0.27 at 128x128 for the full loss; 7e-3 for the ReLU1_1 term (no pooling decision on
# its path), 0.11 / 0.18 / 0.22 / 0.32 for the ReLU2_1 .. ReLU5_1 terms. The GPU's BF16 form is
# therefore held, case by case, to FLOOR_FACTOR times the deviation that BF16 storage causes in
# the oracle itself on the same input (never below TOL_BF16): see bf16_grad_bound().
FLOOR_FACTOR = 1.5
STYLE1_ONLY = (0.2, 0.0, 0.0, 0.0, 0.0)


@functools.lru_cache(maxsize=None)
def oracle_result(H, W, seed, Hv=None, Wv=None, noise=0.1, bias_std=0.0, storage="f64",
                  ws=None, lam=None):
    """FP64 oracle (ws a tuple: results are cached by argument). storage="f64" is the plain
    definition; "f32"/"bf16" round where that form of the path stores values (the FP32 form is
    compared with "f32", so that its ReLU masks and pooling argmaxes are decided in the same
    precision on both sides; "bf16" only serves to measure what BF16 storage alone does)."""
    params, u, v, x = seeded(H, W, seed, Hv, Wv, noise, bias_std)
    P = oracle.pack_params(params)
    ws = np.array(W_STYLE if ws is None else ws, np.float64)
    lam = LAMBDA_C if lam is None else lam
    with oracle.storage(storage):
        ct = oracle.content_target(P, u)
        Gv = oracle.style_grams(P, v)
        E, g, parts, Gx = oracle.loss_grad(P, x, ct, Gv, ws, lam)
    return E, g, parts, Gx, Gv


def bf16_grad_bound(H, W, seed, Hv=None, Wv=None, noise=0.1, bias_std=0.0, ws=None, lam=None):
    """Gradient bound of the BF16 form against the plain FP64 oracle on one problem: the relative
    deviation of the oracle's own BF16-storage evaluation from the definition (the error that
    rounding the stored values alone causes), times FLOOR_FACTOR, at least TOL_BF16. Computed
    from the oracle alone."""
    g64 = oracle_result(H, W, seed, Hv, Wv, noise, bias_std, "f64", ws, lam)[1]
    g16 = oracle_result(H, W, seed, Hv, Wv, noise, bias_std, "bf16", ws, lam)[1]
    return max(TOL_BF16, FLOOR_FACTOR * rel_l2(g16, g64))


def run_gpu(H, W, seed, Hv=None, Wv=None, noise=0.1, bias_std=0.0, x=None, **cfg):
    params, u, v, x0 = seeded(H, W, seed, Hv, Wv, noise, bias_std)
    x = x0 if x is None else x
    cfg.setdefault("w_style", W_STYLE)
    cfg.setdefault("lambda_c", LAMBDA_C)
    ctx = native.Context(synth.flat_params(params), **cfg)
    dev = torch.device("cuda:0")
    ut = torch.from_numpy(u).to(dev)
    vt = torch.from_numpy(v).to(dev)
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    ctx.style_targets(vt)
    ctx.content_targets(ut)
    grad = torch.empty_like(xt)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    ctx.loss_grad(xt, grad, loss)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    parts, grams = ctx.stats()
    out = dict(E=float(loss.item()), g=grad.cpu().numpy().astype(np.float64), parts=parts,
               grams=grams, style_grams=ctx.style_grams(), status=st, pass_info=ctx.pass_info())
    ctx.close()
    return out

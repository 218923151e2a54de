"""The ReLU1_1 Gram statistics of the tensor-core form, held tighter than the path tests hold them.

On the tensor cores the conv1_1 forward takes G^{ReLU1_1} = sum over owned pixels p of V_p V_p^T
(Eq. 4, accumulated block by block as in Algorithm 1, Step 1) from its own output tiles: every
patch of its grid is wholly owned or wholly outside the owned rectangle, and only the owned ones
enter the sum. A patch counted twice or missed would move the Gram by about one patch's share
(0.1-4 % at these sizes), which the 2e-2 bound of the path tests may not see. Against the oracle
in BF16 storage (the same BF16 activations up to FP32-vs-FP64 accumulation, which flips a BF16
rounding only within ~1e-7 of a rounding boundary) the difference is a few 1e-7; the bound here
is 1e-4. G^{ReLU2_1} (the separate Gram kernel) is checked the same way, with odd image sizes,
both schedules, Step 1 (two-pass), the style targets and the resident pass.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_2212_13459_gb300 import native, synth
from tests._gpu import LAMBDA_C, W_STYLE, rel_l2, seeded

pytestmark = pytest.mark.gpu

TOL = 1e-4
CASES = [(96, 128, (2, 2)), (208, 176, (3, 2)), (250, 333, (2, 3))]


@functools.lru_cache(maxsize=None)
def _oracle(H, W, seed):
    params, u, v, x = seeded(H, W, seed)
    P = oracle.pack_params(params)
    with oracle.storage("bf16"):
        ct = oracle.content_target(P, u)
        Gv = oracle.style_grams(P, v)
        _, _, _, Gx = oracle.loss_grad(P, x, ct, Gv, np.asarray(W_STYLE, np.float64), LAMBDA_C)
    return Gx, Gv


@pytest.mark.parametrize("sched", ["two_pass", "resident"])
@pytest.mark.parametrize("H,W,tiles", CASES)
def test_relu1_1_gram_fused_in_conv1_1(H, W, tiles, sched):
    seed = 9
    params, u, v, x = seeded(H, W, seed)
    s = native.SCHED_TWO_PASS if sched == "two_pass" else native.SCHED_AUTO
    ctx = native.Context(synth.flat_params(params), w_style=W_STYLE, lambda_c=LAMBDA_C,
                         tiles_h=tiles[0], tiles_w=tiles[1], schedule=s,
                         precision=native.PREC_BF16, conv_engine=native.CONV_TC)
    ctx.style_targets(torch.from_numpy(v).cuda())
    ctx.content_targets(torch.from_numpy(u).cuda())
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    g = torch.empty_like(xt)
    ctx.loss_grad(xt, g)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert ctx.pass_info()[1] == (sched == "resident")
    _, grams = ctx.stats()
    style = ctx.style_grams()
    ctx.close()
    Gx, Gv = _oracle(H, W, seed)
    errs = [rel_l2(grams[k], Gx[k]) for k in (0, 1)] + [rel_l2(style[k], Gv[k]) for k in (0, 1)]
    print("%dx%d %s: G(x) relu1_1 %.2e relu2_1 %.2e, G(v) relu1_1 %.2e relu2_1 %.2e"
          % (H, W, sched, *errs))
    assert max(errs) <= TOL, errs

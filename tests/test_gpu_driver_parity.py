"""Algorithm 2 and texture synthesis (Section 6.2) end to end, against the oracle's multiscale loop
(oracle/multiscale.py: area downscaling, bicubic upscaling, the untiled loss and the L-BFGS
two-loop recursion).

Two scales (64 x 64 then 128 x 128) of three L-BFGS iterations each, FP32 form on both sides
(the oracle with float32 storage, so ReLU and pooling decisions are taken in one precision). The
library's gradient agrees with that oracle to ~1e-6 per evaluation; three L-BFGS steps per scale
keep the iterates within 1e-4 (the pairs y = g_new - g_old are differences of gradients, so their
relative error is larger than the gradients'). Every evaluation's loss and the final image are
compared; a step, an initialisation or a resampling that differs from the oracle's would differ
at O(1).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import multiscale as orc_ms
from paper_2212_13459_gb300 import driver, native, synth
from tests._gpu import LAMBDA_C, W_STYLE, rel_l2, seeded

pytestmark = pytest.mark.gpu

FP32 = dict(precision=native.PREC_FP32, conv_engine=native.CONV_SIMT)
ITERS = [3, 3]
TOL = 1e-4


def _check(gpu_losses, out, ref_x, ref_losses):
    assert len(gpu_losses) == len(ref_losses)
    for (s, k, e), (so, ko, eo) in zip(gpu_losses, ref_losses):
        assert (s, k) == (so, ko)
        assert abs(e - eo) <= TOL * abs(eo), (s, k, e, eo)
    err = rel_l2(out.cpu().numpy(), ref_x)
    print("final x rel err %.3e" % err)
    assert err <= TOL


def test_multiscale_fp32_matches_oracle_loop():
    params, u, v, _ = seeded(128, 128, 2)
    P = oracle.pack_params(params)
    ref_x, ref_losses = orc_ms.multiscale(P, u, v, 2, ITERS, W_STYLE, LAMBDA_C,
                                          storage_mode="f32")
    losses = []
    out = driver.multiscale(synth.flat_params(params), torch.from_numpy(u).cuda(),
                            torch.from_numpy(v).cuda(), 2, schedule=ITERS, w_style=W_STYLE,
                            lambda_c=LAMBDA_C,
                            callback=lambda s, k, l: losses.append((s, k, l.item())), **FP32)
    _check(losses, out, ref_x, ref_losses)


def test_texture_synthesis_fp32_matches_oracle_loop():
    """Starts from white noise at the coarsest scale (drawn on the host, given to both sides)."""
    params, _, v, _ = seeded(128, 128, 3)
    P = oracle.pack_params(params)
    noise = np.random.default_rng(7).random((3, 64, 64)).astype(np.float32)
    ref_x, ref_losses = orc_ms.multiscale(P, np.zeros((3, 128, 128)), v, 2, ITERS, W_STYLE, 0.0,
                                          x0=noise, storage_mode="f32")
    losses = []
    out = driver.texture_synthesis(synth.flat_params(params), torch.from_numpy(v).cuda(), 128,
                                   128, 2, schedule=ITERS, x0=torch.from_numpy(noise).cuda(),
                                   w_style=W_STYLE,
                                   callback=lambda s, k, l: losses.append((s, k, l.item())),
                                   **FP32)
    _check(losses, out, ref_x, ref_losses)
    assert ref_losses[2][2] < ref_losses[0][2]   # the style loss falls at the first scale

"""GPU parity of the localized loss and image gradient (Algorithm 1) against the FP64 oracle.

Inputs are the seeded synthetic images of the paper's shapes; each case compares libnst's loss,
per-layer Gram matrices and dE/dx with the untiled FP64 definition, element by element.
FP32 form: relative error <= 1e-5; BF16 tensor-core form: <= 2e-2 (tolerances of the method's
precision plan).
"""
import numpy as np
import pytest
import torch

from paper_2212_13459_gb300 import native
from tests._gpu import TOL_BF16, TOL_FP32, oracle_result, rel_l2, run_gpu

pytestmark = pytest.mark.gpu

ENGINES = [("fp32", dict(precision=native.PREC_FP32, conv_engine=native.CONV_SIMT), TOL_FP32),
           ("bf16-simt", dict(precision=native.PREC_BF16, conv_engine=native.CONV_SIMT),
            TOL_BF16)]


def _compare(res, ref, tol, gram_tol=None):
    E, g, parts, Gx, Gv = ref
    assert res["status"] == 0
    for s in range(5):
        assert rel_l2(res["style_grams"][s], Gv[s]) <= (gram_tol or tol), ("G(v)", s)
        assert rel_l2(res["grams"][s], Gx[s]) <= (gram_tol or tol), ("G(x)", s)
    assert abs(res["E"] - E) <= tol * abs(E), (res["E"], E)
    assert abs(res["parts"][5] - parts[5]) <= tol * abs(parts[5]) + 1e-12
    assert rel_l2(res["g"], g) <= tol, rel_l2(res["g"], g)


@pytest.mark.parametrize("name,cfg,tol", ENGINES)
def test_config1_64x64_2x2_tiles(name, cfg, tol):
    ref = oracle_result(64, 64, 0)
    res = run_gpu(64, 64, 0, tiles_h=2, tiles_w=2, **cfg)
    _compare(res, ref, tol)


@pytest.mark.parametrize("name,cfg,tol", ENGINES)
def test_untiled_128(name, cfg, tol):
    ref = oracle_result(128, 128, 1)
    res = run_gpu(128, 128, 1, **cfg)
    _compare(res, ref, tol)


@pytest.mark.parametrize("name,cfg,tol", ENGINES)
def test_ragged_sizes_and_bias(name, cfg, tol):
    """Sizes that are not multiples of 16 (floor pooling drops trailing rows), non-zero biases,
    a style image of another size, 2 x 3 blocks."""
    ref = oracle_result(100, 76, 2, Hv=90, Wv=111, bias_std=0.01)
    res = run_gpu(100, 76, 2, Hv=90, Wv=111, bias_std=0.01, tiles_h=2, tiles_w=3, **cfg)
    _compare(res, ref, tol)


@pytest.mark.parametrize("name,cfg,tol", ENGINES)
def test_margins_cut_blocks(name, cfg, tol):
    """96 x 480 with 1 x 3 blocks: margins of 80 / 160 px really cut the image, so the result
    rests on the margin covering the receptive field (exactness of Algorithm 1)."""
    ref = oracle_result(96, 480, 3)
    res = run_gpu(96, 480, 3, tiles_h=1, tiles_w=3, **cfg)
    _compare(res, ref, tol)


@pytest.mark.parametrize("name,cfg,tol", ENGINES)
def test_batches_of_one_block(name, cfg, tol):
    ref = oracle_result(64, 64, 0)
    res = run_gpu(64, 64, 0, tiles_h=2, tiles_w=2, max_batch_tiles=1, **cfg)
    _compare(res, ref, tol)


@pytest.mark.parametrize("name,cfg,tol", ENGINES)
def test_identity_gives_exact_zero(name, cfg, tol):
    """x = u = v (the identity test of Section 7.2): E = 0 and dE/dx = 0 exactly, because every
    owned feature is computed from identical inputs in the same order in both passes."""
    from tests._gpu import seeded
    params, u, v, x = seeded(192, 160, 4)
    from paper_2212_13459_gb300 import synth
    ctx = native.Context(synth.flat_params(params), tiles_h=2, tiles_w=2, **cfg)
    ut = torch.from_numpy(u).cuda()
    ctx.style_targets(ut)
    ctx.content_targets(ut)
    g = torch.full_like(ut, 7.0)
    loss = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    ctx.loss_grad(ut, g, loss)
    torch.cuda.synchronize()
    assert loss.item() == 0.0
    assert torch.count_nonzero(g).item() == 0


def test_nonfinite_input_is_reported():
    from tests._gpu import seeded
    from paper_2212_13459_gb300 import synth
    params, u, v, x = seeded(64, 64, 0)
    ctx = native.Context(synth.flat_params(params), precision=native.PREC_FP32,
                         conv_engine=native.CONV_SIMT)
    ut = torch.from_numpy(u).cuda()
    ctx.style_targets(ut)
    ctx.content_targets(ut)
    xt = ut.clone()
    xt[1, 5, 7] = float("nan")
    g = torch.empty_like(xt)
    ctx.loss_grad(xt, g)
    assert ctx.sync_status() == native.NST_ERR_NONFINITE
    assert ctx.sync_status() == 0  # latched status is cleared once read


def test_call_order_and_shape_errors():
    from tests._gpu import seeded
    from paper_2212_13459_gb300 import synth
    params, u, v, x = seeded(64, 64, 0)
    ctx = native.Context(synth.flat_params(params), precision=native.PREC_FP32,
                         conv_engine=native.CONV_SIMT)
    ut = torch.from_numpy(u).cuda()
    g = torch.empty_like(ut)
    with pytest.raises(native.NSTError) as e:
        ctx.loss_grad(ut, g)
    assert e.value.code == native.NST_ERR_STATE
    ctx.style_targets(ut)
    ctx.content_targets(ut)
    small = ut[:, :32, :32].contiguous()
    with pytest.raises(native.NSTError) as e:
        ctx.loss_grad(small, torch.empty_like(small))
    assert e.value.code == native.NST_ERR_SHAPE
    tiny = ut[:, :8, :8].contiguous()
    with pytest.raises(native.NSTError) as e:
        ctx.style_targets(tiny)
    assert e.value.code == native.NST_ERR_SHAPE

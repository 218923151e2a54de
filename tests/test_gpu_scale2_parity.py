"""All-layer, full-loss parity at benchmark-sized blocks (Section 4.1, Algorithm 1).

1512 x 2016 with 4 x 4 blocks has blocks of the benchmark's size class (3024 x 4032 with 8 x 8
blocks: inner 336 x 464 .. 496 x 624 px, Step-2 buffer 672 x 784): inner 288 x 416 .. 464 x 592
px with margin 160, Step-1 / Step-2 buffers 512 x 624 and 624 x 752, so every layer runs on maps
of production size (up to 624 x 752 at full resolution, 39 x 47 at 1/16) with the patch shapes
the planner picks for them, at a size the oracle evaluates in about a minute. Inputs follow the multiscale scale-2 configuration: x = the oracle's own bicubic x2
upsampling of a synthetic 756 x 1008 previous-scale result (nothing here comes from the CUDA
path), content 1512 x 2016, style 1057 x 1330 stroke texture, all five Gram terms and the content
term. Compared element by element with the untiled FP64 oracle: every G^L(x) and G^L(v), E, the
content term and dE/dx, for the FP32 form (float32-storage oracle) and for the BF16 tensor-core
form (plain definition) in the printed two-pass schedule and in the resident one.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
from oracle import bicubic
from paper_2212_13459_gb300 import native, synth
from tests._gpu import FLOOR_FACTOR, LAMBDA_C, TOL_BF16, TOL_FP32, W_STYLE, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

H, W, HV, WV, SEED, K = 1512, 2016, 1057, 1330, 5, 4
# FP32 form, gradient: the kernels accumulate up to 4,608 products in FP32 (relative error
# ~sqrt(K) 2^-24, about 4e-6), the float32-storage oracle in FP64 with only its stored values
# rounded (~6e-8). A bicubic x2 upsampling of a smooth image puts adjacent pooling-window values
# within ~1e-4 of each other, so that accumulation noise flips on the order of 1e-3 of the
# pooling decisions, and each flip moves dE/dx locally: 1.85e-2 measured here (the continuous
# outputs, G^L, E and the content term, stay within 1e-5). Noisy inputs of the other parity
# cases have far fewer near-ties (1e-6 .. 5e-3 there).
FP32_SMOOTH_ALLOWANCE = 5e-2


@functools.lru_cache(maxsize=1)
def images():
    small = synth.scale2_result(H // 2, W // 2, SEED)
    x = bicubic.upsample(small.astype(np.float64), H, W).astype(np.float32)
    u = synth.content_image(H, W, SEED)
    v = synth.stroke_style(HV, WV, SEED)
    return np.ascontiguousarray(x), u, v


@functools.lru_cache(maxsize=None)
def oracle_eval(storage):
    x, u, v = images()
    P = oracle.pack_params(synth.vgg19_params(SEED))
    with oracle.storage(storage):
        ct = oracle.content_target(P, u)
        Gv = oracle.style_grams(P, v)
        E, g, parts, Gx = oracle.loss_grad(P, x, ct, Gv, np.asarray(W_STYLE, np.float64),
                                           LAMBDA_C)
    return E, g, parts, Gx, Gv


def gpu_eval(**cfg):
    x, u, v = images()
    ctx = native.Context(synth.flat_params(synth.vgg19_params(SEED)), tiles_h=K, tiles_w=K,
                         w_style=W_STYLE, lambda_c=LAMBDA_C, workspace_limit_bytes=int(64e9),
                         **cfg)
    ctx.style_targets(torch.from_numpy(v).cuda())
    ctx.content_targets(torch.from_numpy(u).cuda())
    xt = torch.from_numpy(x).cuda()
    g = torch.empty_like(xt)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.loss_grad(xt, g, loss)
    torch.cuda.synchronize()
    out = dict(status=ctx.sync_status(), E=loss.item(), g=g.cpu().numpy().astype(np.float64))
    out["parts"], out["grams"] = ctx.stats()
    out["style_grams"] = ctx.style_grams()
    out["pass_info"] = ctx.pass_info()
    ctx.close()
    return out


def compare(res, ref, tol, grad_tol):
    E, g, parts, Gx, Gv = ref
    assert res["status"] == 0
    for s in range(5):
        assert rel_l2(res["style_grams"][s], Gv[s]) <= tol, ("G(v)", s)
        assert rel_l2(res["grams"][s], Gx[s]) <= tol, ("G(x)", s)
    assert abs(res["E"] - E) <= tol * abs(E), (res["E"], E)
    assert abs(res["parts"][5] - parts[5]) <= tol * abs(parts[5])
    err = rel_l2(res["g"], g)
    assert err <= grad_tol, (err, grad_tol)
    return err


@pytest.mark.parametrize("sched", ["two_pass", "resident"])
def test_scale2_all_layers_fp32(sched):
    s = native.SCHED_TWO_PASS if sched == "two_pass" else native.SCHED_AUTO
    res = gpu_eval(precision=native.PREC_FP32, conv_engine=native.CONV_SIMT, schedule=s)
    assert res["pass_info"][1] == (sched == "resident")
    err = compare(res, oracle_eval("f32"), TOL_FP32, FP32_SMOOTH_ALLOWANCE)
    print("scale2 fp32 %s: grad rel err %.3e" % (sched, err))


@pytest.mark.parametrize("sched", ["two_pass", "resident"])
def test_scale2_all_layers_bf16_tensor_cores(sched):
    s = native.SCHED_TWO_PASS if sched == "two_pass" else native.SCHED_AUTO
    res = gpu_eval(precision=native.PREC_BF16, conv_engine=native.CONV_TC, schedule=s)
    assert res["pass_info"][1] == (sched == "resident")
    ref = oracle_eval("f64")
    floor = rel_l2(oracle_eval("bf16")[1], ref[1])
    bound = max(TOL_BF16, FLOOR_FACTOR * floor)
    err = compare(res, ref, TOL_BF16, bound)
    print("scale2 bf16 %s: grad rel err %.3e (oracle BF16-storage floor %.3e, bound %.3e)"
          % (sched, err, floor, bound))

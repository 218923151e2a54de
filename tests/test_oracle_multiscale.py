"""Pins of the multiscale oracle loop (oracle/multiscale.py) against Algorithm 2's text: the scale
sizes, the initialisation of each scale, and the targets of each scale. Small sizes (32 x 32,
16 x 16 at the coarse scale)."""
import numpy as np

import oracle
from oracle import area, bicubic
from oracle import multiscale as ms
from tests._common import LAMBDA_C, W_STYLE, problem


def test_scale_sizes_round_half_up():
    # 4226 x 5319 at scale 1 of 3 (factor 4) -> 1057 x 1330; 6048 / 8 -> 756; at least 16
    assert (ms.scaled(4226, 4), ms.scaled(5319, 4)) == (1057, 1330)
    assert (ms.scaled(6048, 8), ms.scaled(8064, 8)) == (756, 1008)
    assert ms.scaled(40, 4) == 16


def test_each_scale_starts_where_algorithm_2_says():
    """With no iteration at the first scale, the first evaluation of scale 2 is E at the bicubic
    upscaling of the area-downscaled content (x = u at scale 1, then "upscale x by 2"), with the
    targets of the full-size u and v; the first evaluation of scale 1 is E at the downscaled u
    with the downscaled targets."""
    params, P, u, v = problem(32, 32, 0)
    x, losses = ms.multiscale(P, u, v, 2, [1, 1], W_STYLE, LAMBDA_C)
    u1, v1 = area.downscale(u, 16, 16), area.downscale(v, 16, 16)
    E1 = oracle.loss_grad(P, u1, oracle.content_target(P, u1), oracle.style_grams(P, v1),
                          W_STYLE, LAMBDA_C)[0]
    assert losses[0][:2] == (1, 0) and abs(losses[0][2] - E1) <= 1e-12 * abs(E1)
    _, losses0 = ms.multiscale(P, u, v, 2, [0, 1], W_STYLE, LAMBDA_C)
    x2 = bicubic.upsample(u1, 32, 32)
    E2 = oracle.loss_grad(P, x2, oracle.content_target(P, u), oracle.style_grams(P, v),
                          W_STYLE, LAMBDA_C)[0]
    assert losses0[0][:2] == (2, 0) and abs(losses0[0][2] - E2) <= 1e-12 * abs(E2)


def test_given_start_replaces_the_content_at_the_first_scale():
    params, P, u, v = problem(32, 32, 1)
    noise = np.random.default_rng(3).random((3, 16, 16))
    _, losses = ms.multiscale(P, np.zeros((3, 32, 32)), v, 2, [1, 0], W_STYLE, 0.0, x0=noise)
    v1 = area.downscale(v, 16, 16)
    E = oracle.loss_grad(P, noise, np.zeros((512, 2, 2)), oracle.style_grams(P, v1), W_STYLE,
                         0.0)[0]
    assert abs(losses[0][2] - E) <= 1e-12 * abs(E)

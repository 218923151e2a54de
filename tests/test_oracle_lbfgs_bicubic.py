"""Pins of the L-BFGS and bicubic oracles against independent definitions.

* L-BFGS two-loop recursion (Nocedal 1980, the optimizer of Section 3.1) equals the explicit dense
  inverse-BFGS matrix built from the same pairs; on a strictly convex quadratic the driver reaches
  the closed-form minimiser.
* Bicubic x2 upscaling (initialisation of Algorithm 2) equals PyTorch's own bicubic interpolation
  (align_corners=False), reproduces constants, and commutes with mirroring.
"""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import bicubic, lbfgs


def test_two_loop_equals_dense_inverse_bfgs():
    rng = np.random.default_rng(0)
    n, m = 40, 7
    A = rng.standard_normal((n, n))
    Q = A @ A.T + n * np.eye(n)                 # SPD Hessian: y = Q s keeps y^T s > 0
    S = [rng.standard_normal(n) for _ in range(m)]
    Y = [Q @ s for s in S]
    gamma = float(S[-1] @ Y[-1] / (Y[-1] @ Y[-1]))
    g = rng.standard_normal(n)
    d = lbfgs.two_loop(g, S, Y, gamma)
    Hd = lbfgs.dense_inverse_bfgs(S, Y, gamma, n)
    assert np.allclose(d, -Hd @ g, rtol=1e-12, atol=1e-13 * np.abs(Hd @ g).max())


def test_two_loop_catches_swapped_pairs():
    """Reversing the pair order (a plausible indexing slip) changes the result."""
    rng = np.random.default_rng(1)
    n, m = 20, 5
    A = rng.standard_normal((n, n))
    Q = A @ A.T + n * np.eye(n)
    S = [rng.standard_normal(n) for _ in range(m)]
    Y = [Q @ s for s in S]
    g = rng.standard_normal(n)
    d = lbfgs.two_loop(g, S, Y, 1.0)
    d_rev = lbfgs.two_loop(g, S[::-1], Y[::-1], 1.0)
    assert np.abs(d - d_rev).max() > 1e-6 * np.abs(d).max()


def test_lbfgs_minimises_convex_quadratic():
    rng = np.random.default_rng(2)
    n = 30
    A = rng.standard_normal((n, n))
    Q = A @ A.T / n + np.eye(n)
    b = rng.standard_normal(n)
    xstar = np.linalg.solve(Q, b)
    x = np.zeros(n)
    opt = lbfgs.LBFGS(n, m=10)
    for _ in range(200):
        g = Q @ x - b
        if np.linalg.norm(g) < 1e-12:
            break
        opt.step(x, g)
    assert np.linalg.norm(x - xstar) <= 1e-8 * np.linalg.norm(xstar)


def test_first_step_length():
    """First iteration: t = min(1, 1/||g||_1) along -g (H0 = I with no pairs)."""
    g = np.array([3.0, -1.0, 0.5])
    x = np.zeros(3)
    lbfgs.LBFGS(3, 10).step(x, g)
    assert np.allclose(x, -g / 4.5, rtol=1e-15)


def test_bicubic_matches_torch():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, size=(3, 13, 17))
    for (H, W) in [(26, 34), (27, 35), (13, 17), (40, 20)]:
        ref = F.interpolate(torch.tensor(x)[None], size=(H, W), mode="bicubic",
                            align_corners=False)[0].numpy()
        out = bicubic.upsample(x, H, W)
        assert np.abs(out - ref).max() <= 1e-12


def test_bicubic_constant_and_mirror():
    x = np.full((3, 9, 11), 0.37)
    assert np.abs(bicubic.upsample(x, 18, 22) - 0.37).max() <= 1e-15
    # half-pixel centres make the operator commute with mirroring the image
    rng = np.random.default_rng(4)
    y = rng.uniform(0, 1, size=(3, 7, 10))
    up = bicubic.upsample(y, 14, 20)
    upm = bicubic.upsample(y[:, ::-1, ::-1], 14, 20)
    assert np.abs(up[:, ::-1, ::-1] - upm).max() <= 1e-14


def test_area_downscale_matches_torch_adaptive_pool():
    from oracle import area
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, size=(3, 37, 53))
    for (H, W) in [(18, 26), (37, 53), (9, 13), (19, 27), (5, 40)]:
        ref = F.adaptive_avg_pool2d(torch.tensor(x)[None], (H, W))[0].numpy()
        assert np.abs(area.downscale(x, H, W) - ref).max() <= 1e-13


def test_area_downscale_integer_factor_is_box_mean():
    from oracle import area
    rng = np.random.default_rng(9)
    x = rng.uniform(0, 1, size=(3, 16, 24))
    y = area.downscale(x, 4, 6)
    ref = x.reshape(3, 4, 4, 6, 4).mean(axis=(2, 4))
    assert np.abs(y - ref).max() <= 1e-15
    assert abs(y.mean() - x.mean()) <= 1e-14          # mean preserved for exact factors

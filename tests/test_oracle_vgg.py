"""Pins of the FP64 oracle's network-level loss and gradient.

* an independent library route: PyTorch CPU float64 autograd of the same untiled loss;
* central finite differences on 16 random pixels of the 64 x 64 problem (2x2-tile configuration);
* invariants: Gram symmetric PSD with diag = mean of squares, positive 1-homogeneity with zero
  biases, zero loss and zero gradient at x = u = v (the identity test, Section 7.2);
* exactness of Algorithm 1: block-wise statistics and gradient equal the untiled ones once the
  margin covers the receptive field, and visibly differ without margin (Section 4.2, Fig. 3).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from tests._common import LAMBDA_C, W_STYLE, problem, rel_l2

POOL_AFTER = {1, 3, 7, 11}


def torch_loss(params, x, ct, grams, w_style, lam):
    """The transfer loss written with PyTorch's own conv2d / max_pool2d (float64, CPU)."""
    h = x[None]
    feats = {}
    for l, (w, b) in enumerate(params):
        h = F.relu(F.conv2d(h, torch.as_tensor(w, dtype=torch.float64),
                            torch.as_tensor(b, dtype=torch.float64), padding=1))
        feats[l] = h[0]
        if l in POOL_AFTER:
            h = F.max_pool2d(h, 2, 2)
    E = torch.zeros((), dtype=torch.float64)
    for s, l in enumerate(oracle.STYLE_CONVS):
        V = feats[l].reshape(feats[l].shape[0], -1)
        G = V @ V.T / V.shape[1]
        E = E + w_style[s] * ((G - torch.as_tensor(grams[s])) ** 2).sum()
    E = E + lam * ((feats[oracle.CONTENT_CONV] - torch.as_tensor(ct)) ** 2).sum()
    return E


@pytest.fixture(scope="module")
def cfg1():
    params, P, u, v = problem(64, 64, seed=0)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    rng = np.random.default_rng(100)
    x = np.clip(u + 0.1 * rng.standard_normal(u.shape), 0, 1)
    return params, P, u, v, ct, Gv, x


def test_matches_torch_autograd_float64(cfg1):
    params, P, u, v, ct, Gv, x = cfg1
    E, g, parts, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    Et = torch_loss(params, xt, ct, Gv, W_STYLE, LAMBDA_C)
    (gt,) = torch.autograd.grad(Et, xt)
    assert abs(E - Et.item()) <= 1e-12 * abs(E)
    assert rel_l2(g, gt.numpy()) <= 1e-12
    assert parts[5] > 0 and all(p > 0 for p in parts[:5])


def test_matches_torch_autograd_with_biases():
    params, P, u, v = problem(48, 40, seed=5, bias_std=0.01)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    x = 0.5 * (u + v)
    E, g, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    Et = torch_loss(params, xt, ct, Gv, W_STYLE, LAMBDA_C)
    (gt,) = torch.autograd.grad(Et, xt)
    assert abs(E - Et.item()) <= 1e-12 * abs(E)
    assert rel_l2(g, gt.numpy()) <= 1e-12


def test_finite_differences_16_pixels(cfg1):
    params, P, u, v, ct, Gv, x = cfg1
    E0, g, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    rng = np.random.default_rng(7)
    idx = [(int(rng.integers(3)), int(rng.integers(64)), int(rng.integers(64))) for _ in range(16)]

    def E_at(xx):
        return oracle.loss_grad(P, xx, ct, Gv, W_STYLE, LAMBDA_C, want_grad=False)[0]

    ok = 0
    for (c, i, j) in idx:
        est = []
        for h in (2e-5, 1e-5):
            xp = x.copy(); xp[c, i, j] += h
            xm = x.copy(); xm[c, i, j] -= h
            est.append((E_at(xp) - E_at(xm)) / (2 * h))
        scale = max(abs(g[c, i, j]), 1e-3 * np.abs(g).max())
        # a ReLU or pooling kink inside [x-h, x+h] makes the two step sizes disagree: skip those
        if abs(est[0] - est[1]) > 1e-5 * scale:
            continue
        # FP64 rounding of E (~1e-14 relative, E ~ 700) over 2h = 2e-5 bounds the FD noise
        assert abs(est[1] - g[c, i, j]) <= 5e-6 * scale, (c, i, j, est, g[c, i, j])
        ok += 1
    assert ok >= 12


def test_gram_invariants(cfg1):
    params, P, u, v, ct, Gv, x = cfg1
    for s, l in enumerate(oracle.STYLE_CONVS):
        V = oracle.features(P, x, l).reshape(oracle.CONV_COUT[l], -1)
        G = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C, want_grad=False)[3][s]
        assert np.array_equal(G, G.T)
        ev = np.linalg.eigvalsh(G)
        assert ev.min() >= -1e-12 * np.abs(ev).max()
        assert np.allclose(np.diag(G), (V * V).mean(axis=1), rtol=1e-12, atol=0)
        # the Gram against an independent formula: numpy matmul on the oracle's own features
        assert np.allclose(G, V @ V.T / V.shape[1], rtol=1e-12, atol=1e-15)


def test_positive_homogeneity_zero_bias(cfg1):
    params, P, u, v, ct, Gv, x = cfg1
    c = 1.7
    for l in (0, 4, 9, 12):
        a = oracle.features(P, x, l)
        b = oracle.features(P, c * x, l)
        assert np.abs(b - c * a).max() <= 1e-12 * np.abs(c * a).max()


def test_identity_zero_loss_and_gradient(cfg1):
    params, P, u, v, ct, Gv, x = cfg1
    ct_u = oracle.content_target(P, u)
    G_u = oracle.style_grams(P, u)
    E, g, parts, _ = oracle.loss_grad(P, u, ct_u, G_u, W_STYLE, LAMBDA_C)
    assert E == 0.0 and not np.any(g)


def test_content_only_zero_at_content(cfg1):
    params, P, u, v, ct, Gv, x = cfg1
    E, g, parts, _ = oracle.loss_grad(P, u, ct, Gv, np.zeros(5), LAMBDA_C)
    assert E == 0.0 and not np.any(g)


def test_style_targets_equal_loss_statistics(cfg1):
    """G^L(v) from the target routine equals G^L(x) reported by the loss routine at x = v."""
    params, P, u, v, ct, Gv, x = cfg1
    _, _, _, Gx = oracle.loss_grad(P, v, ct, Gv, W_STYLE, LAMBDA_C, want_grad=False)
    for a, b in zip(Gv, Gx):
        assert np.array_equal(a, b)


def test_plan_is_a_partition():
    for L, k in [(64, 2), (100, 3), (3024, 8), (4032, 16), (757, 5)]:
        b = oracle.plan_1d(L, k)
        assert b[0] == 0 and b[-1] == L
        assert all(b[i] < b[i + 1] for i in range(k))
        assert all(bi % 16 == 0 for bi in b[1:-1])


def test_step1_statistics_block_independent():
    """Step 1 of Algorithm 1 with margin 80 >= 70 (the ReLU5_1 receptive-field reach) gives the
    untiled Gram matrices; with margin 0 it does not."""
    params, P, u, v = problem(96, 224, seed=2)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    _, _, _, G0 = oracle.loss_grad(P, u, ct, Gv, W_STYLE, LAMBDA_C, want_grad=False)
    _, _, _, G1 = oracle.loss_grad_tiled(P, u, ct, Gv, W_STYLE, LAMBDA_C, (1, 2), (80, 160),
                                         want_grad=False)
    for a, b in zip(G1, G0):
        assert rel_l2(a, b) <= 1e-13
    _, _, _, Gz = oracle.loss_grad_tiled(P, u, ct, Gv, W_STYLE, LAMBDA_C, (1, 2), (0, 0),
                                         want_grad=False)
    assert rel_l2(Gz[4], G0[4]) > 1e-3


@pytest.mark.slow
def test_algorithm1_gradient_exact_with_margin():
    """64 x 416 image, 1 x 2 blocks (inner boundary at x = 208). The gradient at an image pixel
    reaches 155 px (twice the ReLU5_1 receptive-field half-width), so margin 160 is exact, margin
    144 is not, and margin 0 leaves seams (the paper's Fig. 3 reports 5.23e-1 for its images)."""
    params, P, u, v = problem(64, 416, seed=3)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    rng = np.random.default_rng(9)
    x = np.clip(u + 0.05 * rng.standard_normal(u.shape), 0, 1)
    E0, g0, p0, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    E1, g1, p1, _ = oracle.loss_grad_tiled(P, x, ct, Gv, W_STYLE, LAMBDA_C, (1, 2), (80, 160))
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert rel_l2(g1, g0) <= 1e-12
    _, g2, _, _ = oracle.loss_grad_tiled(P, x, ct, Gv, W_STYLE, LAMBDA_C, (1, 2), (80, 144))
    assert rel_l2(g2, g0) > 1e-9
    _, g3, _, _ = oracle.loss_grad_tiled(P, x, ct, Gv, W_STYLE, LAMBDA_C, (1, 2), (0, 0))
    assert rel_l2(g3, g0) > 1e-2


def test_strip_gram_and_single_block_step2_agree_with_untiled():
    """The helpers used by the full-size sampled GPU checks: the strip-wise ReLU1_1 Gram equals
    the untiled one, and Step 2 on a 5 x 5 block (margin 2 = the ReLU1_1 term's reach) gives
    the untiled gradient of the ReLU1_1 term at the block centre."""
    params, P, u, v = problem(64, 96, seed=11)
    ws = np.array([0.2, 0, 0, 0, 0])
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    E, g, _, Gx = oracle.loss_grad(P, u, ct, Gv, ws, 0.0)
    G1 = oracle.relu11_gram(P, u, strip=10)
    assert np.allclose(G1, Gx[0], rtol=1e-12, atol=1e-15)
    zeros = [np.zeros((c, c)) for c in oracle.STYLE_CHANNELS]
    Gglob = [G1] + zeros[1:]
    npg = [64 * 96, 1, 1, 1, 1]
    for (py, px) in [(30, 40), (2, 5), (63, 95), (10, 0)]:
        y0, y1, x0, x1 = max(0, py - 2), min(64, py + 3), max(0, px - 2), min(96, px + 3)
        d = oracle.block_style_grad(P, u[:, y0:y1, x0:x1], Gglob, Gv, npg, ws)
        assert np.allclose(d[:, py - y0, px - x0], g[:, py, px], rtol=1e-10,
                           atol=1e-12 * np.abs(g).max())

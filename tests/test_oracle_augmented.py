"""Pins of the oracle's augmented style loss (Eq. 5; Table 1 rows 3-4; std from diag(G) - mean^2
as in Algorithm 1, Step 1).

* Table 1 rows 3-4 against central finite differences (np = 7, nc = 5);
* the network-level loss and gradient against PyTorch float64 autograd, which takes std with
  torch.var (population) instead of diag(G) - mean^2 (an independent route);
* Algorithm 1 with the moments accumulated block by block equals the untiled evaluation;
* the identity test (x = u = v gives E = 0 and dE/dx = 0).
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from tests._common import LAMBDA_C, W_STYLE, problem, rel_l2

POOL_AFTER = {1, 3, 7, 11}
W_MEAN = np.array([0.5, 0.3, 0.2, 0.1, 0.1])
W_STD = np.array([0.4, 0.3, 0.2, 0.2, 0.1])


def _fd(f, V, h=1e-6):
    g = np.zeros_like(V)
    for idx in np.ndindex(V.shape):
        Vp, Vm = V.copy(), V.copy()
        Vp[idx] += h
        Vm[idx] -= h
        g[idx] = (f(Vp) - f(Vm)) / (2 * h)
    return g


def test_table1_mean_row():
    rng = np.random.default_rng(21)
    V = rng.standard_normal((7, 5))
    mu = rng.standard_normal(5)
    E, g = oracle.table1_mean(V, mu, 0.7)
    f = lambda X: 0.7 * float(np.sum((X.mean(axis=0) - mu) ** 2))
    assert abs(E - f(V)) <= 1e-12 * abs(E)
    fd = _fd(f, V)
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_table1_std_row():
    rng = np.random.default_rng(22)
    V = rng.standard_normal((7, 5))
    sigma = np.abs(rng.standard_normal(5))
    E, g = oracle.table1_std(V, sigma, 0.9)
    f = lambda X: 0.9 * float(np.sum((X.std(axis=0) - sigma) ** 2))   # numpy: population std
    assert abs(E - f(V)) <= 1e-12 * abs(E)
    fd = _fd(f, V)
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_table1_std_constant_channel_has_zero_gradient():
    V = np.ones((7, 3))
    V[:, 1] = np.arange(7)
    E, g = oracle.table1_std(V, np.array([0.5, 0.5, 0.5]), 1.0)
    assert np.all(np.isfinite(g)) and not np.any(g[:, 0]) and not np.any(g[:, 2])


def torch_aug_loss(params, x, ct, grams, means, stds, ws, wm, wsd, lam):
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
        E = E + ws[s] * ((G - torch.as_tensor(grams[s])) ** 2).sum()
        m = V.mean(dim=1)
        var = V.var(dim=1, unbiased=False)
        pos = var > 0
        sd = torch.where(pos, torch.sqrt(torch.where(pos, var, torch.ones_like(var))), 0 * var)
        E = E + wm[s] * ((m - torch.as_tensor(means[s])) ** 2).sum()
        E = E + wsd[s] * ((sd - torch.as_tensor(stds[s])) ** 2).sum()
    E = E + lam * ((feats[oracle.CONTENT_CONV] - torch.as_tensor(ct)) ** 2).sum()
    return E


@pytest.fixture(scope="module")
def aug_problem():
    params, P, u, v = problem(64, 80, seed=7)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    mv, sv = oracle.style_moments(P, v)
    rng = np.random.default_rng(5)
    x = np.clip(u + 0.1 * rng.standard_normal(u.shape), 0, 1)
    return params, P, u, v, ct, Gv, mv, sv, x


def test_style_moments_against_numpy(aug_problem):
    params, P, u, v, ct, Gv, mv, sv, x = aug_problem
    for s, l in enumerate(oracle.STYLE_CONVS):
        V = oracle.features(P, v, l).reshape(oracle.CONV_COUT[l], -1)
        assert np.allclose(mv[s], V.mean(axis=1), rtol=1e-12, atol=1e-15)
        assert np.allclose(sv[s], V.std(axis=1), rtol=1e-9, atol=1e-9)


def test_augmented_loss_matches_torch_autograd(aug_problem):
    params, P, u, v, ct, Gv, mv, sv, x = aug_problem
    E, g, parts, _ = oracle.loss_grad_aug(P, x, ct, Gv, mv, sv, W_STYLE, W_MEAN, W_STD, LAMBDA_C)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    Et = torch_aug_loss(params, xt, ct, Gv, mv, sv, W_STYLE, W_MEAN, W_STD, LAMBDA_C)
    (gt,) = torch.autograd.grad(Et, xt)
    assert abs(E - Et.item()) <= 1e-12 * abs(E)
    assert rel_l2(g, gt.numpy()) <= 1e-11
    # the moment terms actually contribute
    E0, g0, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    assert E > E0 and rel_l2(g, g0) > 1e-3


def test_augmented_zero_weights_is_plain_gram_loss(aug_problem):
    params, P, u, v, ct, Gv, mv, sv, x = aug_problem
    E, g, _, _ = oracle.loss_grad_aug(P, x, ct, Gv, mv, sv, W_STYLE, np.zeros(5), np.zeros(5),
                                      LAMBDA_C)
    E0, g0, _, _ = oracle.loss_grad(P, x, ct, Gv, W_STYLE, LAMBDA_C)
    assert E == E0 and np.array_equal(g, g0)


def test_augmented_identity(aug_problem):
    params, P, u, v, ct, Gv, mv, sv, x = aug_problem
    ctu = oracle.content_target(P, u)
    Gu = oracle.style_grams(P, u)
    mu, su = oracle.style_moments(P, u)
    E, g, _, _ = oracle.loss_grad_aug(P, u, ctu, Gu, mu, su, W_STYLE, W_MEAN, W_STD, LAMBDA_C)
    assert abs(E) <= 1e-24 and np.max(np.abs(g)) <= 1e-12


def test_augmented_algorithm1_statistics_block_independent():
    """Step 1 with margin 80 gives the untiled mean/std terms (the loss is exact)."""
    params, P, u, v = problem(96, 224, seed=8)
    ct = oracle.content_target(P, u)
    Gv = oracle.style_grams(P, v)
    mv, sv = oracle.style_moments(P, v)
    E0, _, p0, _ = oracle.loss_grad_aug(P, u, ct, Gv, mv, sv, W_STYLE, W_MEAN, W_STD, LAMBDA_C,
                                        want_grad=False)
    E1, _, p1, _ = oracle.loss_grad_aug(P, u, ct, Gv, mv, sv, W_STYLE, W_MEAN, W_STD, LAMBDA_C,
                                        want_grad=False, tiles=(1, 2), margins=(80, 160))
    assert abs(E1 - E0) <= 1e-12 * abs(E0)
    assert np.allclose(p1, p0, rtol=1e-11, atol=1e-14)

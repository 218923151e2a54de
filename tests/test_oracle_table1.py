"""Pins of the oracle's feature-level gradients (Table 1, rows 1-2) by central finite differences.

Random V with np = 7 feature pixels and nc = 5 channels, FP64; h = 1e-6.
"""
import numpy as np

import oracle


def _fd(f, V, h=1e-6):
    g = np.zeros_like(V)
    for idx in np.ndindex(V.shape):
        Vp = V.copy()
        Vm = V.copy()
        Vp[idx] += h
        Vm[idx] -= h
        g[idx] = (f(Vp) - f(Vm)) / (2 * h)
    return g


def test_gram_row_matches_finite_differences():
    rng = np.random.default_rng(11)
    V = rng.standard_normal((7, 5))
    A = rng.standard_normal((9, 5))
    Gref = A.T @ A / 9.0
    w = 0.37
    E, g = oracle.table1_gram(V, Gref, w)
    # the Gram loss written independently: ||V^T V / np - Gref||_F^2 * w
    f = lambda X: w * float(np.sum((X.T @ X / X.shape[0] - Gref) ** 2))
    assert abs(E - f(V)) <= 1e-12 * abs(E)
    fd = _fd(f, V)
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_gram_row_zero_at_reference():
    rng = np.random.default_rng(12)
    V = rng.standard_normal((7, 5))
    Gref = V.T @ V / 7.0
    E, g = oracle.table1_gram(V, Gref, 1.0)
    assert E < 1e-28 and np.max(np.abs(g)) < 1e-14


def test_mse_row_matches_finite_differences():
    rng = np.random.default_rng(13)
    V = rng.standard_normal((7, 5))
    Vref = rng.standard_normal((7, 5))
    lam = 1e-3
    E, g = oracle.table1_mse(V, Vref, lam)
    f = lambda X: lam * float(np.sum((X - Vref) ** 2))
    assert abs(E - f(V)) <= 1e-12 * abs(E)
    fd = _fd(f, V)
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(fd))


def test_gram_row_catches_a_wrong_factor():
    """A gradient off by the factor 2 (a plausible slip: 2/np instead of 4/np) must fail the FD
    comparison above; this checks the tolerance is tight enough to see it."""
    rng = np.random.default_rng(14)
    V = rng.standard_normal((7, 5))
    A = rng.standard_normal((9, 5))
    Gref = A.T @ A / 9.0
    E, g = oracle.table1_gram(V, Gref, 1.0)
    f = lambda X: float(np.sum((X.T @ X / X.shape[0] - Gref) ** 2))
    fd = _fd(f, V)
    assert np.max(np.abs(0.5 * g - fd)) > 1e-3 * np.max(np.abs(fd))

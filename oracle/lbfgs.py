"""L-BFGS oracle (FP64, numpy). TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper minimises the transfer loss with L-BFGS (Section 3.1, after Nocedal 1980), starting from
the content image, with a history of 100 pairs at the first scale and 10 afterwards (Section 5.1).
It fixes nothing else; the readings used here (and by the library) are:

* two-loop recursion over the m most recent pairs (s_i, y_i), rho_i = 1 / (y_i^T s_i);
* initial inverse Hessian H0 = gamma I with gamma = s^T y / y^T y of the newest pair (1 if none);
* a pair is stored only if y^T s > 1e-10 (curvature condition), otherwise skipped;
* no line search: step t = 1, except on the first iteration where t = min(1, 1 / ||g||_1);
* the step taken is s = t d with d = -H g; y is formed at the next call as g_new - g_old.
"""
from __future__ import annotations

import numpy as np

CURV_EPS = 1e-10


def two_loop(g, S, Y, gamma):
    """d = -H g for the inverse-Hessian approximation defined by pairs S[i], Y[i] (oldest first)."""
    q = np.array(g, dtype=np.float64)
    m = len(S)
    rho = [1.0 / float(np.dot(Y[i], S[i])) for i in range(m)]
    alpha = [0.0] * m
    for i in range(m - 1, -1, -1):
        alpha[i] = rho[i] * float(np.dot(S[i], q))
        q -= alpha[i] * Y[i]
    r = gamma * q
    for i in range(m):
        beta = rho[i] * float(np.dot(Y[i], r))
        r += (alpha[i] - beta) * S[i]
    return -r


def dense_inverse_bfgs(S, Y, gamma, n):
    """Explicit inverse-BFGS matrix: H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, H0 = gamma I."""
    H = gamma * np.eye(n)
    I = np.eye(n)
    for s, y in zip(S, Y):
        rho = 1.0 / float(np.dot(y, s))
        H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    return H


class LBFGS:
    """Stateful driver with the library's call convention: step(x, g) updates x in place."""

    def __init__(self, n, m):
        self.n, self.m = n, m
        self.S, self.Y = [], []
        self.k = 0
        self.g_prev = None
        self.s_prev = None
        self.gamma = 1.0

    def step(self, x, g):
        g = np.asarray(g, np.float64)
        if self.k > 0:
            y = g - self.g_prev
            s = self.s_prev
            ys = float(np.dot(y, s))
            if ys > CURV_EPS:
                if len(self.S) == self.m:
                    self.S.pop(0)
                    self.Y.pop(0)
                self.S.append(s.copy())
                self.Y.append(y.copy())
                self.gamma = ys / float(np.dot(y, y))
        d = two_loop(g, self.S, self.Y, self.gamma if self.S else 1.0)
        t = min(1.0, 1.0 / float(np.abs(g).sum())) if self.k == 0 else 1.0
        s = t * d
        x += s
        self.s_prev = s
        self.g_prev = g.copy()
        self.k += 1
        return x

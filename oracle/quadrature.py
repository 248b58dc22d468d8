"""Tensor-product tanh-sinh quadrature on [0,1]^d (oracle, numpy float64).

Used only for the exact tier of the oracle on low-dimensional units: the
double-exponential substitution x = (1 + tanh(pi/2 sinh s))/2 maps [0,1] to the
real line and makes endpoint singularities of log type harmless (Takahasi and
Mori, 1974).  The trapezoidal rule with step h in s is then applied in each
dimension.
"""
from __future__ import annotations

import numpy as np


def tanh_sinh_rule(h=1.0 / 16, smax=3.2):
    """Nodes in (0,1) and weights of the tanh-sinh rule (float64).

    Nodes are returned as x and 1-x computed without cancellation; nodes that
    would round to 0 or 1 are dropped (their weights are below 1e-30).
    """
    k = np.arange(-int(smax / h), int(smax / h) + 1)
    s = k * h
    u = 0.5 * np.pi * np.sinh(s)
    # x = 1/(1+exp(-2u)), 1-x = 1/(1+exp(2u)), weight = h * pi/2 cosh(s) / (2 cosh^2 u)
    x = 1.0 / (1.0 + np.exp(-2.0 * u))
    w = h * 0.5 * np.pi * np.cosh(s) / (2.0 * np.cosh(u) ** 2)
    keep = (x > 0.0) & (x < 1.0) & (w > 1e-300)
    return x[keep], w[keep]


def integrate_box(f, dim, h=1.0 / 16, smax=3.2, chunk=1 << 20):
    """Integrate a vectorised f(X) (X of shape (n, dim)) over [0,1]^dim."""
    x, w = tanh_sinh_rule(h, smax)
    m = len(x)
    total = 0.0
    comp = 0.0
    N = m ** dim
    for start in range(0, N, chunk):
        idx = np.arange(start, min(N, start + chunk))
        X = np.empty((len(idx), dim))
        W = np.ones(len(idx))
        r = idx.copy()
        for d in range(dim - 1, -1, -1):
            X[:, d] = x[r % m]
            W *= w[r % m]
            r //= m
        v = np.sum(W * f(X))
        # Kahan summation over chunks
        y = v - comp
        tt = total + y
        comp = (tt - total) - y
        total = tt
    return total

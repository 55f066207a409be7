"""Integrated autocorrelation time -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  FP64.

The paper compares samplers by the integrated autocorrelation time of the
energy (Sec. III, Sec. IV) without naming an estimator.  We use the standard
windowed estimator with Sokal's automatic window (A. D. Sokal, "Monte Carlo
methods in statistical mechanics", 1997), for one series x_0 .. x_{n-1}:

    m = (1/n) sum_s x_s,   G(t) = (1/n) sum_{s=0}^{n-1-t} (x_s - m)(x_{s+t} - m),
    tau(W) = 1/2 + sum_{t=1}^{W} G(t) / G(0),
    W = the smallest W >= 1 with W >= c tau(W)   (c = 5; W <= n - 1).

A constant series (G(0) = 0) has tau = 1/2 and W = 0.  tau is in units of
the series' steps; for independent samples tau = 1/2.
"""
from __future__ import annotations

import numpy as np


def tau_int(x, c: float = 5.0):
    """(tau, W) of one series by the definitions above."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    d = x - x.mean()
    g0 = np.dot(d, d) / n
    if n < 2 or g0 == 0.0:
        return 0.5, 0
    tau = 0.5
    for t in range(1, n):
        tau += (np.dot(d[:n - t], d[t:]) / n) / g0
        if t >= c * tau:
            return tau, t
    return tau, n - 1


def tau_int_columns(X, c: float = 5.0):
    """tau and W of every column of a (steps, series) array."""
    X = np.asarray(X, dtype=np.float64)
    out = [tau_int(X[:, j], c) for j in range(X.shape[1])]
    return np.array([a for a, _ in out]), np.array([b for _, b in out], dtype=np.int64)

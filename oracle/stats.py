"""Ensemble statistics used to compare precision modes (test infrastructure only).

Sec. 4 of the paper compares each reduced-precision ensemble of states at t_end
with the FP64 ensemble by the two-sample Kolmogorov-Smirnov test and the
Wasserstein-1 distance, plus sample mean and variance.

* KS: D = sup_x |F1(x) - F2(x)| over the pooled sample; the p-value uses the
  asymptotic Kolmogorov distribution with effective size n1 n2 / (n1 + n2)
  (with integer-valued data the test is conservative).
* W1: for one-dimensional empirical laws, W1 = integral |F1 - F2| dx; for
  integer-valued samples that is sum_k |F1(k) - F2(k)|.
"""
from __future__ import annotations

import numpy as np


def ecdf_pair(a, b):
    a = np.sort(np.asarray(a, dtype=np.float64).ravel())
    b = np.sort(np.asarray(b, dtype=np.float64).ravel())
    grid = np.union1d(a, b)
    Fa = np.searchsorted(a, grid, side="right") / a.size
    Fb = np.searchsorted(b, grid, side="right") / b.size
    return grid, Fa, Fb


def ks_statistic(a, b):
    _, Fa, Fb = ecdf_pair(a, b)
    return float(np.max(np.abs(Fa - Fb)))


def kolmogorov_sf(x):
    """P(K > x) for the Kolmogorov distribution: 2 sum_{k>=1} (-1)^(k-1) e^{-2 k^2 x^2}."""
    if x <= 0.0:
        return 1.0
    if x < 0.3:
        # small-x form: sqrt(2 pi)/x sum_{k>=1} e^{-(2k-1)^2 pi^2 / (8 x^2)}
        s = 0.0
        for k in range(1, 50):
            s += np.exp(-((2 * k - 1) ** 2) * np.pi ** 2 / (8.0 * x * x))
        return float(max(0.0, min(1.0, 1.0 - np.sqrt(2.0 * np.pi) / x * s)))
    s = 0.0
    for k in range(1, 200):
        term = np.exp(-2.0 * k * k * x * x)
        s += term if (k % 2) else -term
        if term < 1e-18:
            break
    return float(max(0.0, min(1.0, 2.0 * s)))


def ks_2samp(a, b):
    """(D, p) of the two-sample KS test with the asymptotic p-value."""
    n1, n2 = np.asarray(a).size, np.asarray(b).size
    D = ks_statistic(a, b)
    ne = n1 * n2 / (n1 + n2)
    return D, kolmogorov_sf(D * np.sqrt(ne))


def wasserstein1(a, b):
    """W1 between two empirical laws on the real line (exact)."""
    grid, Fa, Fb = ecdf_pair(a, b)
    if grid.size < 2:
        return 0.0
    return float(np.sum(np.abs(Fa[:-1] - Fb[:-1]) * np.diff(grid)))


def summary(sample):
    s = np.asarray(sample, dtype=np.float64)
    return {"mean": float(s.mean()), "var": float(s.var())}

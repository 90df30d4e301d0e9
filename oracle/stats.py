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


# --------------------------------------------------------------------------
# Histogram-based statistics of integer ensembles (the device statistics
# kernels follow the same definitions, so results compare exactly):
#   count_histogram  h[k] = #{v = k} for k in 0..bins-1, values below 0 or
#                    above bins-1 counted in the end bins and reported;
#   hist_ks_w1       with C_a(k), C_b(k) the cumulative counts and n_a, n_b
#                    the totals, diff(k) = |C_a(k) n_b - C_b(k) n_a| (exact
#                    integers), D = max diff / (n_a n_b) and
#                    W1 = (sum over k of diff) / (n_a n_b), each quotient
#                    one IEEE division of the two integers rounded to
#                    binary64 (NaN when a sample is empty or
#                    bins n_a n_b >= 2^63);
#   dwell_histogram  for each trajectory of a 0/1 series s[k] (k = 0..K-1,
#                    nonzero = OFF), every completed OFF interval: the first
#                    OFF sample after an ON sample starts it, the first ON
#                    sample after that ends it; h[end - start] += 1.
# --------------------------------------------------------------------------
def count_histogram(values, bins):
    v = np.asarray(values, dtype=np.int64).ravel()
    clamped = int(np.count_nonzero((v < 0) | (v >= bins)))
    return np.bincount(np.clip(v, 0, bins - 1), minlength=bins).astype(np.int64), clamped


def hist_ks_w1(ha, hb):
    ha = [int(x) for x in np.asarray(ha).ravel()]
    hb = [int(x) for x in np.asarray(hb).ravel()]
    na, nb = sum(ha), sum(hb)
    if na == 0 or nb == 0 or len(ha) * na * nb >= 2**63:
        return float("nan"), float("nan")
    ca = cb = 0
    dmax = 0
    total = 0
    for x, y in zip(ha, hb):
        ca += x
        cb += y
        d = abs(ca * nb - cb * na)
        dmax = max(dmax, d)
        total += d
    return float(dmax) / float(na * nb), float(total) / float(na * nb)


def dwell_histogram(series):
    """series [K, n]: nonzero = OFF; returns h [K] (h[d] = completed OFF intervals of d samples)."""
    s = np.asarray(series)
    K, n = s.shape
    h = np.zeros(K, dtype=np.int64)
    for j in range(n):
        start = -1
        prev_off = bool(s[0, j] != 0)
        for k in range(1, K):
            off = bool(s[k, j] != 0)
            if off and not prev_off:
                start = k
            elif not off and prev_off and start >= 0:
                h[k - start] += 1
                start = -1
            prev_off = off
    return h

"""Pins of the oracle's tau-leaping (fixed leap; the approximate method family
of Sec. 1 and Sec. 2, in the reduced-precision modes of Sec. 3) against facts
fixed by probability and arithmetic, not by the oracle itself:

* its exponential against numpy's (ulp bound);
* its Poisson sampler, both precisions, both algorithms (multiplication
  method below 10, transformed rejection from 10), against the Poisson
  law by chi-square, mean and variance;
* a pure-birth network, whose leaped state is a sum of independent Poisson
  variables and hence exactly Poisson(k L tau);
* the birth-death network, whose leap map is linear, so mean and variance
  follow closed recursions;
* the leap grid and snapshot rule (prefix consistency, t_final, events);
* clamping, overflow and NaN handling.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2605_00479_gb300 import presets as P


def ulp_distance_f32(a, b):
    ia = a.astype(np.float32).view(np.int32).astype(np.int64)
    ib = b.astype(np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def test_exp_f32_within_two_ulps():
    x = np.linspace(-30.0, 0.0, 40001).astype(np.float32)
    got = oracle.exp_f32(x)
    ref = np.exp(x.astype(np.float64)).astype(np.float32)
    assert ulp_distance_f32(got, ref).max() <= 2
    assert oracle.exp_f32(np.zeros(1, np.float32))[0] == 1.0


def test_exp_f64_relative_error():
    x = np.linspace(-30.0, 0.0, 40001)
    got = oracle.exp_f64(x)
    ref = np.exp(x)
    assert np.max(np.abs(got - ref) / ref) < 4 * np.finfo(np.float64).eps
    assert oracle.exp_f64(np.zeros(1))[0] == 1.0


def chi2_poisson_pvalue(sample, lam):
    """Chi-square goodness of fit to Poisson(lam), tail bins merged to >= 5 expected."""
    n = sample.size
    lo = int(max(0, np.floor(lam - 8 * np.sqrt(lam) - 5)))
    hi = int(np.ceil(lam + 8 * np.sqrt(lam) + 10))
    ks = np.arange(lo, hi + 1)
    p = stats.poisson.pmf(ks, lam)
    p[0] += stats.poisson.cdf(lo - 1, lam) if lo > 0 else 0.0
    p[-1] += stats.poisson.sf(hi, lam)
    obs = np.bincount(np.clip(sample, lo, hi) - lo, minlength=ks.size).astype(float)
    exp = p * n
    # merge bins from both ends until each holds >= 5 expected
    o_m, e_m, acc_o, acc_e = [], [], 0.0, 0.0
    for o, e in zip(obs, exp):
        acc_o += o
        acc_e += e
        if acc_e >= 5.0:
            o_m.append(acc_o)
            e_m.append(acc_e)
            acc_o = acc_e = 0.0
    o_m[-1] += acc_o
    e_m[-1] += acc_e
    o_m, e_m = np.array(o_m), np.array(e_m)
    chi2 = ((o_m - e_m) ** 2 / e_m).sum()
    return stats.chi2.sf(chi2, o_m.size - 1)


@pytest.mark.parametrize("prec64", [False, True])
@pytest.mark.parametrize("lam", [0.3, 2.5, 9.9, 10.0, 37.5, 400.0, 5000.0])
def test_poisson_sampler_law(lam, prec64):
    n = 40000
    k = oracle.poisson(lam, n, prec64=prec64, seed=2605 + int(lam * 10))
    assert k.min() >= 0
    assert chi2_poisson_pvalue(k, lam) > 1e-4
    assert abs(k.mean() - lam) < 5 * np.sqrt(lam / n)
    # variance of the sample variance of a Poisson law: (lam + 2 lam^2 (n/(n-1))) / n
    sd_var = np.sqrt((lam + 2 * lam * lam) / n)
    assert abs(k.var(ddof=1) - lam) < 6 * sd_var


def test_poisson_sampler_zero_rate_and_stream_independence():
    assert np.all(oracle.poisson(0.0, 100) == 0)
    a = oracle.poisson(50.0, 20000, seed=1)
    b = oracle.poisson(50.0, 20000, seed=2)
    assert not np.array_equal(a, b)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.05


def pure_birth(k=3.0):
    return {"order": np.array([[0]]), "stoich": np.array([[1]]), "rate": np.array([k])}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pure_birth_is_exactly_poisson(precision):
    """Zero-order birth at rate k: every leap adds Poisson(k tau), so
    x(L tau) ~ Poisson(k L tau) exactly (sum of independent Poisson laws)."""
    k, tau, t_end, n = 3.0, 0.25, 10.0, 20000
    r = oracle.tau_run(pure_birth(k), [0], n, t_end, tau, [t_end], precision=precision, seed=7)
    x = r["snapshots"][0, 0].astype(np.int64)
    lam = k * t_end
    assert chi2_poisson_pvalue(x, lam) > 1e-4
    assert np.array_equal(r["n_events"], x)
    assert np.all(r["status"] == 0)
    assert np.all(r["t_final"] == 40 * tau)


@pytest.mark.parametrize("precision,rounding", [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "rn"),
                                                ("uniform_f16", "sr")])
def test_birth_death_mean_and_variance_recursions(precision, rounding):
    """Birth-death leap x' = x + Poi(k tau) - Poi(gamma tau x) is linear:
    m' = (1 - gamma tau) m + k tau,  v' = (1 - gamma tau)^2 v + k tau + gamma tau m."""
    k, g, tau, t_end, n = 10.0, 0.1, 0.5, 20.0, 20000
    samples = np.array([2.0, 5.0, 10.0, 20.0])
    r = oracle.tau_run(P.birth_death(k, g), [0], n, t_end, tau, samples, precision=precision, rounding=rounding,
                       seed=11)
    m, v = 0.0, 0.0
    expect = {}
    for leap in range(int(t_end / tau)):
        m, v = (1 - g * tau) * m + k * tau, (1 - g * tau) ** 2 * v + k * tau + g * tau * m
        expect[(leap + 1) * tau] = (m, v)
    for kk, s in enumerate(samples):
        em, ev = expect[s]
        x = r["snapshots"][kk, 0].astype(np.float64)
        assert abs(x.mean() - em) < 5 * np.sqrt(ev / n) + 1e-3 * em, (s, x.mean(), em)
        assert abs(x.var(ddof=1) - ev) < 6 * np.sqrt((ev + 2 * ev * ev) / n) + 1e-3 * ev, (s, x.var(), ev)
    assert np.all((r["status"] & ~np.uint32(16)) == 0)


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16", "uniform_f16"])
def test_leap_grid_prefix_consistency(precision):
    """Leap n draws from counters (n, trajectory), so a run to m tau ends in the
    state that a longer run shows at s = m tau; a sample inside a leap shows
    the state at the start of that leap."""
    model = P.birth_death(10.0, 0.1)
    tau, n = 0.3, 64
    long = oracle.tau_run(model, [5], n, 6.0, tau, [0.0, 0.15, 0.3, 0.45, 1.5, 6.0], precision=precision, seed=3)
    snaps = long["snapshots"][:, 0]
    assert np.all(snaps[0] == 5) and np.all(snaps[1] == 5)
    one = oracle.tau_run(model, [5], n, 0.3, tau, [0.3], precision=precision, seed=3)
    assert np.array_equal(one["snapshots"][0, 0], snaps[2])
    assert np.array_equal(snaps[3], snaps[2])
    five = oracle.tau_run(model, [5], n, 1.5, tau, [1.5], precision=precision, seed=3)
    assert np.array_equal(five["snapshots"][0, 0], snaps[4])
    assert np.all(long["t_final"] == 20 * tau)
    # t_end not on the grid: ceil(t_end / tau) leaps
    odd = oracle.tau_run(model, [5], n, 1.0, tau, [1.0], precision=precision, seed=3)
    assert np.all(odd["t_final"] == 4 * tau)


def test_clamping_keeps_counts_non_negative():
    """Pure death with gamma tau = 2: leaps overshoot; counts are set to 0 and flagged."""
    model = {"order": np.array([[1]]), "stoich": np.array([[-1]]), "rate": np.array([1.0])}
    r = oracle.tau_run(model, [50], 2000, 20.0, 2.0, [2.0, 4.0, 20.0], precision="fp64", seed=5)
    assert r["snapshots"].min() >= 0
    assert np.any(r["status"] & 16)
    assert np.all(r["snapshots"][-1] == 0)
    assert np.all((r["status"] & ~np.uint32(16)) == 0)


def test_overflow_and_nan_stop_the_trajectory():
    # fp32: lambda = 3e38 * 10 overflows binary32 but not binary64
    model = {"order": np.array([[0]]), "stoich": np.array([[1]]), "rate": np.array([3e38])}
    r32 = oracle.tau_run(model, [7], 4, 10.0, 10.0, [10.0], precision="fp32", seed=1)
    assert np.all(r32["status"] == 1)
    assert np.all(r32["snapshots"][0, 0] == 7)
    assert np.all(r32["n_events"] == 0) and np.all(r32["t_final"] == 0.0)
    # binary16: the rate itself rounds to +inf
    m16 = {"order": np.array([[0]]), "stoich": np.array([[1]]), "rate": np.array([1e5])}
    r16 = oracle.tau_run(m16, [0], 4, 1.0, 0.5, [1.0], precision="mixed_f16", seed=1)
    assert np.all(r16["status"] == 1)
    # uniform binary16: a Hill amplitude beyond the format's range rounds to
    # +inf (overflow); with X^2 also +inf the quotient inf / inf is NaN
    hill = P.hill_self(alpha0=1.0, alpha=1e6, h=2, gamma=1.0)
    rh = oracle.tau_run(hill, [0], 4, 1.0, 0.5, [1.0], precision="uniform_f16", seed=1)
    assert np.all(rh["status"] == 1)
    rn = oracle.tau_run(hill, [300], 4, 1.0, 0.5, [1.0], precision="uniform_f16", seed=1)
    assert np.all(rn["status"] == 8)
    assert np.all(rn["snapshots"][0, 0] == 300)

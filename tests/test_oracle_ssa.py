"""Pins for the oracle's direct-method simulation (CPU only).

The fp64 mode is pinned by closed-form laws and master-equation solutions; the
reduced-precision modes by exact reductions (modes whose arithmetic is exact
must reproduce the fp32 trajectories bit for bit), exact invariants, the SR
unbiasedness seen in ensembles, and the qualitative failures the paper reports.
"""
import math
import os

import numpy as np
import pytest
import scipy.special
import scipy.stats

import oracle
from oracle import cme, stats
from paper_2605_00479_gb300 import presets as P

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ALL_MODES = [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_f16", "sr"), ("mixed_bf16", "rn"),
             ("mixed_bf16", "sr"), ("uniform_f16", "rn"), ("uniform_f16", "sr"), ("uniform_bf16", "rn"),
             ("uniform_bf16", "sr")]


def chi2_pvalue(samples, pmf, min_expected=5.0):
    """Chi-square goodness of fit of integer samples against a pmf on 0..len-1;
    the upper tail is lumped into one bin and small bins are merged."""
    n = samples.size
    counts = np.bincount(samples, minlength=pmf.size)
    tail_obs = counts[pmf.size:].sum() if counts.size > pmf.size else 0
    counts = counts[:pmf.size].astype(float)
    exp = pmf * n
    obs_bins, exp_bins = [], []
    o = e = 0.0
    for ci, ei in zip(counts, exp):
        o += ci
        e += ei
        if e >= min_expected:
            obs_bins.append(o)
            exp_bins.append(e)
            o = e = 0.0
    o += tail_obs
    e += max(0.0, n - exp.sum())
    if obs_bins:
        obs_bins[-1] += o
        exp_bins[-1] += e
    obs_bins, exp_bins = np.array(obs_bins), np.array(exp_bins)
    chi2 = np.sum((obs_bins - exp_bins) ** 2 / exp_bins)
    return scipy.stats.chi2.sf(chi2, max(1, obs_bins.size - 1))


# --------------------------------------------------------- closed forms
def test_birth_death_transient_poisson():
    """From X(0) = 0 the birth-death law is Poisson(k/gamma (1 - e^{-gamma t}))
    at every t (Sec. 4.1 gives the stationary limit Poisson(kb/kd))."""
    m = P.birth_death(20.0, 1.0)
    ts = P.even_samples(5.0, 6)
    r = oracle.run(m, [0], 20000, 5.0, ts, "fp64", seed=11)
    assert np.all(r["status"] == 0)
    for k, t in enumerate(ts):
        lam = 20.0 * (1.0 - math.exp(-t))
        x = r["snapshots"][k, 0]
        if t == 0:
            assert np.all(x == 0)
            continue
        pmf = scipy.stats.poisson.pmf(np.arange(200), lam)
        assert chi2_pvalue(x, pmf) > 1e-4, (t, x.mean(), lam)


def beta_poisson_pmf(n, a, b, lam):
    """Telegraph stationary law (Sec. 4.3: governed by a = kon/beta,
    b = koff/beta, lambda = alpha/beta): the Poisson mixture over a
    Beta(a, b)-distributed on-fraction,
    P(n) = lam^n/n! Gamma(a+n)Gamma(a+b)/(Gamma(a)Gamma(a+b+n)) 1F1(a+n; a+b+n; -lam)."""
    n = np.asarray(n, dtype=float)
    logc = (n * math.log(lam) - scipy.special.gammaln(n + 1) + scipy.special.gammaln(a + n)
            + scipy.special.gammaln(a + b) - scipy.special.gammaln(a) - scipy.special.gammaln(a + b + n))
    return np.exp(logc) * scipy.special.hyp1f1(a + n, a + b + n, -lam)


def test_beta_poisson_reproduces_paper_moments():
    """Sec. 4.3 bimodal set (a = b = 0.05, lambda = 20): ~42% mass at zero and
    mean ~10; the underflow-stress set (a = 0.01, b = 0.1, lambda = 5): P(0) ~ 0.90."""
    n = np.arange(400)
    p = beta_poisson_pmf(n, 0.05, 0.05, 20.0)
    assert abs(p.sum() - 1) < 1e-9 and abs(p[0] - 0.42) < 0.01 and abs((n * p).sum() - 10.0) < 0.05
    p2 = beta_poisson_pmf(n, 0.01, 0.1, 5.0)
    assert abs(p2[0] - 0.90) < 0.01


def test_telegraph_stationary_beta_poisson():
    m = P.telegraph(kon=1.0, koff=1.5, km=12.0, gamma=1.0)
    r = oracle.run(m, P.TELEGRAPH_X0, 20000, 25.0, [25.0], "fp64", seed=5)
    x = r["snapshots"][-1, 2]
    pmf = beta_poisson_pmf(np.arange(120), 1.0, 1.5, 12.0)
    assert chi2_pvalue(x, pmf) > 1e-4
    g = r["snapshots"][-1, :2]
    assert np.all(g.sum(axis=0) == 1)


def test_dimer_detailed_balance_and_conservation():
    """Sec. 4.4: nA + 2 nD is conserved; the stationary law follows from
    detailed balance, pi(d) proportional to (kf/(2 kr))^d n0!/((n0-2d)! d!)."""
    n0, kf, kr = 100, 1e-3, 0.1
    m = P.dimer(kf, kr)
    ts = P.even_samples(60.0, 7)
    r = oracle.run(m, P.dimer_x0(n0), 10000, 60.0, ts, "fp64", seed=9)
    s = r["snapshots"]
    assert np.all(s[:, 0, :] + 2 * s[:, 1, :] == n0)
    d = np.arange(n0 // 2 + 1)
    logp = d * math.log(kf / (2 * kr)) + scipy.special.gammaln(n0 + 1) - scipy.special.gammaln(n0 - 2 * d + 1) \
        - scipy.special.gammaln(d + 1)
    pmf = np.exp(logp - logp.max())
    pmf /= pmf.sum()
    assert chi2_pvalue(s[-1, 1], pmf) > 1e-4
    # the paper's n0 = 100 moments: <nA> ~ 62, <nD> ~ 19
    assert abs((d * pmf).sum() - 19.0) < 0.5


def test_hill_self_repression_stationary_law():
    """Hill law of Sec. 4.5 on a one-species chain: birth alpha0 + alpha/(1+n^h),
    death gamma n; stationary law by detailed balance."""
    a0, a, h, g = 1.0, 30.0, 2, 1.0
    m = P.hill_self(a0, a, h, g)
    r = oracle.run(m, [0], 20000, 20.0, [20.0], "fp64", seed=13)
    pmf = cme.stationary_birth_death_chain(lambda n: a0 + a / (1.0 + n ** h), lambda n: g * n, 150)
    assert chi2_pvalue(r["snapshots"][-1, 0], pmf) > 1e-4


# ---------------------------------------------------- master equation
@pytest.mark.parametrize("name", ["birth_death", "telegraph", "dimer", "repressilator_small"])
def test_transient_law_matches_truncated_cme(name):
    """Brute force on small state spaces: the empirical law at every sample
    time must match p(t) = p(0) exp(Q t) of the truncated master equation."""
    if name == "birth_death":
        m, x0, bounds, t_end = P.birth_death(6.0, 0.7), [3], [80], 4.0
    elif name == "telegraph":
        m, x0, bounds, t_end = P.telegraph(0.4, 0.3, 5.0, 1.0), P.TELEGRAPH_X0, [1, 1, 60], 4.0
    elif name == "dimer":
        m, x0, bounds, t_end = P.dimer(0.05, 0.3), P.dimer_x0(12), [12, 6], 3.0
    else:
        m = P.repressilator(alpha0=0.3, alpha=1.5, h=2, beta=0.8, mdecay=1.0, pdecay=1.0)
        x0, bounds, t_end = [0, 0, 0, 2, 0, 0], [5, 5, 5, 5, 5, 5], 0.8
    ts = P.even_samples(t_end, 5)
    r = oracle.run(m, x0, 8000, t_end, ts, "fp64", seed=21)
    states, Pt = cme.transient(m, x0, bounds, ts)
    index = {s: i for i, s in enumerate(states)}
    assert Pt[-1].sum() > 0.995   # the truncation loses little probability
    for k in range(1, ts.size):
        snaps = r["snapshots"][k].T
        ids = np.array([index.get(tuple(int(v) for v in s), -1) for s in snaps])
        assert np.mean(ids < 0) < 0.01
        ids = ids[ids >= 0]
        pmf = Pt[k] / Pt[k].sum()
        order = np.argsort(-pmf)   # merge small bins in decreasing probability
        rank = np.empty_like(order)
        rank[order] = np.arange(order.size)
        assert chi2_pvalue(rank[ids], pmf[order]) > 1e-4, (name, k)


def test_schlogl_transient_matches_cme_and_paper_table():
    """Sec. 4.2: the FP64 row of the Schloegl table (mean 317.2, variance 56674,
    N = 10^4, t_end = 10) is the law at t = 10, which the truncated CME gives
    (stored in tests/golden/schlogl_cme_t10.txt by tests/golden/make_golden.py)."""
    g = np.loadtxt(os.path.join(GOLDEN, "schlogl_cme_t10.txt"))
    x, p = g[:, 0].astype(int), g[:, 1]
    mean = float((x * p).sum())
    var = float((x * x * p).sum() - mean ** 2)
    se = math.sqrt(56674.0 / 1e4)
    assert abs(mean - 317.2) < 3 * se
    assert abs(var - 56674.0) / 56674.0 < 0.05
    m = P.schlogl()
    r = oracle.run(m, P.schlogl_x0(m), 400, 10.0, P.even_samples(10.0, 50), "fp64", seed=17)
    xs = r["snapshots"][-1, 0]
    cdf = np.cumsum(p)
    emp = np.searchsorted(np.sort(xs), x, side="right") / xs.size
    D = np.max(np.abs(emp - cdf))
    assert scipy.stats.kstwobign.sf(D * math.sqrt(xs.size)) > 1e-3
    # bimodal: mass near both modes (the paper's modes are ~90 and ~560)
    assert np.mean(xs < 250) > 0.2 and np.mean(xs > 400) > 0.2


# -------------------------------------------------------- exact reductions
def test_mixed_modes_reduce_to_fp32_when_arithmetic_is_exact():
    """Birth-death with kb = 20, kd = 1 and counts < 256: every propensity
    operation is exact in binary16 and bfloat16, so every mixed mode (RN or
    SR) must reproduce the fp32 trajectories bit for bit; the paper's
    birth-death table shows all six mixed rows identical."""
    m = P.birth_death(20.0, 1.0)
    ts = P.even_samples(10.0, 11)
    ref = oracle.run(m, [0], 3000, 10.0, ts, "fp32", seed=3)
    for prec in ("mixed_f16", "mixed_bf16"):
        for rnd in ("rn", "sr"):
            r = oracle.run(m, [0], 3000, 10.0, ts, prec, rnd, seed=3)
            np.testing.assert_array_equal(r["snapshots"], ref["snapshots"])
            np.testing.assert_array_equal(r["n_events"], ref["n_events"])
            np.testing.assert_array_equal(r["t_final"], ref["t_final"])
    f64 = oracle.run(m, [0], 3000, 10.0, ts, "fp64", seed=3)
    assert np.mean(np.all(f64["snapshots"] == ref["snapshots"], axis=(0, 1))) > 0.98


def test_mixed_sr_equals_rn_for_telegraph_with_unit_decay():
    """Sec. 4.3 tables: mixed SR rows equal the RN rows because with beta = 1
    and a gene count in {0, 1} every propensity product is exact."""
    m = P.telegraph(0.05, 0.05, 20.0, 1.0)
    for prec in ("mixed_f16", "mixed_bf16"):
        a = oracle.run(m, P.TELEGRAPH_X0, 2000, 50.0, [25.0, 50.0], prec, "rn", seed=4)
        b = oracle.run(m, P.TELEGRAPH_X0, 2000, 50.0, [25.0, 50.0], prec, "sr", seed=4)
        np.testing.assert_array_equal(a["snapshots"], b["snapshots"])


@pytest.mark.parametrize("prec,rnd", ALL_MODES)
def test_dimer_conservation_in_every_mode(prec, rnd):
    """nA + 2 nD = n0 exactly at every snapshot: the integer state update is
    exact whatever the propensity precision (Sec. 3.2, Sec. 4.4)."""
    r = oracle.run(P.dimer(), P.dimer_x0(300), 300, 20.0, P.even_samples(20.0, 9), prec, rnd, seed=2,
                   max_events=200000)
    s = r["snapshots"]
    assert np.all(s[:, 0, :] + 2 * s[:, 1, :] == 300)


def test_sr_differs_from_rn_when_propensities_round():
    """The dimer's kf nA(nA-1)/2 is inexact in 16 bits, so SR must change some
    trajectories (the paper's dimer table has distinct SR and RN rows)."""
    a = oracle.run(P.dimer(), P.dimer_x0(300), 500, 20.0, [20.0], "mixed_bf16", "rn", seed=6)
    b = oracle.run(P.dimer(), P.dimer_x0(300), 500, 20.0, [20.0], "mixed_bf16", "sr", seed=6)
    assert np.any(a["snapshots"] != b["snapshots"])


# ------------------------------------------------- the paper's patterns
def test_schlogl_fp16_overflow_without_normalisation():
    """Sec. 4.2 table: with A = 1e5 the binary16 propensity overflows; every
    trajectory stays at X0 = 250 (mean 250.0, variance 0).  Folding the
    reservoirs into the rate constants (normalisation) removes the overflow."""
    m = P.schlogl()
    x0 = P.schlogl_x0(m)
    for prec in ("mixed_f16", "uniform_f16"):
        for rnd in ("rn", "sr"):
            r = oracle.run(m, x0, 200, 10.0, P.even_samples(10.0, 50), prec, rnd, seed=1)
            assert np.all(r["status"] == oracle.STATUS_OVERFLOW)
            assert np.all(r["snapshots"][:, 0, :] == 250)
    r = oracle.run(m, x0, 100, 10.0, P.even_samples(10.0, 50), "mixed_f16", "rn", normalise=True, seed=1)
    assert np.all(r["status"] == 0) and r["snapshots"][-1, 0].std() > 50


def test_telegraph_underflow_uniform_bf16_rn_collapses_and_sr_recovers():
    """Sec. 4.3 underflow-stress set (kon = 0.01, koff = 0.1, alpha = 5,
    beta = 1): uniform BF16 RTN collapses the mRNA mean (0.444 -> 0.006) while
    uniform BF16+SR matches FP64 (KS p = 0.943)."""
    m = P.telegraph(0.01, 0.1, 5.0, 1.0)
    n = 16000
    ref = oracle.run_parallel(m, P.TELEGRAPH_X0, n, 200.0, [200.0], precision="fp64", seed=101)["snapshots"][-1, 2]
    rn = oracle.run_parallel(m, P.TELEGRAPH_X0, n, 200.0, [200.0], precision="uniform_bf16", rounding="rn",
                             seed=202, max_events=100000)["snapshots"][-1, 2]
    sr = oracle.run_parallel(m, P.TELEGRAPH_X0, n, 200.0, [200.0], precision="uniform_bf16", rounding="sr",
                             seed=303, max_events=100000)["snapshots"][-1, 2]
    assert 0.40 < ref.mean() < 0.50
    assert rn.mean() < 0.2 and stats.ks_2samp(ref, rn)[1] < 1e-6
    assert stats.ks_2samp(ref, sr)[1] > 0.01


def test_birth_death_uniform_fp16_rn_biased_and_sr_unbiased():
    """Sec. 4.1 table (uniform precision): FP16 RTN shifts the law (KS
    p = 2.3e-8, mean 19.78) while FP16+SR passes (KS p = 0.681)."""
    m = P.birth_death(20.0, 1.0)
    n = 16000
    ref = oracle.run_parallel(m, [0], n, 100.0, [100.0], precision="fp64", seed=404)["snapshots"][-1, 0]
    rn = oracle.run_parallel(m, [0], n, 100.0, [100.0], precision="uniform_f16", rounding="rn", seed=505,
                             max_events=100000)["snapshots"][-1, 0]
    sr = oracle.run_parallel(m, [0], n, 100.0, [100.0], precision="uniform_f16", rounding="sr", seed=606,
                             max_events=100000)["snapshots"][-1, 0]
    assert rn.mean() < 19.9 and stats.ks_2samp(ref, rn)[1] < 1e-3
    assert stats.ks_2samp(ref, sr)[1] > 0.01 and abs(sr.mean() - 20.0) < 0.15


# ------------------------------------------------------------ status codes
def test_max_events_status_and_fill():
    m = P.birth_death(20.0, 1.0)
    r = oracle.run(m, [0], 50, 10.0, P.even_samples(10.0, 11), "fp32", seed=1, max_events=7)
    assert np.all(r["status"] == oracle.STATUS_MAX_EVENTS) and np.all(r["n_events"] == 7)
    last = r["snapshots"][-1, 0]
    assert np.all(r["snapshots"][-2, 0] == last)


def test_absorbing_state_ends_quietly():
    m = P.birth_death(0.0, 1.0)   # pure death: a0 = 0 once X = 0
    r = oracle.run(m, [5], 100, 1000.0, P.even_samples(1000.0, 5), "fp64", seed=1)
    assert np.all(r["status"] == 0) and np.all(r["n_events"] == 5)
    assert np.all(r["snapshots"][-1, 0] == 0)


def test_int16_storage_range_flag():
    m = P.birth_death(40000.0, 0.0)   # pure birth beyond the int16 range
    r = oracle.run(m, [0], 4, 1.0, [0.5, 1.0], "fp32", seed=1, state_bytes=2)
    assert np.all(r["status"] & oracle.STATUS_STATE_RANGE)
    assert np.all(r["snapshots"][-1, 0] == 32767)


def test_negative_count_flag():
    m = {"order": np.array([[0]]), "stoich": np.array([[-1]]), "rate": np.array([1.0]), "law": np.array([0])}
    r = oracle.run(m, [2], 3, 100.0, [100.0], "fp64", seed=1)
    assert np.all(r["status"] == oracle.STATUS_STATE_RANGE) and np.all(r["n_events"] == 3)


def test_trajectories_depend_only_on_global_id():
    """Splitting a run by trajectory-id ranges changes nothing."""
    m = P.telegraph(0.3, 0.2, 10.0, 1.0)
    whole = oracle.run(m, P.TELEGRAPH_X0, 64, 10.0, [5.0, 10.0], "uniform_f16", "sr", seed=9)
    part = oracle.run(m, P.TELEGRAPH_X0, 32, 10.0, [5.0, 10.0], "uniform_f16", "sr", seed=9, g0=32)
    np.testing.assert_array_equal(whole["snapshots"][:, :, 32:], part["snapshots"])
    np.testing.assert_array_equal(whole["t_final"][32:], part["t_final"])


def test_selective_sr_recovers_the_underflow_failure():
    """Sec. 3.3 names selective SR (SR only at accumulation points) without
    testing it: with the partial sums and the clock rounded stochastically and
    everything else to nearest, uniform BF16 no longer swamps kon = 0.01."""
    m = P.telegraph(0.01, 0.1, 5.0, 1.0)
    n = 16000
    ref = oracle.run_parallel(m, P.TELEGRAPH_X0, n, 200.0, [200.0], precision="fp64", seed=101)["snapshots"][-1, 2]
    sra = oracle.run_parallel(m, P.TELEGRAPH_X0, n, 200.0, [200.0], precision="uniform_bf16", rounding="sra",
                              seed=404, max_events=100000)["snapshots"][-1, 2]
    assert stats.ks_2samp(ref, sra)[1] > 0.01 and abs(sra.mean() - ref.mean()) < 0.05


def test_selective_sr_rounds_only_accumulations():
    """Selective SR differs from RN only through the sums and the clock: with
    the clock kept exact (t_end tiny and dyadic rates), and one reaction, the
    partial sums do not exist and the two runs agree step for step."""
    m = {"order": np.array([[1]]), "stoich": np.array([[-1]]), "rate": np.array([1.0]), "law": np.array([0])}
    a = oracle.run(m, [40], 500, 0.25, [0.125, 0.25], "uniform_f16", "rn", seed=3)
    b = oracle.run(m, [40], 500, 0.25, [0.125, 0.25], "uniform_f16", "sra", seed=3)
    # same draws and RN propensities; only t_new's rounding may differ
    assert np.mean(np.all(a["snapshots"] == b["snapshots"], axis=(0, 1))) > 0.5
    with pytest.raises(ValueError):
        oracle.run(m, [40], 10, 1.0, [1.0], "mixed_f16", "sra", seed=3)

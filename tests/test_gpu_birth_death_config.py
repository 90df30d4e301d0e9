"""The small birth-death configuration end to end on the GPU: 0 -> X at k = 10,
X -> 0 at gamma X with gamma = 0.1, X0 = 0, 10^4 trajectories to t_end = 100
with 101 evenly spaced snapshots, Philox seed 0, fp64 and mixed precision
(binary16 propensities, binary32 sum and clock, int32 state).  Every
trajectory equals the oracle bit for bit, and the ensemble follows the law the
model fixes: from X(0) = 0 the count is Poisson(k/gamma (1 - e^{-gamma t})) at
every t (Sec. 4.1: the stationary limit Poisson(k/gamma) = Poisson(100))."""
import math

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_RATE, GAMMA, N, T_END, K = 10.0, 0.1, 10_000, 100.0, 101


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    assert torch.cuda.is_available()
    mod.lib()
    return mod


def chi2_pvalue(x, lam):
    """Goodness of fit of integer samples to Poisson(lam), bins with an
    expected count of at least 5 (tails pooled)."""
    n = x.size
    ks = np.arange(0, int(lam + 10 * math.sqrt(lam)) + 1)
    pmf = scipy.stats.poisson.pmf(ks, lam)
    keep = pmf * n >= 5
    lo, hi = ks[keep][0], ks[keep][-1]
    obs = np.array([np.sum(x <= lo)] + [np.sum(x == k) for k in range(lo + 1, hi)] + [np.sum(x >= hi)], float)
    exp = np.array([scipy.stats.poisson.cdf(lo, lam)] +
                   [scipy.stats.poisson.pmf(k, lam) for k in range(lo + 1, hi)] +
                   [scipy.stats.poisson.sf(hi - 1, lam)]) * n
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    return scipy.stats.chi2.sf(chi2, obs.size - 1)


@pytest.mark.parametrize("prec", ["fp64", "mixed_f16"])
def test_small_birth_death_configuration(ssa, prec):
    md = P.birth_death(K_RATE, GAMMA)
    samples = P.even_samples(T_END, K)
    m = ssa.Model.from_dict(md)
    r = ssa.ensemble_run(m, N, [0], T_END, samples, prec, "rn", False, 0, 10**9)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in r.items()}
    o = oracle.run_parallel(md, [0], N, T_END, samples, precision=prec, rounding="rn", seed=0)
    np.testing.assert_array_equal(g["snapshots"], o["snapshots"])
    np.testing.assert_array_equal(g["n_events"], o["n_events"])
    np.testing.assert_array_equal(g["t_final"].view(np.uint64), o["t_final"].view(np.uint64))
    assert np.all(g["status"] == 0)
    # the transient Poisson law at t = 25, 50 and the last snapshot (t = 100: Poisson(99.995))
    for k in (25, 50, K - 1):
        t = samples[k]
        lam = K_RATE / GAMMA * (1.0 - math.exp(-GAMMA * t))
        x = g["snapshots"][k, 0].astype(np.int64)
        assert abs(x.mean() - lam) < 4.0 * math.sqrt(lam / N), (t, x.mean(), lam)
        assert chi2_pvalue(x, lam) > 1e-4, (t, lam)

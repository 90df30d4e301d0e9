"""GPU parity of the on-device ensemble statistics (histograms, two-sample KS
statistic and Wasserstein-1 distance, OFF-dwell extraction) with the
oracle's integer-exact definitions."""
import numpy as np
import pytest

from oracle import stats as ost
from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    assert torch.cuda.is_available()
    mod.lib()
    return mod


@pytest.mark.parametrize("dtype,bins", [(np.int32, 64), (np.int16, 700), (np.int32, 20000)])
def test_count_histogram_exact_and_accumulating(ssa, dtype, bins):
    rng = np.random.default_rng(bins)
    v1 = rng.integers(-5, bins + 5, size=100003).astype(dtype)
    v2 = rng.integers(0, bins, size=7777).astype(dtype)
    h, c = ssa.count_histogram(torch.from_numpy(v1).cuda(), bins)
    ssa.count_histogram(torch.from_numpy(v2).cuda(), bins, hist=h, clamped=c)
    torch.cuda.synchronize()
    o1, oc1 = ost.count_histogram(v1, bins)
    o2, oc2 = ost.count_histogram(v2, bins)
    np.testing.assert_array_equal(h.cpu().numpy(), o1 + o2)
    assert int(c.item()) == oc1 + oc2


@pytest.mark.parametrize("na,nb,lam_a,lam_b,bins", [(1000, 1000, 10.0, 10.0, 64), (250000, 100000, 300.0, 302.0, 2048),
                                                    (5, 70000, 3.0, 40.0, 9000), (100000, 3, 1.0, 1.0, 16)])
def test_ks_w1_bit_exact(ssa, na, nb, lam_a, lam_b, bins):
    rng = np.random.default_rng(na + nb)
    a = rng.poisson(lam_a, na).astype(np.int32)
    b = rng.poisson(lam_b, nb).astype(np.int32)
    ha, _ = ssa.count_histogram(torch.from_numpy(a).cuda(), bins)
    hb, _ = ssa.count_histogram(torch.from_numpy(b).cuda(), bins)
    out = ssa.hist_ks_w1(ha, hb).cpu().numpy()
    D, W1 = ost.hist_ks_w1(ost.count_histogram(a, bins)[0], ost.count_histogram(b, bins)[0])
    assert out.view(np.uint64)[0] == np.float64(D).view(np.uint64)
    assert out.view(np.uint64)[1] == np.float64(W1).view(np.uint64)


def test_ks_w1_empty_sample_is_nan(ssa):
    ha = torch.zeros(32, dtype=torch.int64, device="cuda")
    hb = torch.ones(32, dtype=torch.int64, device="cuda")
    out = ssa.hist_ks_w1(ha, hb).cpu().numpy()
    assert np.all(np.isnan(out))


@pytest.mark.parametrize("state_bytes", [4, 2])
def test_dwell_histogram_of_a_telegraph_ensemble(ssa, state_bytes):
    md = P.telegraph(0.3, 0.3, 20.0, 1.0)
    m = ssa.Model.from_dict(md)
    K = 257
    r = ssa.ensemble_run(m, 3001, P.TELEGRAPH_X0, 50.0, P.even_samples(50.0, K), "mixed_f16", "rn", seed=5,
                         max_events=10**6, state_bytes=state_bytes)
    snaps = r["snapshots"]
    h = ssa.dwell_histogram(snaps, 0)
    torch.cuda.synchronize()
    o = ost.dwell_histogram(snaps[:, 0, :].cpu().numpy())
    np.testing.assert_array_equal(h.cpu().numpy(), o)
    assert o.sum() > 1000


def test_ensemble_comparison_on_device(ssa):
    """KS / W1 between two precision modes' ensembles, on the device, equal
    the oracle's value on the same arrays."""
    md = P.schlogl()
    m = ssa.Model.from_dict(md)
    x0 = P.schlogl_x0(md)
    a = ssa.ensemble_run(m, 20000, x0, 2.0, [2.0], "fp32", "rn", True, seed=1, max_events=10**6)["snapshots"][0, 0]
    b = ssa.ensemble_run(m, 30000, x0, 2.0, [2.0], "uniform_bf16", "sr", True, seed=2,
                         max_events=10**6)["snapshots"][0, 0]
    bins = 4096
    ha, ca = ssa.count_histogram(a.contiguous(), bins)
    hb, cb = ssa.count_histogram(b.contiguous(), bins)
    out = ssa.hist_ks_w1(ha, hb).cpu().numpy()
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    D, W1 = ost.hist_ks_w1(ost.count_histogram(an, bins)[0], ost.count_histogram(bn, bins)[0])
    assert int(ca.item()) == 0 and int(cb.item()) == 0
    assert out[0] == D and out[1] == W1

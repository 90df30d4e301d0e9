"""Pins for the oracle's arithmetic primitives (CPU only).

Each primitive is checked against something other than itself: published
known-answer vectors, a library implementation, the IEEE-754 definition via
numpy/torch conversions, or exact rational arithmetic.
"""
import decimal
import os
import subprocess
import sys
import textwrap
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from oracle import stats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Known-answer vectors distributed with Random123 (Salmon et al., SC'11)
    for philox4x32 with 10 rounds."""
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        assert list(oracle.philox(ctr, key)[0]) == want


def test_philox_matches_triton_library():
    """Triton's Philox4x32-10 (run by its CPU interpreter) on counters
    (i, 0, 0, 0) and a 64-bit seed must equal the oracle's blocks."""
    pytest.importorskip("triton")
    script = textwrap.dedent("""
        import os, sys
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl
        @triton.jit
        def k(out_ptr, seed, n: tl.constexpr):
            offs = tl.arange(0, n)
            a, b, c, d = tl.randint4x(seed, offs)
            tl.store(out_ptr + offs * 4 + 0, a)
            tl.store(out_ptr + offs * 4 + 1, b)
            tl.store(out_ptr + offs * 4 + 2, c)
            tl.store(out_ptr + offs * 4 + 3, d)
        out = torch.zeros(64 * 4, dtype=torch.int32)
        k[(1,)](out, int(sys.argv[1]), 64)
        print(" ".join(str(v) for v in out.numpy().view(np.uint32)))
    """)
    seed = 0x0123456789ABCDEF
    res = subprocess.run([sys.executable, "-c", script, str(seed)], capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-200:])
    got = np.array([int(v) for v in res.stdout.split()], dtype=np.uint32).reshape(64, 4)
    want = oracle.philox([0, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32], 64)
    np.testing.assert_array_equal(got, want)


# ------------------------------------------------------- 16-bit conversions
def _patterns(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    # add every binary32 pattern whose low 16 bits are a tie or a tie +- 1
    hi = np.arange(0, 2**16, dtype=np.uint32) << 16
    ties = np.concatenate([hi | 0x1000, hi | 0x0FFF, hi | 0x1001, hi | 0x8000, hi | 0x7FFF, hi | 0x8001,
                           hi | 0x3000, hi | 0x2000])
    return np.concatenate([u, ties]).view(np.float32)


def test_f16_round_to_nearest_matches_numpy():
    x = _patterns(2_000_000, 1)
    with np.errstate(over="ignore", invalid="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    got = oracle.f32_to_f16(x)
    nan = np.isnan(x)
    np.testing.assert_array_equal(got[~nan], ref[~nan])
    assert np.all(np.isnan(got[nan].view(np.float16)))


def test_bf16_round_to_nearest_matches_torch():
    x = _patterns(2_000_000, 2)
    ref = torch.from_numpy(x.copy()).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = oracle.f32_to_bf16(x)
    nan = np.isnan(x)
    np.testing.assert_array_equal(got[~nan], ref[~nan])


def test_f16_widening_all_patterns():
    h = np.arange(65536, dtype=np.uint16)
    ref = h.view(np.float16).astype(np.float32)
    got = oracle.f16_to_f32(h)
    ok = ~np.isnan(ref)
    np.testing.assert_array_equal(got.view(np.uint32)[ok], ref.view(np.uint32)[ok])


def _neighbours_f16(x):
    """(x-, x+): the binary16 values adjacent to |x| toward and away from zero.
    Above the largest finite value 65504, x+ is infinity."""
    ax = abs(float(x))
    if ax >= 65504.0:
        return 65504.0, np.inf
    h = np.float16(ax)
    if float(h) > ax:
        h = np.nextafter(h, np.float16(0))
    return float(h), float(np.nextafter(h, np.float16(np.inf)))


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_stochastic_rounding_probability_is_exact(fmt):
    """SR equation of Sec. 3.3: P(round away) = (x - x-)/(x+ - x-).  With R
    random bits the count of rounding-up draws over all 2^R values must be
    floor(2^R (x - x-)/(x+ - x-)), exactly (R = 13 for binary16, 16 for
    bfloat16; exact whenever the discarded fraction has <= R bits)."""
    rng = np.random.default_rng(11)
    xs = []
    for e in range(-30, 16):   # binary16 subnormal, normal and overflow edge
        xs += list((rng.random(4) + 1.0) * 2.0 ** e)
    xs += [65504.5, 65519.0, 65535.9, 3.0e-8, 1.0e-9, 0.1, 1.0 / 3.0]
    xs = np.array(xs, dtype=np.float32)
    xs = np.concatenate([xs, -xs[:20]])
    R = 13 if fmt == "f16" else 16
    r = np.arange(2**R, dtype=np.uint32)
    for x in xs:
        xv = np.full(r.shape, x, dtype=np.float32)
        if fmt == "f16":
            out = oracle.f32_to_f16(xv, sr=True, r=r).view(np.float16).astype(np.float64)
            lo, hi = _neighbours_f16(x)
        else:
            out = oracle.f32_to_bf16(xv, sr=True, r=r)
            out = (out.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
            b = np.float32(abs(x)).view(np.uint32) & np.uint32(0xFFFF0000)
            lo = float(np.uint32(b).view(np.float32))
            hi = float(np.uint32(b + 0x10000).view(np.float32))
        sgn = -1.0 if x < 0 else 1.0
        vals = set(np.unique(np.abs(out)).tolist())
        assert vals <= {lo, hi}, (x, vals, lo, hi)
        frac = (Fraction(abs(float(x))) - Fraction(lo)) / (Fraction(hi) - Fraction(lo)) if np.isfinite(hi) \
            else (Fraction(abs(float(x))) - Fraction(lo)) / (Fraction(65536) - Fraction(lo))
        want = int(frac * 2**R)   # floor
        ups = int(np.sum(np.abs(out) == hi))
        assert ups == want, (x, ups, want)
        assert np.all(np.sign(out[out != 0]) == sgn)


def test_stochastic_rounding_keeps_representable_values():
    rng = np.random.default_rng(5)
    h = rng.integers(0, 0x7C00, size=4000).astype(np.uint16)
    x = h.view(np.float16).astype(np.float32)
    r = rng.integers(0, 2**32, size=x.size, dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(oracle.f32_to_f16(x, sr=True, r=r), h)
    b = (x.view(np.uint32) & 0xFFFF0000).view(np.float32)
    np.testing.assert_array_equal(oracle.f32_to_bf16(b, sr=True, r=r), (b.view(np.uint32) >> 16).astype(np.uint16))


def test_stochastic_rounding_overflow_gives_infinity():
    r = np.array([0x1FFF], dtype=np.uint32)
    assert oracle.f32_to_f16(np.array([65535.0], np.float32), sr=True, r=r)[0] == 0x7C00
    assert oracle.f32_to_f16(np.array([65535.0], np.float32), sr=True, r=np.array([0], np.uint32))[0] == 0x7BFF
    assert oracle.f32_to_f16(np.array([1e6], np.float32), sr=True, r=np.array([0], np.uint32))[0] == 0x7C00


# ------------------------------------------------------------------ log
def test_log_f32_error_bound():
    """|log32(x) - ln x| <= 2 ulp over (0, 1] (uniform variates) and beyond."""
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.random(400_000).astype(np.float32),
                        (np.float32(1) - rng.random(2000).astype(np.float32) * np.float32(1e-5)),
                        (rng.random(20000) * 1e4).astype(np.float32),
                        np.array([2.0**-24, 1.0, 0.5, 2.0, np.sqrt(0.5), np.sqrt(2.0)], np.float32)])
    x = x[x > 0]
    got = oracle.log_f32(x).astype(np.float64)
    ref = np.log(x.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    nz = ref != 0
    assert np.max(np.abs(got[nz] - ref[nz]) / ulp[nz]) <= 2.0
    assert np.all(got[~nz] == 0)


def test_log_f64_error_bound():
    """|log64(x) - ln x| <= 2 ulp against 50-digit decimal logarithms."""
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.random(3000), 1 - rng.random(200) * 1e-9, [2.0**-53, 2.0**-32, 1.0, 0.5, 2.0]])
    got = oracle.log_f64(x)
    decimal.getcontext().prec = 50
    worst = 0.0
    for g, v in zip(got, x):
        ref = decimal.Decimal(float(v)).ln()
        if ref == 0:
            assert g == 0.0
            continue
        err = abs(decimal.Decimal(float(g)) - ref) / decimal.Decimal(float(np.spacing(abs(float(ref)))))
        worst = max(worst, float(err))
    assert worst <= 2.0


# ----------------------------------------------------------- statistics
def test_ks_and_wasserstein_match_scipy():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(0)
    for lam_b in (20.0, 20.4, 23.0):
        a = rng.poisson(20.0, 5000)
        b = rng.poisson(lam_b, 3000)
        D, p = stats.ks_2samp(a, b)
        ref = scipy_stats.ks_2samp(a, b)
        assert abs(D - ref.statistic) < 1e-12
        ne = 5000 * 3000 / 8000
        assert abs(p - scipy_stats.kstwobign.sf(D * np.sqrt(ne))) < 1e-9
        assert abs(stats.wasserstein1(a, b) - scipy_stats.wasserstein_distance(a, b)) < 1e-9


def test_histogram_statistics_against_scipy_and_brute_force():
    """The histogram form of KS and W1 equals scipy's sample-based values on
    integer data; the dwell extraction equals an interval search written
    differently (runs of equal values)."""
    import scipy.stats as scipy_stats
    from oracle import stats as ost
    rng = np.random.default_rng(5)
    for na, nb, lam1, lam2 in [(500, 700, 20.0, 21.5), (3000, 2000, 3.0, 3.0), (50, 4000, 100.0, 80.0)]:
        a = rng.poisson(lam1, na)
        b = rng.poisson(lam2, nb)
        bins = int(max(a.max(), b.max())) + 3
        ha, ca = ost.count_histogram(a, bins)
        hb, cb = ost.count_histogram(b, bins)
        assert ca == cb == 0 and ha.sum() == na and hb.sum() == nb
        D, W1 = ost.hist_ks_w1(ha, hb)
        assert abs(D - scipy_stats.ks_2samp(a, b).statistic) < 1e-12
        assert abs(W1 - scipy_stats.wasserstein_distance(a, b)) < 1e-12
    h, c = ost.count_histogram([-3, 0, 5, 9, 12], 10)
    assert c == 2 and h[0] == 2 and h[9] == 2 and h[5] == 1
    assert np.isnan(ost.hist_ks_w1(np.zeros(4), np.ones(4))[0])
    # dwell: runs of OFF (nonzero) bounded by ON samples on both sides
    s = rng.integers(0, 2, size=(60, 40))
    want = np.zeros(60, dtype=np.int64)
    for j in range(40):
        col = s[:, j] != 0
        runs, k = [], 0
        while k < 60:
            e = k
            while e + 1 < 60 and col[e + 1] == col[k]:
                e += 1
            runs.append((col[k], k, e))
            k = e + 1
        for idx, (off, k0, k1) in enumerate(runs):
            if off and idx > 0 and idx + 1 < len(runs):
                want[k1 - k0 + 1] += 1
    np.testing.assert_array_equal(ost.dwell_histogram(s), want)

"""The engine's 16-bit rounding step against the oracle's emulation (paper
Sec. 3.1 formats, Sec. 3.3 stochastic rounding), value by value.

ssa_round16 applies the kernels' own device functions (cvt.rn and cvt.rs on
sm_103a) to arrays.  The oracle rounds with integer operations on bit
patterns (reading R5: 13 random bits of resolution for binary16, 16 for
bfloat16).  Parity is exact: for each sampled x every one of the 2^16 random
values is tried, in both halves of the random word, so the probability of
rounding up, the bits used and their alignment are compared completely.
The inputs cover normal values in several binades, binary16 subnormal
results and values below its smallest subnormal, the 65504 -> infinity edge,
both signs, values that are exactly representable (they must never move),
zeros and infinities.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    mod.lib()
    return mod


def _oracle_round(x, fmt, sr, r):
    if fmt == "f16":
        return oracle.f16_to_f32(oracle.f32_to_f16(x, sr=sr, r=r))
    h = oracle.f32_to_bf16(x, sr=sr, r=r)
    return (h.astype(np.uint32) << 16).view(np.float32)


def _inputs(fmt):
    rng = np.random.default_rng(11 if fmt == "f16" else 12)
    xs = []
    xs += list(rng.uniform(1.0, 2.0, 6))
    xs += list(rng.uniform(250.0, 2100.0, 4))                  # counts where the chains round
    xs += list(np.exp(rng.uniform(-20, 20, 8)))
    if fmt == "f16":
        xs += [65504.0, 65519.0, 65520.0, 65535.9, 65000.5]    # last binade and the overflow edge
        xs += list(rng.uniform(2.0**-24, 2.0**-14, 6))           # subnormal results
        xs += [2.0**-25, 2.0**-24 * 0.75, 2.0**-30, 3 * 2.0**-25, 2.0**-14 * 0.999]
        xs += [1.0 + 2.0**-10, 2.0**-14, 2.0**-24, 2048.0]      # exactly representable
    else:
        big = np.float32(np.finfo(np.float32).max)
        xs += [float(big), float(np.float32(3.389e38)), 1e38]  # bfloat16 overflow edge
        xs += list(np.exp(rng.uniform(-85, -80, 3)))            # binary32 subnormal range
        xs += [1.0 + 2.0**-7, 256.0, 3.0 * 2.0**100]            # exactly representable
    xs = np.array(xs, dtype=np.float32)
    xs = np.concatenate([xs, -xs[::3], np.array([0.0, -0.0, np.inf, -np.inf], np.float32)])
    return xs.astype(np.float32)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_stochastic_rounding_every_random_value(ssa, fmt):
    xs = _inputs(fmt)
    r16 = np.arange(1 << 16, dtype=np.uint32)
    x = np.repeat(xs, r16.size)
    r = np.tile(r16, xs.size)
    expect = _oracle_round(x, fmt, True, r)
    xd = torch.from_numpy(x).cuda()
    for half in (0, 1):
        words = (r << 16) if half else (r | (np.uint32(0xA5A5) << 16))   # the other half holds noise
        got = ssa.round16(xd, torch.from_numpy(words.view(np.int32)).cuda(), fmt, "sr", half).cpu().numpy()
        np.testing.assert_array_equal(got.view(np.uint32), expect.view(np.uint32))
    # Sec. 3.3's probability, from the values alone: per finite x below the
    # largest finite 16-bit value, the number of the 2^16 words that round
    # |x| up is floor(2^R (|x| - x-)/(x+ - x-)) 2^(16-R), R = 13 (binary16)
    # or 16 (bfloat16); x+ - x- is a power of two, so the quotient is exact.
    ax = np.abs(xs.astype(np.float64))
    if fmt == "f16":
        R, top = 13, 65504.0
        with np.errstate(all="ignore"):   # values beyond binary16 are masked out below
            lo = np.abs(xs).astype(np.float16).astype(np.float64)
            lo = np.where(lo > ax, np.nextafter(lo.astype(np.float16), np.float16(0)).astype(np.float64), lo)
            hi = np.nextafter(lo.astype(np.float16), np.float16(np.inf)).astype(np.float64)
    else:
        R, top = 16, float((np.uint32(0x7F7F) << 16).view(np.float32))
        u = np.abs(xs).view(np.uint32)
        lo = (u & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
        hi = ((u & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    ok = np.isfinite(ax) & (ax < top)
    frac = (ax[ok] - lo[ok]) / (hi[ok] - lo[ok])
    expect_up = np.floor(frac * 2.0**R) * 2.0 ** (16 - R)
    up = (np.abs(got.reshape(xs.size, -1)[ok].astype(np.float64)) > lo[ok][:, None]).sum(axis=1)
    np.testing.assert_array_equal(up, expect_up)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_round_to_nearest_random_patterns(ssa, fmt):
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2**32, size=1 << 21, dtype=np.uint64).astype(np.uint32)
    x = bits.view(np.float32)
    x = x[~np.isnan(x)]
    # every binary16 and bfloat16 tie (exact midpoints between neighbours)
    if fmt == "f16":
        h = np.arange(0x7BFF, dtype=np.uint16)
        lo = oracle.f16_to_f32(h).astype(np.float64)
        hi = oracle.f16_to_f32(h + 1).astype(np.float64)
    else:
        h = np.arange(0x7F7F, dtype=np.uint32)
        lo = (h << 16).view(np.float32).astype(np.float64)
        hi = ((h + 1) << 16).view(np.float32).astype(np.float64)
    ties = ((lo + hi) / 2).astype(np.float32)
    x = np.concatenate([x, ties, -ties]).astype(np.float32)
    got = ssa.round16(torch.from_numpy(x).cuda(), None, fmt, "rn").cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), _oracle_round(x, fmt, False, None).view(np.uint32))
    if fmt == "f16":   # and the library conversion
        ref = x.astype(np.float16).astype(np.float32)
        np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_round16_rejects_bad_arguments(ssa):
    x = torch.zeros(4, device="cuda")
    for args in ((x, None, 7, 0, 0), (x, None, 0, 1, 0), (x, None, 0, 0, 2)):
        rc = ssa.lib().ssa_round16(ssa._dev_ptr(args[0]), None, 4, args[2], args[3], args[4], ssa._dev_ptr(x), None)
        assert rc == ssa.SSA_EINVAL

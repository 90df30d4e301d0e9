"""Pins of the oracle's RDME (reaction-diffusion master equation on a lattice,
the spatial setting the paper names in Sec. 1 and Sec. 5) against facts that do
not come from the oracle:

* one voxel: operation for operation the well-mixed direct method (Sec. 2),
  whose own oracle is pinned separately;
* pure diffusion: independent random walkers, so each voxel's count is
  Binomial(n0, p_v(t)) with p(t) the walker's law exp(tQ) (matrix exponential
  of the hop generator), in one, two and three dimensions;
* birth, death and diffusion (linear): surviving initial molecules are
  binomial, newborn ones Poisson, giving closed-form means and variances;
* conservation: walkers, and A + 2B under dimerisation with diffusion, in
  every precision mode including stochastic rounding.
"""
import numpy as np
import pytest
from scipy import linalg, stats

import oracle
from paper_2605_00479_gb300 import presets as P

MODES = [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_f16", "sr"), ("mixed_bf16", "rn"),
         ("mixed_bf16", "sr"), ("uniform_f16", "rn"), ("uniform_f16", "sr"), ("uniform_bf16", "rn"),
         ("uniform_bf16", "sr")]


def walker_generator(dims, D):
    """Generator Q of one walker hopping at rate D to each existing neighbour."""
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    S = nx * ny * nz
    Q = np.zeros((S, S))
    for v in range(S):
        ix, iy, iz = v % nx, (v // nx) % ny, v // (nx * ny)
        for dx, dy, dz in [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
            jx, jy, jz = ix + dx, iy + dy, iz + dz
            if 0 <= jx < nx and 0 <= jy < ny and 0 <= jz < nz:
                w = jx + nx * (jy + ny * jz)
                Q[v, w] += D
                Q[v, v] -= D
    return Q


def inert(n=1):
    """n species, one zero-rate reaction (diffusion only)."""
    return {"order": np.zeros((1, n), np.int32), "stoich": np.zeros((1, n), np.int32), "rate": np.array([0.0])}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_f16", "mixed_bf16", "uniform_f16", "uniform_bf16"])
@pytest.mark.parametrize("name", ["dimer", "schlogl", "repressilator"])
def test_single_voxel_is_the_well_mixed_method(name, prec):
    if name == "dimer":
        m, x0, t_end, norm = P.dimer(), P.dimer_x0(300), 20.0, False
    elif name == "schlogl":
        m, x0, t_end, norm = P.schlogl(), P.schlogl_x0(P.schlogl()), 2.0, True
    else:
        m, x0, t_end, norm = P.repressilator(), P.REPRESSILATOR_X0, 5.0, False
    N = len(x0)
    const = m.get("constant")
    D = np.full(N, 0.7) if const is None else np.where(np.asarray(const) != 0, 0.0, 0.7)
    samples = P.even_samples(t_end, 6)
    cap = 40000          # stagnating uniform-mode clocks reach it: MAX_EVENTS paths are compared too
    a = oracle.run(m, x0, 40, t_end, samples, precision=prec, rounding="rn", normalise=norm, seed=9, max_events=cap)
    b = oracle.rdme_run(m, (1,), D, x0, 40, t_end, samples, precision=prec, rounding="rn", normalise=norm, seed=9,
                        max_events=cap)
    np.testing.assert_array_equal(a["snapshots"], b["snapshots"][:, 0])
    np.testing.assert_array_equal(a["status"], b["status"])
    np.testing.assert_array_equal(a["n_events"], b["n_events"])
    np.testing.assert_array_equal(a["t_final"].view(np.uint64), b["t_final"].view(np.uint64))


@pytest.mark.parametrize("dims,D,t", [((8,), 1.0, 1.5), ((4, 3), 0.5, 2.0), ((3, 2, 2), 0.8, 1.0)])
def test_pure_diffusion_is_binomial(dims, D, t):
    S = int(np.prod(dims))
    n0, n = 30, 6000
    x0 = np.zeros((S, 1), np.int32)
    x0[0, 0] = n0
    r = oracle.rdme_run(inert(), dims, [D], x0, n, t, [t], seed=4)
    x = r["snapshots"][0, :, 0, :].astype(np.int64)          # [S, n]
    assert np.all(x.sum(axis=0) == n0)
    p = linalg.expm(t * walker_generator(dims, D))[0]
    for v in range(S):
        mean, var = n0 * p[v], n0 * p[v] * (1 - p[v])
        assert abs(x[v].mean() - mean) < 5 * np.sqrt(var / n) + 1e-9, (v, x[v].mean(), mean)
        if var > 1:
            assert abs(x[v].var() - var) < 6 * np.sqrt(2 * var * var / n) + 0.05 * var, (v, x[v].var(), var)
    # full law of the corner voxel by chi-square against Binomial(n0, p_0)
    k = np.arange(n0 + 1)
    pmf = stats.binom.pmf(k, n0, p[0])
    keep = pmf * n >= 5
    obs = np.bincount(x[0], minlength=n0 + 1)
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(pmf[keep] * n, pmf[~keep].sum() * n)
    if e[-1] < 5:
        o[-2] += o[-1]; e[-2] += e[-1]; o, e = o[:-1], e[:-1]
    assert stats.chisquare(o, e).pvalue > 1e-4


def test_birth_death_diffusion_moments():
    """0 -> X at k per voxel, X -> 0 at gamma, hops at D; n0 molecules start in
    voxel 0.  x_v(t) = Binomial(n0, e^{-gamma t} p_v(t)) + Poisson((k/gamma)(1 - e^{-gamma t}))."""
    k, g, D, t, n0, n = 2.0, 0.5, 0.7, 1.2, 20, 8000
    dims = (6,)
    m = P.birth_death(k, g)
    x0 = np.zeros((6, 1), np.int32)
    x0[0, 0] = n0
    r = oracle.rdme_run(m, dims, [D], x0, n, t, [t], seed=21)
    x = r["snapshots"][0, :, 0, :].astype(np.float64)
    p = linalg.expm(t * walker_generator(dims, D))[0]
    surv = np.exp(-g * t)
    lam = k / g * (1 - surv)
    for v in range(6):
        q = surv * p[v]
        mean, var = n0 * q + lam, n0 * q * (1 - q) + lam
        assert abs(x[v].mean() - mean) < 5 * np.sqrt(var / n), (v, x[v].mean(), mean)
        assert abs(x[v].var() - var) < 6 * np.sqrt((var + 2 * var * var) / n), (v, x[v].var(), var)
    tot = x.sum(axis=0)
    mt, vt = n0 * surv + 6 * lam, n0 * surv * (1 - surv) + 6 * lam
    assert abs(tot.mean() - mt) < 5 * np.sqrt(vt / n)


@pytest.mark.parametrize("prec,rnd", MODES)
def test_conservation_in_every_mode(prec, rnd):
    """Hops move molecules and A + A <-> B keeps A + 2B: both totals are
    conserved at every snapshot in every precision mode."""
    m = P.dimer(2e-2, 0.1)
    dims = (3, 3)
    x0 = np.zeros((9, 2), np.int32)
    x0[4, 0] = 60
    x0[0, 0] = 20
    r = oracle.rdme_run(m, dims, [0.5, 0.2], x0, 60, 5.0, P.even_samples(5.0, 6), precision=prec, rounding=rnd,
                        seed=17, max_events=200000)
    snaps = r["snapshots"].astype(np.int64)          # [K, S, N, n]
    total = snaps[:, :, 0, :].sum(axis=1) + 2 * snaps[:, :, 1, :].sum(axis=1)
    assert np.all(total == 80)
    assert snaps.min() >= 0
    assert np.all((r["status"] & ~np.uint32(2)) == 0)
    assert r["n_events"].min() > 0


@pytest.mark.parametrize("prec,rnd", [("mixed_f16", "sr"), ("uniform_f16", "sr"), ("uniform_bf16", "sr"),
                                      ("fp32", "rn")])
def test_diffusion_profile_in_reduced_precision(prec, rnd):
    """The walker law survives reduced precision with SR (means within 5 sigma
    plus a small rounding allowance)."""
    dims, D, t, n0, n = (5,), 1.0, 1.0, 30, 4000
    x0 = np.zeros((5, 1), np.int32)
    x0[2, 0] = n0
    r = oracle.rdme_run(inert(), dims, [D], x0, n, t, [t], precision=prec, rounding=rnd, seed=8)
    x = r["snapshots"][0, :, 0, :].astype(np.float64)
    p = linalg.expm(t * walker_generator(dims, D))[2]
    for v in range(5):
        mean, var = n0 * p[v], n0 * p[v] * (1 - p[v])
        assert abs(x[v].mean() - mean) < 5 * np.sqrt(var / n) + 0.02 * mean, (prec, v, x[v].mean(), mean)
    assert np.all(x.sum(axis=0) == n0)


def test_stationary_walkers_are_uniform():
    dims, D, n0, n = (2, 2), 2.0, 12, 4000
    x0 = np.zeros((4, 1), np.int32)
    x0[3, 0] = n0
    r = oracle.rdme_run(inert(), dims, [D], x0, n, 20.0, [20.0], seed=2)
    x = r["snapshots"][0, :, 0, :]
    for v in range(4):
        assert abs(x[v].mean() - n0 / 4) < 5 * np.sqrt(n0 * 0.25 * 0.75 / n)


def test_rejects_invalid_lattices():
    m = P.birth_death()
    with pytest.raises(ValueError):
        oracle.rdme_run(m, (0,), [1.0], [[0]], 1, 1.0, [1.0])
    with pytest.raises(ValueError):
        oracle.rdme_run(m, (2,), [-1.0], [[0], [0]], 1, 1.0, [1.0])
    with pytest.raises(ValueError):
        oracle.rdme_run(m, (2,), [1.0], [[0], [0]], 1, 1.0, [1.0], precision="fp64", rounding="sr")

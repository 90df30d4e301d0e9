"""Longest-first scheduling of the direct method: launch 1 runs every
trajectory up to the parking point and parks the unfinished ones, three
kernels order them by predicted remaining work, launch 2 resumes them largest
first.  A parked trajectory resumes whole and random numbers are keyed by
(trajectory id, event count), so every output must equal the oracle (and the
unsplit run) bit for bit, whatever the parking point, launch shape, storage
format or species mask."""
import numpy as np
import pytest

import oracle
from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    assert torch.cuda.is_available()
    mod.lib()
    yield mod
    mod.set_longest_first()


def general_network():
    """Matches no compiled structure (general kernel, runtime loops)."""
    return {
        "order": np.array([[1, 0, 1], [2, 0, 0], [0, 1, 0], [0, 3, 0], [0, 0, 0], [1, 0, 0]], np.int32),
        "stoich": np.array([[1, 0, -1], [-2, 1, 0], [1, -1, 0], [0, -3, 0], [0, 1, 0], [-1, 0, 0]], np.int32),
        "rate": np.array([0.02, 0.01, 0.5, 0.001, 2.0, 0.1]),
        "law": np.zeros(6, np.int32),
        "constant": np.array([0, 0, 1], np.uint8),
    }


CASES = {
    # name: (model, x0, n_traj, t_end, samples, normalise, max_events, precision, rounding, park_events)
    "schlogl_uniform_f16_sr": (P.schlogl(), None, 20000, 2.0, P.even_samples(2.0, 5), True, 10**6,
                               "uniform_f16", "sr", 64),
    "schlogl_mixed_bf16_rn": (P.schlogl(), None, 20000, 2.0, P.even_samples(2.0, 9), True, 10**6,
                              "mixed_bf16", "rn", 2048),
    "schlogl_uniform_bf16_rn_capped": (P.schlogl(), None, 9000, 2.0, P.even_samples(2.0, 5), True, 3000,
                                       "uniform_bf16", "rn", 2998),
    "telegraph_mixed_bf16_sr": (P.telegraph(0.5, 0.5, 20.0, 1.0), P.TELEGRAPH_X0, 12000, 20.0,
                                P.even_samples(20.0, 7), False, 10**6, "mixed_bf16", "sr", 100),
    "repressilator_fp32": (P.repressilator(), P.REPRESSILATOR_X0, 3000, 2.0, P.even_samples(2.0, 3), False,
                           10**6, "fp32", "rn", 128),
    "general_uniform_f16_sra": (general_network(), [10, 5, 50], 8000, 20.0, P.even_samples(20.0, 5), True,
                                10**6, "uniform_f16", "sra", 32),
    "dimer_fp64": (P.dimer(), P.dimer_x0(300), 4000, 5.0, P.even_samples(5.0, 4), False, 10**6, "fp64", "rn", 64),
    "birth_death_mixed_f16_rn": (P.birth_death(), [0], 30000, 30.0, P.even_samples(30.0, 6), False, 10**6,
                                 "mixed_f16", "rn", 2),
    "hill_general_uniform_bf16_sr": (P.hill_self(1.0, 30.0, 2, 1.0), [0], 12000, 20.0, P.even_samples(20.0, 5),
                                     False, 10**6, "uniform_bf16", "sr", 40),
}

_ORACLE = {}


def oracle_case(name, seed, state_bytes=4, out_species=0):
    key = (name, seed, state_bytes, out_species)
    if key not in _ORACLE:
        md, x0, n, t_end, samples, norm, cap, prec, rnd, _ = CASES[name]
        x0 = P.schlogl_x0(md) if x0 is None else x0
        _ORACLE[key] = oracle.run_parallel(md, x0, n, t_end, samples, precision=prec, rounding=rnd, normalise=norm,
                                           seed=seed, max_events=cap, state_bytes=state_bytes,
                                           out_species=out_species)
    return _ORACLE[key]


def gpu_run(ssa, name, seed, mode, park, state_bytes=4, out_species=0):
    md, x0, n, t_end, samples, norm, cap, prec, rnd, _ = CASES[name]
    x0 = P.schlogl_x0(md) if x0 is None else x0
    m = ssa.Model.from_dict(md)
    ssa.set_longest_first(mode, park)
    try:
        before = ssa.direct_kernel_launches()
        r = ssa.ensemble_run(m, n, x0, t_end, samples, prec, rnd, norm, seed, cap, state_bytes,
                             out_species=out_species)
        torch.cuda.synchronize()
        launched = ssa.direct_kernel_launches() - before
    finally:
        ssa.set_longest_first()
    return {k: v.cpu().numpy() for k, v in r.items()}, launched


def assert_same(g, o):
    np.testing.assert_array_equal(g["snapshots"], o["snapshots"])
    np.testing.assert_array_equal(g["status"].view(np.uint32), np.asarray(o["status"]).view(np.uint32))
    np.testing.assert_array_equal(g["n_events"], o["n_events"])
    gt, ot = g["t_final"], o["t_final"]
    both_nan = np.isnan(gt) & np.isnan(ot)
    np.testing.assert_array_equal(gt.view(np.uint64)[~both_nan], ot.view(np.uint64)[~both_nan])


@pytest.mark.parametrize("name", list(CASES))
def test_split_run_matches_oracle(ssa, name):
    """Forced split at the case's parking point: five kernels, results equal
    the oracle, and parking really happened (some trajectory ran past it)."""
    park = CASES[name][-1]
    o = oracle_case(name, 43)
    g, launched = gpu_run(ssa, name, 43, 2, park)
    assert launched == 5
    assert (o["n_events"] > park).any(), "no trajectory reached the parking point"
    assert_same(g, o)


@pytest.mark.parametrize("block,blocks_per_sm,slice_pairs,compaction",
                         [(256, 1, 1, True), (128, 0, 16, False), (64, 2, 3, True)])
@pytest.mark.parametrize("name", ["schlogl_uniform_f16_sr", "general_uniform_f16_sra", "telegraph_mixed_bf16_sr"])
def test_split_run_independent_of_launch_shape(ssa, name, block, blocks_per_sm, slice_pairs, compaction):
    park = CASES[name][-1]
    o = oracle_case(name, 43)
    try:
        ssa.set_launch_config(block, blocks_per_sm, slice_pairs)
        ssa.set_tail_compaction(compaction)
        g, launched = gpu_run(ssa, name, 43, 2, park)
    finally:
        ssa.set_tail_compaction(True)
        ssa.set_launch_config()
    assert launched == 5
    assert_same(g, o)


@pytest.mark.parametrize("park", [2, 6, 1000, 50000])
def test_parking_points(ssa, park):
    """From the first step pair to beyond every trajectory's length (then
    nothing is parked and launch 2 finds an empty order)."""
    name = "schlogl_mixed_bf16_rn"
    o = oracle_case(name, 43)
    g, launched = gpu_run(ssa, name, 43, 2, park)
    assert launched == 5
    assert_same(g, o)


def test_parking_point_at_or_beyond_the_cap_runs_one_launch(ssa):
    name = "schlogl_uniform_bf16_rn_capped"   # max_events 3000
    o = oracle_case(name, 43)
    g, launched = gpu_run(ssa, name, 43, 2, 3000)
    assert launched == 1
    assert_same(g, o)
    # two events below the cap: trajectories park, resume and stop at the cap
    g, launched = gpu_run(ssa, name, 43, 2, 2998)
    assert launched == 5
    assert (np.asarray(o["status"]) & 2).any()
    assert_same(g, o)


def test_off_and_automatic_modes_on_small_runs(ssa):
    """Automatic mode leaves small ensembles in one launch; off never splits."""
    name = "schlogl_mixed_bf16_rn"
    o = oracle_case(name, 43)
    for mode in (0, 1):
        g, launched = gpu_run(ssa, name, 43, mode, 0)
        assert launched == 1
        assert_same(g, o)


@pytest.mark.parametrize("state_bytes,out_species", [(2, 0), (4, 0b001), (2, 0b101)])
def test_split_run_storage_and_species_mask(ssa, state_bytes, out_species):
    name = "schlogl_uniform_f16_sr"
    o = oracle_case(name, 43, state_bytes, out_species)
    g, launched = gpu_run(ssa, name, 43, 2, 64, state_bytes, out_species)
    assert launched == 5
    assert_same(g, o)


@pytest.mark.parametrize("pinned", [False, True])
def test_split_run_through_the_host_entry_point(ssa, pinned):
    """ssa_ensemble_run_host splits the same way (device staging for
    pageable outputs; this sparse snapshot stream goes straight into
    page-locked ones)."""
    name = "schlogl_uniform_f16_sr"
    md, x0, n, t_end, samples, norm, cap, prec, rnd, park = CASES[name]
    x0 = P.schlogl_x0(md) if x0 is None else x0
    o = oracle_case(name, 43)
    m = ssa.Model.from_dict(md)
    K = len(samples)
    if pinned:
        bufs = [torch.empty((K, m.N, n), dtype=torch.int32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory(),
                torch.empty(n, dtype=torch.int64).pin_memory(), torch.empty(n, dtype=torch.float64).pin_memory()]
        out, st, ev, tf = (b.numpy() for b in bufs)
        st = st.view(np.uint32)
    else:
        out = st = ev = tf = None
    ssa.set_longest_first(2, park)
    try:
        before = ssa.direct_kernel_launches()
        r = ssa.ensemble_run_host(m, n, x0, t_end, samples, prec, rnd, norm, 43, cap, 4, out=out, status=st,
                                  n_events=ev, t_final=tf)
        launched = ssa.direct_kernel_launches() - before
    finally:
        ssa.set_longest_first()
    assert launched == 5
    assert_same(r, o)


@pytest.mark.parametrize("prec,rnd", [("mixed_bf16", "rn"), ("uniform_f16", "sr")])
def test_full_size_schlogl_split_equals_unsplit(ssa, prec, rnd):
    """The benchmark's workload (10^6 trajectories, t_end = 10, 50 snapshots
    of X): the automatic mode splits it, and the whole ensemble equals the
    unsplit run; sampled ids equal the oracle."""
    md = P.schlogl()
    x0 = P.schlogl_x0(md)
    samples = P.even_samples(10.0, 50)
    m = ssa.Model.from_dict(md)
    res = {}
    for mode in (1, 0):
        ssa.set_longest_first(mode, 0)
        try:
            before = ssa.direct_kernel_launches()
            r = ssa.ensemble_run(m, 10**6, x0, 10.0, samples, prec, rnd, True, 77, 200000, out_species=0b001)
            torch.cuda.synchronize()
            res[mode] = ({k: v.cpu().numpy() for k, v in r.items()}, ssa.direct_kernel_launches() - before)
        finally:
            ssa.set_longest_first()
    assert res[1][1] == 5 and res[0][1] == 1
    assert_same(res[1][0], res[0][0])
    on = res[1][0]
    for i in [0, 4099, 523456, 999999]:
        o = oracle.run(md, x0, 1, 10.0, samples, prec, rnd, True, 77, 200000, g0=i, out_species=0b001)
        np.testing.assert_array_equal(on["snapshots"][:, :, i], o["snapshots"][:, :, 0])
        assert on["n_events"][i] == o["n_events"][0]

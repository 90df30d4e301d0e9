"""Batched heterogeneous runs (one persistent launch over several model
groups with parameter sweeps) against the oracle, set by set."""
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
    mod.lib()
    return mod


def sweep_groups(ssa, n_sets=(6, 5, 3), traj=(50, 40, 20)):
    tel = P.telegraph()
    tr = P.telegraph_sweep(n_sets[0], seed=11)
    dm = P.dimer()
    dr = P.dimer_sweep(n_sets[1], seed=12)
    rp = P.repressilator()
    rr, rh = P.repressilator_sweep(n_sets[2], seed=13)
    groups = [
        # longest trajectories first
        {"dict": rp, "model": ssa.Model.from_dict(rp), "x0": np.tile(P.REPRESSILATOR_X0, (n_sets[2], 1)),
         "rates": rr, "hill": rh[:, :, :2], "traj_per_set": traj[2], "traj_offset": 0},
        {"dict": tel, "model": ssa.Model.from_dict(tel), "x0": np.tile(P.TELEGRAPH_X0, (n_sets[0], 1)),
         "rates": tr, "traj_per_set": traj[0], "traj_offset": 10**6},
        {"dict": dm, "model": ssa.Model.from_dict(dm), "x0": np.tile(P.dimer_x0(300), (n_sets[1], 1)),
         "rates": dr, "traj_per_set": traj[1], "traj_offset": 2 * 10**6},
    ]
    return groups


def oracle_group(G, t_end, samples, prec, rnd, norm, seed, cap):
    parts = []
    for q in range(G["x0"].shape[0]):
        md = dict(G["dict"])
        if G.get("rates") is not None:
            md["rate"] = np.asarray(G["rates"][q], dtype=np.float64)
        if G.get("hill") is not None:
            h = np.array(md["hill"], dtype=np.float64, copy=True)
            h[:, :2] = G["hill"][q]
            md["hill"] = h
        parts.append(oracle.run(md, G["x0"][q], G["traj_per_set"], t_end, samples, prec, rnd, norm, seed, cap,
                                g0=G["traj_offset"] + q * G["traj_per_set"]))
    return {k: np.concatenate([p[k] for p in parts], axis=-1) for k in parts[0]}


def check(batch, groups, t_end, samples, prec, rnd, norm, seed, cap):
    torch.cuda.synchronize()
    for g, G in enumerate(groups):
        o = oracle_group(G, t_end, samples, prec, rnd, norm, seed, cap)
        out = {k: v.cpu().numpy() for k, v in batch.outputs[g].items()}
        np.testing.assert_array_equal(out["snapshots"], o["snapshots"])
        np.testing.assert_array_equal(out["status"].view(np.uint32), o["status"])
        np.testing.assert_array_equal(out["n_events"], o["n_events"])
        np.testing.assert_array_equal(out["t_final"].view(np.uint64), o["t_final"].view(np.uint64))


@pytest.mark.parametrize("prec,rnd", [("mixed_f16", "rn"), ("uniform_bf16", "sr"), ("fp64", "rn"), ("mixed_bf16", "sr")])
def test_sweep_batch_matches_oracle(ssa, prec, rnd):
    groups = sweep_groups(ssa)
    t_end, samples = 20.0, [10.0, 20.0]
    api = [{k: v for k, v in G.items() if k != "dict"} for G in groups]
    b = ssa.Batch(api, t_end, samples, prec, rnd, seed=77, max_events=100000)
    b.launch()   # NULL stream: direct launch
    check(b, groups, t_end, samples, prec, rnd, False, 77, 100000)
    # graph capture on a stream, replayed twice (the queues are reset inside the graph)
    s = torch.cuda.Stream()
    for _ in range(2):
        for o in b.outputs:
            o["snapshots"].fill_(-1)
        b.launch(s)
        s.synchronize()
        check(b, groups, t_end, samples, prec, rnd, False, 77, 100000)


def test_mixed_family_batch_uses_full_kernel(ssa):
    """Birth-death, Schloegl (normalised) and a general-kernel network in one launch."""
    bd, sch, gen = P.birth_death(), P.schlogl(), P.hill_self(1.0, 30.0, 2, 1.0)
    groups = [
        {"dict": sch, "model": ssa.Model.from_dict(sch), "x0": np.tile(P.schlogl_x0(sch), (2, 1)),
         "rates": np.array([[3e-7, 1e-4, 1e-3, 3.5], [3.3e-7, 1e-4, 1e-3, 3.4]]), "traj_per_set": 24, "traj_offset": 5},
        {"dict": bd, "model": ssa.Model.from_dict(bd), "x0": np.array([[0], [50]]), "traj_per_set": 70,
         "traj_offset": 1000},
        {"dict": gen, "model": ssa.Model.from_dict(gen), "x0": np.array([[0]]), "traj_per_set": 90,
         "traj_offset": 3000},
    ]
    assert groups[2]["model"].family == "general"
    api = [{k: v for k, v in G.items() if k != "dict"} for G in groups]
    for prec, rnd in [("mixed_f16", "sr"), ("uniform_f16", "rn")]:
        b = ssa.Batch(api, 2.0, [1.0, 2.0], prec, rnd, normalise=True, seed=5, max_events=50000)
        b.launch()
        check(b, groups, 2.0, [1.0, 2.0], prec, rnd, True, 5, 50000)


def test_autotune_keeps_results(ssa):
    groups = sweep_groups(ssa, n_sets=(20, 10, 2), traj=(64, 64, 16))
    api = [{k: v for k, v in G.items() if k != "dict"} for G in groups]
    b = ssa.Batch(api, 10.0, [10.0], "mixed_f16", "rn", seed=3, max_events=100000)
    s = torch.cuda.Stream()
    cfg = b.autotune(s)
    assert cfg["threads_per_block"] in (64, 128, 256) and cfg["slice_pairs"] in (1, 4, 16) and cfg["ms"] > 0
    b.launch(s)
    s.synchronize()
    check(b, groups, 10.0, [10.0], "mixed_f16", "rn", False, 3, 100000)


@pytest.mark.parametrize("prec,rnd,park", [("mixed_f16", "rn", 64), ("uniform_bf16", "sr", 200), ("fp64", "rn", 2)])
def test_longest_first_batch_matches_oracle(ssa, prec, rnd, park):
    """Longest-first scheduling forced on a batch: launch 1 parks every group's
    trajectories at `park` events, the ordering kernels sort each group by
    predicted remaining work with each set's own rate constants, launch 2
    resumes them.  Direct launch and graph replay equal the oracle set by set
    and the library counts five kernels per group plus two."""
    groups = sweep_groups(ssa)
    t_end, samples = 20.0, [10.0, 20.0]
    api = [{k: v for k, v in G.items() if k != "dict"} for G in groups]
    ssa.set_longest_first(2, park)
    try:
        b = ssa.Batch(api, t_end, samples, prec, rnd, seed=77, max_events=100000)
    finally:
        ssa.set_longest_first()
    n0 = ssa.direct_kernel_launches()
    b.launch()
    torch.cuda.synchronize()
    assert ssa.direct_kernel_launches() - n0 == 2 + 3 * len(groups)
    check(b, groups, t_end, samples, prec, rnd, False, 77, 100000)
    s = torch.cuda.Stream()
    for _ in range(2):
        for o in b.outputs:
            o["snapshots"].fill_(-1)
            o["n_events"].fill_(-1)
        b.launch(s)
        s.synchronize()
        check(b, groups, t_end, samples, prec, rnd, False, 77, 100000)
    # the autotuner times plain launches and keeps the split for the real ones
    b.autotune(s)
    b.launch(s)
    s.synchronize()
    check(b, groups, t_end, samples, prec, rnd, False, 77, 100000)


def test_longest_first_batch_cap_below_parking_point(ssa):
    """A parking point at or above the event cap parks nothing: one launch."""
    groups = sweep_groups(ssa)
    api = [{k: v for k, v in G.items() if k != "dict"} for G in groups]
    ssa.set_longest_first(2, 5000)
    try:
        b = ssa.Batch(api, 20.0, [20.0], "mixed_f16", "rn", seed=9, max_events=5000)
    finally:
        ssa.set_longest_first()
    n0 = ssa.direct_kernel_launches()
    b.launch()
    torch.cuda.synchronize()
    assert ssa.direct_kernel_launches() - n0 == 1
    check(b, groups, 20.0, [20.0], "mixed_f16", "rn", False, 9, 5000)


def test_longest_first_full_family_batch(ssa):
    """The full batch instantiation (birth-death, Schloegl normalised and a
    general-kernel Hill network) with every group parked and resumed."""
    bd, sch, gen = P.birth_death(), P.schlogl(), P.hill_self(1.0, 30.0, 2, 1.0)
    groups = [
        {"dict": sch, "model": ssa.Model.from_dict(sch), "x0": np.tile(P.schlogl_x0(sch), (2, 1)),
         "rates": np.array([[3e-7, 1e-4, 1e-3, 3.5], [3.3e-7, 1e-4, 1e-3, 3.4]]), "traj_per_set": 24, "traj_offset": 5},
        {"dict": bd, "model": ssa.Model.from_dict(bd), "x0": np.array([[0], [50]]), "traj_per_set": 70,
         "traj_offset": 1000},
        {"dict": gen, "model": ssa.Model.from_dict(gen), "x0": np.array([[0]]), "traj_per_set": 90,
         "traj_offset": 3000},
    ]
    api = [{k: v for k, v in G.items() if k != "dict"} for G in groups]
    for prec, rnd, park in [("mixed_f16", "sr", 16), ("uniform_f16", "rn", 100)]:
        ssa.set_longest_first(2, park)
        try:
            b = ssa.Batch(api, 2.0, [1.0, 2.0], prec, rnd, normalise=True, seed=5, max_events=50000)
        finally:
            ssa.set_longest_first()
        n0 = ssa.direct_kernel_launches()
        b.launch()
        torch.cuda.synchronize()
        assert ssa.direct_kernel_launches() - n0 == 2 + 3 * len(groups)
        check(b, groups, 2.0, [1.0, 2.0], prec, rnd, True, 5, 50000)

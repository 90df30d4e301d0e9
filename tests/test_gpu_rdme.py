"""GPU parity of the RDME engine (lattice of well-mixed voxels with hops,
every precision mode) against the oracle, through the C ABI.

Both sides follow one contract (voxel channel chains, sum-tree selection,
incremental recomputation, epoch-keyed stochastic-rounding bits); snapshots,
status bits and event counts must be equal and final times bit-identical.
"""
import numpy as np
import pytest

import oracle
from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_f16", "sr"), ("mixed_bf16", "rn"),
         ("mixed_bf16", "sr"), ("uniform_f16", "rn"), ("uniform_f16", "sr"), ("uniform_bf16", "rn"),
         ("uniform_bf16", "sr")]


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    assert torch.cuda.is_available()
    mod.lib()
    return mod


def inert():
    return {"order": np.zeros((1, 1), np.int32), "stoich": np.zeros((1, 1), np.int32), "rate": np.array([0.0])}


def general_network():
    """Species (X, Y, Z) with Z a reservoir; orders up to 3; no compiled structure."""
    return {
        "order": np.array([[1, 0, 1], [2, 0, 0], [0, 1, 0], [0, 3, 0], [0, 0, 0], [1, 0, 0]], np.int32),
        "stoich": np.array([[1, 0, -1], [-2, 1, 0], [1, -1, 0], [0, -3, 0], [0, 1, 0], [-1, 0, 0]], np.int32),
        "rate": np.array([0.02, 0.01, 0.5, 0.001, 2.0, 0.1]),
        "law": np.zeros(6, np.int32),
        "constant": np.array([0, 0, 1], np.uint8),
    }


def point_source(S, N, counts):
    x0 = np.zeros((S, N), np.int32)
    x0[0] = counts
    return x0


def schlogl_chain():
    m = P.schlogl()
    x0 = np.tile(P.schlogl_x0(m), (4, 1)).astype(np.int32)
    x0[:, 0] = [250, 100, 400, 250]
    return m, x0


CASES = {
    # name: (model, dims, diffusion, x0 [S, N], n_traj, t_end, samples, normalise, max_events)
    "diffusion_1d": (inert(), (8,), [1.0], point_source(8, 1, [40]), 1000, 2.0, P.even_samples(2.0, 5), False, 10**6),
    "dimer_2d": (P.dimer(2e-2, 0.1), (3, 3), [0.5, 0.2], point_source(9, 2, [80, 0]), 300, 5.0,
                 P.even_samples(5.0, 6), False, 10**6),
    "birth_death_3d": (P.birth_death(2.0, 0.5), (3, 2, 2), [0.7], point_source(12, 1, [20]), 500, 3.0,
                       P.even_samples(3.0, 4), False, 10**6),
    "schlogl_chain": (*schlogl_chain()[:1], (4,), [2.0, 0.0, 0.0], schlogl_chain()[1], 64, 0.5,
                      P.even_samples(0.5, 3), True, 60000),
    "repressilator_pair": (P.repressilator(), (2,), [0.5, 0.5, 0.5, 0.1, 0.1, 0.1],
                           np.tile(P.REPRESSILATOR_X0, (2, 1)), 60, 2.0, P.even_samples(2.0, 3), False, 60000),
    "schlogl_chain_raw": (*schlogl_chain()[:1], (4,), [2.0, 0.0, 0.0], schlogl_chain()[1], 32, 0.2,
                          P.even_samples(0.2, 3), False, 30000),
    "general_reservoir": (general_network(), (2, 2), [0.3, 0.6, 0.0], np.tile([10, 5, 50], (4, 1)), 200, 5.0,
                          P.even_samples(5.0, 4), True, 20000),
    "single_voxel": (P.dimer(), (1,), [1.0, 1.0], P.dimer_x0(300)[None, :], 200, 10.0, P.even_samples(10.0, 5),
                     False, 10**6),
}


def gpu_rdme(ssa, model, dims, D, x0, n, t_end, samples, prec, rnd, norm, seed, cap, state_bytes=4, traj_offset=0):
    m = ssa.Model.from_dict(model)
    r = ssa.rdme_run(m, dims, D, x0, n, t_end, samples, prec, rnd, norm, seed, cap, state_bytes,
                     traj_offset=traj_offset)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def assert_same(g, o):
    np.testing.assert_array_equal(g["snapshots"], o["snapshots"])
    np.testing.assert_array_equal(g["status"].view(np.uint32), o["status"])
    np.testing.assert_array_equal(g["n_events"], o["n_events"])
    np.testing.assert_array_equal(g["t_final"].view(np.uint64), o["t_final"].view(np.uint64))


@pytest.mark.parametrize("prec,rnd", MODES)
@pytest.mark.parametrize("name", list(CASES))
def test_rdme_parity_with_oracle(ssa, name, prec, rnd):
    model, dims, D, x0, n, t_end, samples, norm, cap = CASES[name]
    seed = 500 + len(name)
    g = gpu_rdme(ssa, model, dims, D, x0, n, t_end, samples, prec, rnd, norm, seed, cap)
    o = oracle.rdme_run(model, dims, D, x0, n, t_end, samples, precision=prec, rounding=rnd, normalise=norm,
                        seed=seed, max_events=cap)
    assert_same(g, o)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_bf16", "uniform_f16"])
def test_single_voxel_matches_the_well_mixed_engine(ssa, prec):
    """One voxel: the RDME kernel and the direct-method kernel agree exactly."""
    dm = P.dimer()
    m = ssa.Model.from_dict(dm)
    x0 = P.dimer_x0(300)
    samples = P.even_samples(10.0, 5)
    a = ssa.ensemble_run(m, 333, x0, 10.0, samples, prec, "rn", False, 12, 10**6)
    b = ssa.rdme_run(m, (1,), [1.0, 1.0], x0[None, :], 333, 10.0, samples, prec, "rn", False, 12, 10**6)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a["snapshots"].cpu().numpy(), b["snapshots"][:, 0].cpu().numpy())
    np.testing.assert_array_equal(a["n_events"].cpu().numpy(), b["n_events"].cpu().numpy())
    np.testing.assert_array_equal(a["t_final"].cpu().numpy().view(np.uint64),
                                  b["t_final"].cpu().numpy().view(np.uint64))


def test_rdme_ragged_offset_int16_and_launch_shape(ssa):
    model, dims, D, x0, _, t_end, samples, norm, cap = CASES["dimer_2d"]
    n, off = 1037, 2**32 - 1037
    o = oracle.rdme_run(model, dims, D, x0, n, t_end, samples, precision="uniform_bf16", rounding="sr", seed=77,
                        max_events=cap, state_bytes=2, g0=off)
    try:
        for block, per_sm in [(128, 0), (32, 1), (64, 2)]:
            ssa.set_launch_config(block, per_sm, 1)
            g = gpu_rdme(ssa, model, dims, D, x0, n, t_end, samples, "uniform_bf16", "sr", norm, 77, cap,
                         state_bytes=2, traj_offset=off)
            assert g["snapshots"].dtype == np.int16
            assert_same(g, o)
    finally:
        ssa.set_launch_config()


def test_rdme_event_cap_and_overflow(ssa):
    model, dims, D, x0, _, t_end, samples, norm, _ = CASES["dimer_2d"]
    g = gpu_rdme(ssa, model, dims, D, x0, 100, t_end, samples, "mixed_f16", "sr", norm, 3, 50)
    o = oracle.rdme_run(model, dims, D, x0, 100, t_end, samples, precision="mixed_f16", rounding="sr", seed=3,
                        max_events=50)
    assert_same(g, o)
    assert np.all(o["status"] & 2)
    big = {"order": np.array([[0]], np.int32), "stoich": np.array([[1]], np.int32), "rate": np.array([1e5])}
    g = gpu_rdme(ssa, big, (4,), [1.0], np.zeros((4, 1), np.int32), 50, 1.0, [1.0], "uniform_f16", "rn", False, 1, 100)
    o = oracle.rdme_run(big, (4,), [1.0], np.zeros((4, 1), np.int32), 50, 1.0, [1.0], precision="uniform_f16",
                        rounding="rn", seed=1, max_events=100)
    assert_same(g, o)
    assert np.all(o["status"] & 1)


def test_rdme_outputs_in_page_locked_host_memory(ssa):
    """Page-locked host buffers passed as the outputs: the kernel writes into
    host memory directly; results equal the device-buffer run."""
    model, dims, D, x0, _, t_end, samples, norm, cap = CASES["dimer_2d"]
    m = ssa.Model.from_dict(model)
    n = 3001
    S = int(np.prod(dims))
    K = len(samples)
    host = {"out": torch.full((K, S, m.N, n), -9, dtype=torch.int32).pin_memory(),
            "status": torch.full((n,), -9, dtype=torch.int32).pin_memory(),
            "n_events": torch.full((n,), -9, dtype=torch.int64).pin_memory(),
            "t_final": torch.full((n,), -9.0, dtype=torch.float64).pin_memory()}
    ssa.rdme_run(m, dims, D, x0, n, t_end, samples, "mixed_f16", "sr", norm, 12, cap, **host)
    torch.cuda.synchronize()
    g = gpu_rdme(ssa, model, dims, D, x0, n, t_end, samples, "mixed_f16", "sr", norm, 12, cap)
    np.testing.assert_array_equal(host["out"].numpy(), g["snapshots"])
    np.testing.assert_array_equal(host["status"].numpy(), g["status"])
    np.testing.assert_array_equal(host["n_events"].numpy(), g["n_events"])
    np.testing.assert_array_equal(host["t_final"].numpy().view(np.uint64), g["t_final"].view(np.uint64))

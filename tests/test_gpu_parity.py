"""GPU parity: the CUDA engine, called through the C ABI, against the oracle.

Integer results (snapshots, event counts, status bits) must match exactly;
the final time must match bit for bit (both sides round every operation
identically, so the required tolerance is zero).  Sizes span several thread
blocks with a ragged tail; the uniform round-to-nearest modes, whose clocks
may stagnate, run under an event cap so that MAX_EVENTS paths are compared
too.
"""
import zlib

import numpy as np
import pytest

import oracle
from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_f16", "sr"), ("mixed_bf16", "rn"),
         ("mixed_bf16", "sr"), ("uniform_f16", "rn"), ("uniform_f16", "sr"), ("uniform_bf16", "rn"),
         ("uniform_bf16", "sr"), ("uniform_f16", "sra"), ("uniform_bf16", "sra")]


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    assert torch.cuda.is_available()
    mod.lib()
    return mod


def general_network():
    """Species (X, Y, Z) with Z a reservoir; orders up to 3; matches no
    compiled structure, so it runs on the general kernel."""
    return {
        "order": np.array([[1, 0, 1], [2, 0, 0], [0, 1, 0], [0, 3, 0], [0, 0, 0], [1, 0, 0]], np.int32),
        "stoich": np.array([[1, 0, -1], [-2, 1, 0], [1, -1, 0], [0, -3, 0], [0, 1, 0], [-1, 0, 0]], np.int32),
        "rate": np.array([0.02, 0.01, 0.5, 0.001, 2.0, 0.1]),
        "law": np.zeros(6, np.int32),
        "constant": np.array([0, 0, 1], np.uint8),
    }


CASES = {
    # name: (model, x0, n_traj, t_end, samples, normalise, max_events)
    "birth_death": (P.birth_death(10.0, 0.1), [0], 1000, 100.0, P.even_samples(100.0, 101), False, 20000),
    "schlogl": (P.schlogl(), None, 96, 10.0, P.even_samples(10.0, 50), True, 200000),
    "telegraph": (P.telegraph(0.5, 0.5, 20.0, 1.0), P.TELEGRAPH_X0, 1000, 50.0, P.even_samples(50.0, 11), False, 20000),
    "dimer": (P.dimer(), P.dimer_x0(300), 500, 20.0, P.even_samples(20.0, 21), False, 20000),
    "repressilator": (P.repressilator(), P.REPRESSILATOR_X0, 160, 10.0, P.even_samples(10.0, 11), False, 40000),
    "general_hill3": (P.repressilator(h=3), P.REPRESSILATOR_X0, 100, 5.0, P.even_samples(5.0, 6), False, 40000),
    "general_network": (general_network(), [10, 5, 50], 300, 20.0, P.even_samples(20.0, 5), True, 20000),
}


def gpu_run(ssa, model_dict, x0, n_traj, t_end, samples, prec, rnd, normalise, seed, max_events, state_bytes=4,
            traj_offset=0):
    m = ssa.Model.from_dict(model_dict)
    r = ssa.ensemble_run(m, n_traj, x0, t_end, samples, prec, rnd, normalise, seed, max_events, state_bytes,
                         traj_offset=traj_offset)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}, m.family


def assert_same(g, o):
    np.testing.assert_array_equal(g["snapshots"], o["snapshots"])
    np.testing.assert_array_equal(g["status"].view(np.uint32), o["status"])
    np.testing.assert_array_equal(g["n_events"], o["n_events"])
    gt, ot = g["t_final"], o["t_final"]
    both_nan = np.isnan(gt) & np.isnan(ot)
    np.testing.assert_array_equal(gt.view(np.uint64)[~both_nan], ot.view(np.uint64)[~both_nan])


@pytest.mark.parametrize("prec,rnd", MODES)
@pytest.mark.parametrize("name", list(CASES))
def test_parity_with_oracle(ssa, name, prec, rnd):
    model, x0, n, t_end, samples, norm, cap = CASES[name]
    if x0 is None:
        x0 = P.schlogl_x0(model)
    seed = 0x5EED0000 + zlib.crc32(f"{name}{prec}{rnd}".encode()) % 1000
    g, fam = gpu_run(ssa, model, x0, n, t_end, samples, prec, rnd, norm, seed, cap)
    o = oracle.run_parallel(model, x0, n, t_end, samples, precision=prec, rounding=rnd, normalise=norm, seed=seed,
                            max_events=cap)
    if name.startswith("general"):
        assert fam == "general"
    else:
        assert fam == name
    assert_same(g, o)


@pytest.mark.parametrize("prec,rnd", [("mixed_f16", "rn"), ("mixed_f16", "sr"), ("uniform_f16", "sr")])
def test_schlogl_unnormalised_fp16_overflow_parity(ssa, prec, rnd):
    """Sec. 4.2: without folding, A = 1e5 overflows binary16; every trajectory
    stops at X0 = 250 with status OVERFLOW, on both sides."""
    m = P.schlogl()
    x0 = P.schlogl_x0(m)
    g, _ = gpu_run(ssa, m, x0, 257, 10.0, P.even_samples(10.0, 50), prec, rnd, False, 3, 10**6)
    o = oracle.run(m, x0, 257, 10.0, P.even_samples(10.0, 50), prec, rnd, False, 3, 10**6)
    assert_same(g, o)
    assert np.all(g["status"] == 1) and np.all(g["snapshots"][:, 0, :] == 250)


def test_edge_cases(ssa):
    bd = P.birth_death(20.0, 1.0)
    # no trajectories: nothing launched, nothing written
    m = ssa.Model.from_dict(bd)
    r = ssa.ensemble_run(m, 0, [0], 10.0, [10.0], "fp32")
    torch.cuda.synchronize()
    assert r["snapshots"].numel() == 0
    # one trajectory, single sample at t_end
    for n in (1, 31, 33):
        g, _ = gpu_run(ssa, bd, [0], n, 10.0, [10.0], "mixed_bf16", "sr", False, 7, 10**6)
        assert_same(g, oracle.run(bd, [0], n, 10.0, [10.0], "mixed_bf16", "sr", False, 7, 10**6))
    # event cap of zero: every snapshot holds x0
    g, _ = gpu_run(ssa, bd, [3], 64, 10.0, P.even_samples(10.0, 4), "fp64", "rn", False, 1, 0)
    assert np.all(g["status"] == 2) and np.all(g["snapshots"] == 3) and np.all(g["n_events"] == 0)
    # int16 storage overflow: clamped and flagged
    birth = P.birth_death(40000.0, 0.0)
    g, _ = gpu_run(ssa, birth, [0], 40, 1.0, [0.5, 1.0], "fp32", "rn", False, 2, 10**6, state_bytes=2)
    o = oracle.run(birth, [0], 40, 1.0, [0.5, 1.0], "fp32", "rn", False, 2, 10**6, state_bytes=2)
    assert_same(g, o)
    assert np.all(g["status"] & 4) and np.all(g["snapshots"][-1] == 32767)
    # absorbing state and negative counts
    death = P.birth_death(0.0, 1.0)
    g, _ = gpu_run(ssa, death, [5], 50, 100.0, [50.0, 100.0], "uniform_f16", "sr", False, 4, 10**6)
    assert_same(g, oracle.run(death, [5], 50, 100.0, [50.0, 100.0], "uniform_f16", "sr", False, 4, 10**6))
    neg = {"order": np.array([[0]]), "stoich": np.array([[-1]]), "rate": np.array([1.0]), "law": np.array([0])}
    g, _ = gpu_run(ssa, neg, [2], 40, 100.0, [100.0], "fp64", "rn", False, 5, 10**6)
    assert_same(g, oracle.run(neg, [2], 40, 100.0, [100.0], "fp64", "rn", False, 5, 10**6))
    assert np.all(g["status"] == 4)
    # trajectory ids at the top of the 32-bit range
    off = 2**32 - 300
    g, _ = gpu_run(ssa, bd, [0], 300, 5.0, [5.0], "uniform_bf16", "sr", False, 6, 10**6, traj_offset=off)
    assert_same(g, oracle.run(bd, [0], 300, 5.0, [5.0], "uniform_bf16", "sr", False, 6, 10**6, g0=off))


def test_results_independent_of_launch_shape(ssa):
    tel = P.telegraph(0.3, 0.2, 10.0, 1.0)
    base = None
    try:
        for block, per_sm, slice_pairs in [(128, 0, 1), (128, 0, 16), (256, 0, 32), (32, 1, 3), (256, 2, 16), (64, 0, 2)]:
            ssa.set_launch_config(block, per_sm, slice_pairs)
            g, _ = gpu_run(ssa, tel, P.TELEGRAPH_X0, 700, 20.0, P.even_samples(20.0, 5), "uniform_f16", "sr",
                           False, 8, 10**6)
            if base is None:
                base = g
            else:
                assert_same(g, base)
    finally:
        ssa.set_launch_config()


def test_host_entry_point_matches_device(ssa):
    dm = P.dimer()
    m = ssa.Model.from_dict(dm)
    h = ssa.ensemble_run_host(m, 777, P.dimer_x0(300), 10.0, P.even_samples(10.0, 3), "mixed_f16", "sr", seed=9,
                              max_events=10**6)
    g, _ = gpu_run(ssa, dm, P.dimer_x0(300), 777, 10.0, P.even_samples(10.0, 3), "mixed_f16", "sr", False, 9, 10**6)
    assert_same({**h, "status": h["status"].view(np.int32)}, {**g, "status": g["status"].view(np.uint32)})


@pytest.mark.parametrize("state_bytes", [4, 2])
def test_large_host_entry_point_matches_device(ssa, state_bytes):
    """The host entry point (staging memory from the library's pool) at 3e5
    trajectories with an id offset equals the device entry point."""
    tel = P.telegraph(0.5, 0.5, 20.0, 1.0)
    m = ssa.Model.from_dict(tel)
    n, off = 300001, 12345
    samples = P.even_samples(5.0, 4)
    h = ssa.ensemble_run_host(m, n, P.TELEGRAPH_X0, 5.0, samples, "uniform_bf16", "sr", seed=31, max_events=10**5,
                              state_bytes=state_bytes, traj_offset=off)
    g, _ = gpu_run(ssa, tel, P.TELEGRAPH_X0, n, 5.0, samples, "uniform_bf16", "sr", False, 31, 10**5,
                   state_bytes=state_bytes, traj_offset=off)
    assert_same({**h, "status": h["status"].view(np.int32)}, {**g, "status": g["status"].view(np.uint32)})


@pytest.mark.parametrize("stream_kind", ["sparse", "dense"])
@pytest.mark.parametrize("pinned", ["all", "all_but_status", "no_optional"])
def test_host_entry_point_page_locked_outputs(ssa, pinned, stream_kind):
    """Page-locked outputs with a sparse snapshot stream take the direct-write
    path (the kernel writes into host memory: Schloegl, X stored, ~10^4
    events per trajectory); a dense stream (telegraph, every species at 6
    times over a few events) or a pageable buffer among the outputs goes
    through device staging.  Results equal the device entry point either way."""
    if stream_kind == "sparse":
        md = P.schlogl()
        x0, t_end, mask, norm, n, prec = P.schlogl_x0(md), 5.0, 0b001, True, 20011, "mixed_bf16"
    else:
        md = P.telegraph(0.5, 0.5, 20.0, 1.0)
        x0, t_end, mask, norm, n, prec = P.TELEGRAPH_X0, 5.0, 0, False, 200003, "mixed_bf16"
    m = ssa.Model.from_dict(md)
    off = 777
    samples = P.even_samples(t_end, 6)
    K = len(samples)
    Ns = m.N if not mask else bin(mask).count("1")
    out = torch.full((K, Ns, n), -5, dtype=torch.int32).pin_memory()
    st = torch.full((n,), -5, dtype=torch.int32)
    st = st.pin_memory() if pinned != "all_but_status" else st
    ev = torch.full((n,), -5, dtype=torch.int64).pin_memory() if pinned != "no_optional" else None
    tf = torch.full((n,), -5.0, dtype=torch.float64).pin_memory() if pinned != "no_optional" else None
    import ctypes
    vp = ctypes.c_void_p
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    rc = ssa.lib().ssa_ensemble_run_host(
        m.handle, n, off, x0.ctypes.data_as(vp), t_end, K, smp.ctypes.data_as(vp), ssa.PRECISION[prec],
        ssa.ROUNDING["sr"], int(norm), 13, 10**5, 4, mask, vp(out.data_ptr()), vp(st.data_ptr()),
        None if ev is None else vp(ev.data_ptr()), None if tf is None else vp(tf.data_ptr()), None)
    assert rc == 0, ssa.lib().ssa_last_error()
    r = ssa.ensemble_run(m, n, x0, t_end, samples, prec, "sr", norm, 13, 10**5, traj_offset=off, out_species=mask)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.numpy(), r["snapshots"].cpu().numpy())
    np.testing.assert_array_equal(st.numpy(), r["status"].cpu().numpy())
    if ev is not None:
        np.testing.assert_array_equal(ev.numpy(), r["n_events"].cpu().numpy())
        np.testing.assert_array_equal(tf.numpy().view(np.uint64), r["t_final"].cpu().numpy().view(np.uint64))


BENCH_MODES = [("mixed_f16", "rn"), ("mixed_bf16", "rn"), ("uniform_f16", "rn"), ("uniform_f16", "sr"),
               ("uniform_bf16", "sr"), ("uniform_f16", "sra"), ("mixed_f16", "sr")]


@pytest.mark.parametrize("prec,rnd", BENCH_MODES)
def test_full_size_schlogl_sampled_trajectories(ssa, prec, rnd):
    """The benchmark's workload (10^6 Schloegl trajectories, 50 snapshots,
    t_end = 10, reservoirs folded, 2e5-event cap) in its launch configuration;
    24 trajectory ids spread over the range are recomputed one by one on the
    oracle, including the last id."""
    m = P.schlogl()
    x0 = P.schlogl_x0(m)
    n = 1_000_000
    samples = P.even_samples(10.0, 50)
    g, _ = gpu_run(ssa, m, x0, n, 10.0, samples, prec, rnd, True, 2605, 200000)
    ids = np.linspace(0, n - 1, 24).astype(np.int64)
    for r in ids:
        o = oracle.run(m, x0, 1, 10.0, samples, prec, rnd, True, 2605, 200000, g0=int(r))
        np.testing.assert_array_equal(g["snapshots"][:, :, r], o["snapshots"][:, :, 0])
        assert g["n_events"][r] == o["n_events"][0]
        assert g["status"][r] == o["status"][0]
        assert g["t_final"][r] == o["t_final"][0]
    # properties over the whole ensemble: conservation of the reservoirs, valid statuses
    assert np.all(g["snapshots"][:, 1:, :] == x0[1:][None, :, None])
    assert np.all((g["status"] & ~2) == 0)
    if rnd != "rn" or prec.startswith("mixed"):
        xs = g["snapshots"][-1, 0]
        assert np.mean(xs < 250) > 0.2 and np.mean(xs > 400) > 0.1


@pytest.mark.parametrize("mask,sb", [(0b001, 2), (0b101, 4), (0b110, 2)])
def test_species_mask_matches_oracle(ssa, mask, sb):
    """Snapshots of a subset of species (out_species): the Schloegl reservoirs
    left out, or stored beside X; int16 storage clamps (and flags) stored
    species only.  Device and host entry points against the oracle."""
    m = P.schlogl()
    x0 = P.schlogl_x0(m)
    smp = P.even_samples(2.0, 6)
    o = oracle.run(m, x0, 1500, 2.0, smp, "uniform_f16", "sr", True, 21, 10**6, state_bytes=sb, out_species=mask)
    model = ssa.Model.from_dict(m)
    g = ssa.ensemble_run(model, 1500, x0, 2.0, smp, "uniform_f16", "sr", True, 21, 10**6, sb, out_species=mask)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g["snapshots"].cpu().numpy(), o["snapshots"])
    np.testing.assert_array_equal(g["status"].cpu().numpy().view(np.uint32), o["status"])
    np.testing.assert_array_equal(g["n_events"].cpu().numpy(), o["n_events"])
    h = ssa.ensemble_run_host(model, 1500, x0, 2.0, smp, "uniform_f16", "sr", True, 21, 10**6, sb, out_species=mask)
    np.testing.assert_array_equal(h["snapshots"], o["snapshots"])
    np.testing.assert_array_equal(h["status"], o["status"])


def test_species_mask_rejects_unknown_species(ssa):
    m = ssa.Model.from_dict(P.schlogl())
    with pytest.raises(ssa.SSAError):
        ssa.ensemble_run(m, 10, P.schlogl_x0(P.schlogl()), 1.0, [1.0], "fp64", "rn", True, 1, 100, 4,
                         out=torch.zeros((1, 1, 10), dtype=torch.int32, device="cuda"), out_species=0b1000)

"""ssa_sweep_run_noalloc: the parameter-sweep entry point that allocates no
memory, for callers that cannot allocate device memory while they simulate
(memory owned by another allocator or held to a fixed budget, real-time
loops).  Its scratch lives in a static device array shared by every call.

The test calls it through the C ABI and compares its output, trajectory by
trajectory, with the allocating entry point ssa_ensemble_run run set by set
(results must be identical: both launch the same kernel on the same
arithmetic).  Two different sweeps run back to back, so the second call
starts from the scratch contents the first one left behind.  This file is
collected last so that a failure here stops a -x run only after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    mod.lib()
    return mod


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def run_noalloc(ssa, model, rates, hill, x0, traj_per_set, offset, t_end, samples, prec, rnd, seed, cap,
                normalise=False, state_bytes=4):
    S = x0.shape[0]
    n = S * traj_per_set
    K = len(samples)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.full((K, model.N, n), -7, dtype=torch.int16 if state_bytes == 2 else torch.int32, device=dev)
    st = torch.full((n,), -7, dtype=torch.int32, device=dev)
    ev = torch.full((n,), -7, dtype=torch.int64, device=dev)
    tf = torch.full((n,), -7.0, dtype=torch.float64, device=dev)
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    rc = ssa.lib().ssa_sweep_run_noalloc(
        model.handle, S, traj_per_set, _ptr(rates), _ptr(hill), _ptr(x0), offset, float(t_end), K, _ptr(smp),
        ssa.PRECISION[prec], ssa.ROUNDING[rnd], int(normalise), seed, cap, state_bytes, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(tf.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ssa.lib().ssa_last_error()
    torch.cuda.synchronize()
    return {"snapshots": out.cpu().numpy(), "status": st.cpu().numpy(), "n_events": ev.cpu().numpy(),
            "t_final": tf.cpu().numpy()}


def run_existing(ssa, model_dict, rates, hill, x0, traj_per_set, offset, t_end, samples, prec, rnd, seed, cap,
                 normalise=False, state_bytes=4):
    parts = []
    for q in range(x0.shape[0]):
        md = dict(model_dict)
        if rates is not None:
            md["rate"] = rates[q]
        if hill is not None:
            h = np.array(md["hill"], dtype=np.float64, copy=True)
            h[:, :2] = hill[q]
            md["hill"] = h
        m = ssa.Model.from_dict(md)
        r = ssa.ensemble_run(m, traj_per_set, x0[q], t_end, samples, prec, rnd, normalise, seed, cap,
                             state_bytes=state_bytes, traj_offset=offset + q * traj_per_set)
        torch.cuda.synchronize()
        parts.append({k: v.cpu().numpy() for k, v in r.items()})
    return {k: np.concatenate([p[k] for p in parts], axis=-1) for k in parts[0]}


def same(a, b):
    for k in ("snapshots", "status", "n_events"):
        np.testing.assert_array_equal(a[k], b[k])
    np.testing.assert_array_equal(a["t_final"].view(np.uint64), b["t_final"].view(np.uint64))


def test_noalloc_sweep_matches_existing_entry_point_twice(ssa):
    # call 1: telegraph sweep, 37 sets x 29 trajectories, mixed binary16 with SR
    tel = P.telegraph()
    rates = np.ascontiguousarray(P.telegraph_sweep(37, seed=91))
    x0 = np.ascontiguousarray(np.tile(P.TELEGRAPH_X0, (37, 1)), dtype=np.int32)
    m = ssa.Model.from_dict(tel)
    args = (rates, None, x0, 29, 1000, 20.0, [10.0, 20.0], "mixed_f16", "sr", 123, 100000)
    a = run_noalloc(ssa, m, *args)
    b = run_existing(ssa, tel, *args)
    same(a, b)
    assert np.all(a["status"] == 0)
    # call 2, straight after: a different model and size (repressilator sweep with
    # Hill amplitudes per set), so the scratch holds the previous call's tables
    rp = P.repressilator()
    rr, rh = P.repressilator_sweep(5, seed=92)
    rr = np.ascontiguousarray(rr)
    rh = np.ascontiguousarray(rh[:, :, :2])
    x0r = np.ascontiguousarray(np.tile(P.REPRESSILATOR_X0, (5, 1)), dtype=np.int32)
    mr = ssa.Model.from_dict(rp)
    args = (rr, rh, x0r, 33, 50000, 5.0, [2.5, 5.0], "uniform_bf16", "sr", 7, 100000)
    a = run_noalloc(ssa, mr, *args)
    b = run_existing(ssa, rp, *args)
    same(a, b)


def test_noalloc_rejects_sweeps_beyond_the_scratch(ssa):
    tel = ssa.Model.from_dict(P.telegraph())
    limit = ssa.lib().ssa_sweep_noalloc_scratch_bytes(3, 4, 10**6)
    assert limit > 1 << 20
    S = 10**6
    x0 = np.zeros((S, 3), np.int32)
    x0[:, 0] = 1
    smp = np.array([1.0])
    rc = ssa.lib().ssa_sweep_run_noalloc(tel.handle, S, 1, None, None, _ptr(x0), 0, 1.0, 1, _ptr(smp), 2, 0, 0,
                                         0, 1000, 4, ctypes.c_void_p(8), ctypes.c_void_p(8), None, None, None)
    assert rc == ssa.SSA_EINVAL
    assert b"scratch" in ssa.lib().ssa_last_error()


def test_noalloc_single_set_normalised_reservoirs_and_int16(ssa):
    """Paths the sweep test above leaves out: with one set the kernel reads the
    scalar rate, Hill and x0 fields (filled from set 0); with normalise=1 every
    set folds its own reservoir counts into c' (Sec. 4.2 rescaling), so sets
    that differ only in A and B differ in their rates; int16 storage clamps the
    reservoir columns.  Each call is compared with ssa_ensemble_run."""
    sch = P.schlogl()
    m = ssa.Model.from_dict(sch)
    x0 = np.ascontiguousarray(P.schlogl_x0(sch), dtype=np.int32)
    # one set, normalised, int32
    args = (None, None, x0[None, :], 300, 77, 2.0, [0.5, 1.0, 2.0], "mixed_bf16", "sr", 5, 10**6)
    a = run_noalloc(ssa, m, *args, normalise=True)
    b = run_existing(ssa, sch, *args, normalise=True)
    same(a, b)
    # four sets with different reservoir counts, normalised, int16 storage
    xs = np.tile(x0, (4, 1))
    xs[:, 1] = [100000, 90000, 110000, 100000]
    xs[:, 2] = [200000, 210000, 190000, 180000]
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    args = (None, None, xs, 64, 4000, 1.0, [0.5, 1.0], "uniform_f16", "sr", 9, 10**6)
    a = run_noalloc(ssa, m, *args, normalise=True, state_bytes=2)
    b = run_existing(ssa, sch, *args, normalise=True, state_bytes=2)
    same(a, b)
    assert a["snapshots"].dtype == np.int16
    # the reservoir columns are clamped to int16 and flagged
    assert np.all(a["snapshots"][:, 1:, :] == 32767) and np.all(a["status"] & 4)
    # different reservoirs mean different folded rates: the sets' X columns differ
    X = a["snapshots"][-1, 0, :].reshape(4, 64).astype(np.float64)
    assert len({round(float(r.mean()), 3) for r in X}) > 1


def test_noalloc_refuses_a_capturing_stream(ssa):
    """The per-set tables are staged from host memory that lives only for the
    call, so a captured call would replay stale tables: it is refused."""
    tel = P.telegraph()
    m = ssa.Model.from_dict(tel)
    x0 = np.ascontiguousarray(np.tile(P.TELEGRAPH_X0, (2, 1)), dtype=np.int32)
    smp = np.array([1.0])
    n = 2 * 32
    out = torch.zeros((1, m.N, n), dtype=torch.int32, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    # warm-up call on this device outside capture (it looks up the scratch address)
    run_noalloc(ssa, m, None, None, x0, 32, 0, 1.0, [1.0], "mixed_f16", "rn", 1, 1000)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    rc = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            rc = ssa.lib().ssa_sweep_run_noalloc(m.handle, 2, 32, None, None, _ptr(x0), 0, 1.0, 1, _ptr(smp), 2, 0,
                                                 0, 1, 1000, 4, ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.c_void_p(st.data_ptr()), None, None,
                                                 ctypes.c_void_p(s.cuda_stream))
        finally:
            g.capture_end()
    assert rc == ssa.SSA_EINVAL
    assert b"capturing" in ssa.lib().ssa_last_error()


def test_noalloc_rejects_set_counts_that_would_wrap(ssa):
    tel = ssa.Model.from_dict(P.telegraph())
    assert ssa.lib().ssa_sweep_noalloc_scratch_bytes(3, 4, 2**62) == 2**64 - 1
    x0 = np.zeros((1, 3), np.int32)
    smp = np.array([1.0])
    for S, T in ((2**61, 1), (2, 2**62)):
        rc = ssa.lib().ssa_sweep_run_noalloc(tel.handle, S, T, None, None, _ptr(x0), 0, 1.0, 1, _ptr(smp), 2, 0,
                                             0, 0, 1000, 4, ctypes.c_void_p(8), ctypes.c_void_p(8), None, None, None)
        assert rc == ssa.SSA_EINVAL

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


def run_noalloc(ssa, model, rates, hill, x0, traj_per_set, offset, t_end, samples, prec, rnd, seed, cap):
    S = x0.shape[0]
    n = S * traj_per_set
    K = len(samples)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = torch.full((K, model.N, n), -7, dtype=torch.int32, device=dev)
    st = torch.full((n,), -7, dtype=torch.int32, device=dev)
    ev = torch.full((n,), -7, dtype=torch.int64, device=dev)
    tf = torch.full((n,), -7.0, dtype=torch.float64, device=dev)
    smp = np.ascontiguousarray(samples, dtype=np.float64)
    rc = ssa.lib().ssa_sweep_run_noalloc(
        model.handle, S, traj_per_set, _ptr(rates), _ptr(hill), _ptr(x0), offset, float(t_end), K, _ptr(smp),
        ssa.PRECISION[prec], ssa.ROUNDING[rnd], 0, seed, cap, 4, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(ev.data_ptr()), ctypes.c_void_p(tf.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ssa.lib().ssa_last_error()
    torch.cuda.synchronize()
    return {"snapshots": out.cpu().numpy(), "status": st.cpu().numpy(), "n_events": ev.cpu().numpy(),
            "t_final": tf.cpu().numpy()}


def run_existing(ssa, model_dict, rates, hill, x0, traj_per_set, offset, t_end, samples, prec, rnd, seed, cap):
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
        r = ssa.ensemble_run(m, traj_per_set, x0[q], t_end, samples, prec, rnd, False, seed, cap,
                             traj_offset=offset + q * traj_per_set)
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

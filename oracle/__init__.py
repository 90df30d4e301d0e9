"""Oracle for the reduced-precision Gillespie direct method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It is a plain, slow,
single-threaded CPU reference (``ssa_oracle.c``) plus the statistics and
master-equation checkers used to pin it; it shares no code with the CUDA engine.

Functions here marshal numpy arrays into the C oracle; the arithmetic itself
lives in ``ssa_oracle.c`` (see its header for the paper passages followed).

Parity notes: the binary16/bfloat16 conversions, the log, Philox and the fp64
direct method are pinned by tests against library routines, closed forms and
master-equation solutions.  The bit-level schedule of the mixed and uniform
16-bit modes (which random bits feed which rounding) is a convention the paper
does not fix: parity unpinned at the bit level by the paper; it is pinned by
properties (exactness reductions, conservation, unbiasedness) and by the
statistical behaviour the paper reports.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

PRECISIONS = {"fp64": 0, "fp32": 1, "mixed_f16": 2, "mixed_bf16": 3, "uniform_f16": 4, "uniform_bf16": 5}
ROUNDINGS = {"rn": 0, "sr": 1, "sra": 2}   # sra: SR at accumulation points only
STATUS_OVERFLOW, STATUS_MAX_EVENTS, STATUS_STATE_RANGE, STATUS_NAN = 1, 2, 4, 8


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.oracle_run.restype = ctypes.c_int
        L.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P,
                                 ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                 ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, P, P, P, P]
        for name in ("oracle_f32_to_f16_array", "oracle_f32_to_bf16_array"):
            getattr(L, name).argtypes = [P, ctypes.c_int64, ctypes.c_int, P, P]
        L.oracle_f16_to_f32_array.argtypes = [P, ctypes.c_int64, P]
        L.oracle_log_f32_array.argtypes = [P, ctypes.c_int64, P]
        L.oracle_log_f64_array.argtypes = [P, ctypes.c_int64, P]
        L.oracle_philox_array.argtypes = [P, P, ctypes.c_int64, P]
        _LIB = L
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- primitives
def philox(ctr, key, n=1):
    """Philox4x32-10 blocks for counters (ctr0 + i, ctr1, ctr2, ctr3), i < n."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros((n, 4), dtype=np.uint32)
    lib().oracle_philox_array(_p(c), _p(k), n, _p(out))
    return out


def f32_to_f16(x, sr=False, r=None):
    """binary32 -> binary16 bit patterns (RN-even, or SR with 13 bits of r)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    rr = None if r is None else np.ascontiguousarray(np.broadcast_to(r, x.shape), dtype=np.uint32)
    out = np.zeros(x.shape, dtype=np.uint16)
    lib().oracle_f32_to_f16_array(_p(x), x.size, int(sr), _p(rr), _p(out))
    return out


def f32_to_bf16(x, sr=False, r=None):
    """binary32 -> bfloat16 bit patterns (RN-even, or SR with 16 bits of r)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    rr = None if r is None else np.ascontiguousarray(np.broadcast_to(r, x.shape), dtype=np.uint32)
    out = np.zeros(x.shape, dtype=np.uint16)
    lib().oracle_f32_to_bf16_array(_p(x), x.size, int(sr), _p(rr), _p(out))
    return out


def f16_to_f32(h):
    h = np.ascontiguousarray(h, dtype=np.uint16)
    out = np.zeros(h.shape, dtype=np.float32)
    lib().oracle_f16_to_f32_array(_p(h), h.size, _p(out))
    return out


def log_f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.shape, dtype=np.float32)
    lib().oracle_log_f32_array(_p(x), x.size, _p(out))
    return out


def log_f64(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.shape, dtype=np.float64)
    lib().oracle_log_f64_array(_p(x), x.size, _p(out))
    return out


# ---------------------------------------------------------------- the SSA
def run(model, x0, n_traj, t_end, sample_times, precision="fp64", rounding="rn", normalise=False,
        seed=0, max_events=10**9, state_bytes=4, g0=0, out_species=0):
    """Simulate trajectories g0 .. g0+n_traj-1 of ``model`` on the oracle.

    ``model`` is a mapping with numpy arrays ``order`` [M,N], ``stoich`` [M,N],
    ``rate`` [M], ``law`` [M], optional ``hill`` [M,4] and ``constant`` [N].
    Returns a dict with ``snapshots`` [K,N,n_traj], ``status``, ``n_events`` and
    ``t_final`` (time of the last applied event, widened to binary64).
    """
    order = np.ascontiguousarray(model["order"], dtype=np.int32)
    M, N = order.shape
    stoich = np.ascontiguousarray(model["stoich"], dtype=np.int32)
    rate = np.ascontiguousarray(model["rate"], dtype=np.float64)
    law = np.ascontiguousarray(model.get("law", np.zeros(M)), dtype=np.int32)
    hill = model.get("hill")
    hill = None if hill is None else np.ascontiguousarray(hill, dtype=np.float64).reshape(M, 4)
    const = model.get("constant")
    const = None if const is None else np.ascontiguousarray(const, dtype=np.uint8)
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    st = np.ascontiguousarray(sample_times, dtype=np.float64)
    K = st.size
    Ns = N if not out_species else bin(int(out_species)).count("1")
    out = np.zeros((K, Ns, n_traj), dtype=np.int16 if state_bytes == 2 else np.int32)
    status = np.zeros(n_traj, dtype=np.uint32)
    nev = np.zeros(n_traj, dtype=np.int64)
    tf = np.zeros(n_traj, dtype=np.float64)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rnd = ROUNDINGS[rounding] if isinstance(rounding, str) else int(rounding)
    rc = lib().oracle_run(N, M, _p(order), _p(stoich), _p(rate), _p(law), _p(hill), _p(const), _p(x0),
                          int(n_traj), int(g0), float(t_end), K, _p(st), prec, rnd, int(bool(normalise)),
                          int(seed) & 0xFFFFFFFFFFFFFFFF, int(max_events), int(state_bytes), int(out_species),
                          _p(out), _p(status), _p(nev), _p(tf))
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    return {"snapshots": out, "status": status, "n_events": nev, "t_final": tf}


def trace_step(model, x0, step, precision="fp64", rounding="rn", normalise=False, seed=0, g=0, t_end=1e30):
    """Inputs and intermediates of direct-method step ``step`` of trajectory
    ``g`` (the oracle's own arithmetic, recorded as it runs): a dict with n,
    t (before the step), x (before), a (propensities), S (partial sums), a0,
    u1, u2, E, U2, tau, target, t_new, mu; None if the trajectory ended
    earlier.  For tests that recompute one step independently."""
    M, N = np.asarray(model["order"]).shape
    buf = np.zeros(160, dtype=np.float64)
    L = lib()
    L.oracle_trace_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    L.oracle_trace_step(_p(buf), int(step))
    try:
        run(model, x0, 1, t_end, [t_end], precision, rounding, normalise, seed, max_events=int(step) + 1, g0=g)
    finally:
        L.oracle_trace_step(None, -1)
    if buf[0] != 1.0:
        return None
    return {"n": int(buf[1]), "t": buf[2], "x": buf[3:3 + N].astype(np.int64), "a": buf[16:16 + M].copy(),
            "S": buf[48:48 + M].copy(), "a0": buf[80], "u1": buf[81], "u2": buf[82], "E": buf[83], "U2": buf[84],
            "tau": buf[85], "target": buf[86], "t_new": buf[87], "mu": int(buf[88])}


def _run_chunk(args):
    kwargs = dict(args)
    return run(**kwargs)


def run_parallel(model, x0, n_traj, t_end, sample_times, workers=None, **kw):
    """``run`` split over trajectory-id ranges in a spawned process pool.

    Trajectories are independent and keyed by their global id, so the result
    equals a single ``run`` call; this only shortens wall time."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or max(1, min(os.cpu_count() or 1, 16))
    g0 = int(kw.pop("g0", 0))
    if workers == 1 or n_traj < 2 * workers:
        return run(model, x0, n_traj, t_end, sample_times, g0=g0, **kw)
    bounds = np.linspace(0, n_traj, workers + 1).astype(np.int64)
    jobs = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        if b > a:
            jobs.append(dict(model=model, x0=x0, n_traj=int(b - a), t_end=t_end,
                             sample_times=sample_times, g0=g0 + int(a), **kw))
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_run_chunk, jobs))
    return {
        "snapshots": np.concatenate([p["snapshots"] for p in parts], axis=2),
        "status": np.concatenate([p["status"] for p in parts]),
        "n_events": np.concatenate([p["n_events"] for p in parts]),
        "t_final": np.concatenate([p["t_final"] for p in parts]),
    }


# ------------------------------------------------------------ tau-leaping
def _tau_lib():
    L = lib()
    if not getattr(L, "_tau_ready", False):
        P = ctypes.c_void_p
        L.oracle_tau_run.restype = ctypes.c_int
        L.oracle_tau_run.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int64, ctypes.c_uint64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, P, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_uint64, ctypes.c_int, P, P, P, P]
        L.oracle_poisson_array.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, P]
        L.oracle_exp_f32_array.argtypes = [P, ctypes.c_int64, P]
        L.oracle_exp_f64_array.argtypes = [P, ctypes.c_int64, P]
        L._tau_ready = True
    return L


def exp_f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.shape, dtype=np.float32)
    _tau_lib().oracle_exp_f32_array(_p(x), x.size, _p(out))
    return out


def exp_f64(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(x.shape, dtype=np.float64)
    _tau_lib().oracle_exp_f64_array(_p(x), x.size, _p(out))
    return out


def poisson(lam, n, prec64=False, seed=0):
    """n variates of the oracle's Poisson sampler (binary32 or binary64)."""
    out = np.zeros(n, dtype=np.int64)
    _tau_lib().oracle_poisson_array(float(lam), int(bool(prec64)), int(seed), int(n), _p(out))
    return out


def tau_run(model, x0, n_traj, t_end, tau, sample_times, precision="fp64", rounding="rn", normalise=False, seed=0,
            state_bytes=4, g0=0):
    """Tau-leaping trajectories (fixed leap tau) on the oracle; same outputs as ``run``
    (n_events = reactions fired, t_final = end of the last leap)."""
    order = np.ascontiguousarray(model["order"], dtype=np.int32)
    M, N = order.shape
    stoich = np.ascontiguousarray(model["stoich"], dtype=np.int32)
    rate = np.ascontiguousarray(model["rate"], dtype=np.float64)
    law = np.ascontiguousarray(model.get("law", np.zeros(M)), dtype=np.int32)
    hill = model.get("hill")
    hill = None if hill is None else np.ascontiguousarray(hill, dtype=np.float64).reshape(M, 4)
    const = model.get("constant")
    const = None if const is None else np.ascontiguousarray(const, dtype=np.uint8)
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    st = np.ascontiguousarray(sample_times, dtype=np.float64)
    K = st.size
    out = np.zeros((K, N, n_traj), dtype=np.int16 if state_bytes == 2 else np.int32)
    status = np.zeros(n_traj, dtype=np.uint32)
    nev = np.zeros(n_traj, dtype=np.int64)
    tf = np.zeros(n_traj, dtype=np.float64)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rnd = ROUNDINGS[rounding] if isinstance(rounding, str) else int(rounding)
    rc = _tau_lib().oracle_tau_run(N, M, _p(order), _p(stoich), _p(rate), _p(law), _p(hill), _p(const), _p(x0),
                                   int(n_traj), int(g0), float(t_end), float(tau), K, _p(st), prec, rnd,
                                   int(bool(normalise)), int(seed) & 0xFFFFFFFFFFFFFFFF, int(state_bytes),
                                   _p(out), _p(status), _p(nev), _p(tf))
    if rc != 0:
        raise ValueError("oracle_tau_run rejected its arguments")
    return {"snapshots": out, "status": status, "n_events": nev, "t_final": tf}


def _rdme_lib():
    L = lib()
    if not getattr(L, "_rdme_ready", False):
        P = ctypes.c_void_p
        i, i64, u64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.oracle_rdme_run.restype = i
        L.oracle_rdme_run.argtypes = [i, i, P, P, P, P, P, P, i, i, i, P, P, i64, u64, d, i, P, i, i, i, u64, i64, i,
                                      P, P, P, P]
        L._rdme_ready = True
    return L


def rdme_run(model, dims, diffusion, x0, n_traj, t_end, sample_times, precision="fp64", rounding="rn",
             normalise=False, seed=0, max_events=10**9, state_bytes=4, g0=0):
    """RDME trajectories on an nx x ny x nz lattice (dims) with hop rates per
    direction ``diffusion`` [N] and initial counts ``x0`` [S, N]; snapshots
    [K, S, N, n_traj] plus status, n_events (reactions and hops), t_final."""
    order = np.ascontiguousarray(model["order"], dtype=np.int32)
    M, N = order.shape
    stoich = np.ascontiguousarray(model["stoich"], dtype=np.int32)
    rate = np.ascontiguousarray(model["rate"], dtype=np.float64)
    law = np.ascontiguousarray(model.get("law", np.zeros(M)), dtype=np.int32)
    hill = model.get("hill")
    hill = None if hill is None else np.ascontiguousarray(hill, dtype=np.float64).reshape(M, 4)
    const = model.get("constant")
    const = None if const is None else np.ascontiguousarray(const, dtype=np.uint8)
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    S = nx * ny * nz
    x0 = np.ascontiguousarray(np.broadcast_to(np.asarray(x0, dtype=np.int32), (S, N)))
    D = np.ascontiguousarray(diffusion, dtype=np.float64)
    st = np.ascontiguousarray(sample_times, dtype=np.float64)
    K = st.size
    out = np.zeros((K, S, N, n_traj), dtype=np.int16 if state_bytes == 2 else np.int32)
    status = np.zeros(n_traj, dtype=np.uint32)
    nev = np.zeros(n_traj, dtype=np.int64)
    tf = np.zeros(n_traj, dtype=np.float64)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rnd = ROUNDINGS[rounding] if isinstance(rounding, str) else int(rounding)
    rc = _rdme_lib().oracle_rdme_run(N, M, _p(order), _p(stoich), _p(rate), _p(law), _p(hill), _p(const), nx, ny, nz,
                                     _p(D), _p(x0), int(n_traj), int(g0), float(t_end), K, _p(st), prec, rnd,
                                     int(bool(normalise)), int(seed) & 0xFFFFFFFFFFFFFFFF, int(max_events),
                                     int(state_bytes), _p(out), _p(status), _p(nev), _p(tf))
    if rc != 0:
        raise ValueError("oracle_rdme_run rejected its arguments")
    return {"snapshots": out, "status": status, "n_events": nev, "t_final": tf}


def _named_chunk(job):
    fn = {"tau_run": tau_run, "rdme_run": rdme_run}[job.pop("fn")]
    r = fn(**job)
    return {"n_events": r["n_events"], "status": r["status"]}


def events_parallel(fn, n_traj, workers=None, **kw):
    """Event counts and status of ``tau_run`` or ``rdme_run`` (named by ``fn``)
    over trajectory ids g0 .. g0+n_traj-1, split over a spawned process pool
    (trajectories are independent, so this only shortens wall time)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or max(1, min(os.cpu_count() or 1, 16))
    g0 = int(kw.pop("g0", 0))
    bounds = np.linspace(0, n_traj, workers + 1).astype(np.int64)
    jobs = [dict(fn=fn, n_traj=int(b - a), g0=g0 + int(a), **kw) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    if len(jobs) == 1:
        return _named_chunk(jobs[0])
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_named_chunk, jobs))
    return {"n_events": np.concatenate([p["n_events"] for p in parts]),
            "status": np.concatenate([p["status"] for p in parts])}

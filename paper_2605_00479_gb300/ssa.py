"""Python binding of the C ABI in include/ssa.h (argument marshalling only).

Every step of the simulation runs in the CUDA kernels of libssa_gb300.so;
this module converts Python/numpy/torch arguments into pointers and sizes.
PyTorch supplies device memory and streams.  If the library has not been
built, ``lib()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libssa_gb300.so")

PRECISION = {"fp64": 0, "fp32": 1, "mixed_f16": 2, "mixed_bf16": 3, "uniform_f16": 4, "uniform_bf16": 5}
ROUNDING = {"rn": 0, "sr": 1, "sra": 2}   # sra: SR at accumulation points only
STATUS_OVERFLOW, STATUS_MAX_EVENTS, STATUS_STATE_RANGE, STATUS_NAN, STATUS_TAU_CLAMPED = 1, 2, 4, 8, 16
SSA_OK, SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA, SSA_ETIMEDOUT = 0, -1, -2, -3, -4
FAMILIES = {0: "general", 1: "birth_death", 2: "schlogl", 3: "telegraph", 4: "dimer", 5: "repressilator"}

# name -> (restype, argtypes) for every function declared in include/ssa.h
_P = ctypes.c_void_p
_I, _I64, _U64, _D = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
_RUN_ARGS = [_P, _I64, _U64, _P, _D, _I, _P, _I, _I, _I, _U64, _I64, _I, ctypes.c_uint32, _P, _P, _P, _P, _P]
SIGNATURES = {
    "ssa_model_create": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "ssa_model_destroy": (None, [_P]),
    "ssa_model_kernel_family": (_I, [_P]),
    "ssa_ensemble_run": (_I, _RUN_ARGS),
    "ssa_ensemble_run_host": (_I, _RUN_ARGS),
    "ssa_tau_run": (_I, [_P, _I64, _U64, _P, _D, _D, _I, _P, _I, _I, _I, _U64, _I, _P, _P, _P, _P, _P]),
    "ssa_rdme_run": (_I, [_P, _I, _I, _I, _P, _I64, _U64, _P, _D, _I, _P, _I, _I, _I, _U64, _I64, _I, _P, _P, _P, _P,
                          _P]),
    "ssa_set_launch_config": (_I, [_I, _I, _I]),
    "ssa_set_tail_compaction": (_I, [_I]),
    "ssa_set_tail_lock_limit": (_I, [_I]),
    "ssa_tail_stats": (_I, [ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "ssa_set_longest_first": (_I, [_I, _I64]),
    "ssa_direct_kernel_launches": (_I, [ctypes.POINTER(_I64)]),
    "ssa_batch_create": (_I, [_I, _P, _D, _I, _P, _I, _I, _I, _U64, _I64, _I, ctypes.POINTER(_P)]),
    "ssa_batch_launch": (_I, [_P, _P]),
    "ssa_batch_autotune": (_I, [_P, _P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                ctypes.POINTER(_D)]),
    "ssa_batch_destroy": (None, [_P]),
    "ssa_sweep_noalloc_scratch_bytes": (ctypes.c_size_t, [_I, _I, _I64]),
    "ssa_sweep_run_noalloc": (_I, [_P, _I64, _I64, _P, _P, _P, _U64, _D, _I, _P, _I, _I, _I, _U64, _I64, _I,
                                   _P, _P, _P, _P, _P]),
    "ssa_mlp_gemm_bf16": (_I, [_I, _I, _I, _P, _P, _P, _P]),
    "ssa_mlp_set_wait_test": (_I, [_I, _I]),
    "ssa_mlp_gemm_epi": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ssa_mlp_softmax_xent": (_I, [_I, _P, _P, _P, _P, _P, _P, _P]),
    "ssa_surrogate_param_count": (_I64, []),
    "ssa_surrogate_create": (_I, [_I, _U64, ctypes.POINTER(_P)]),
    "ssa_surrogate_destroy": (None, [_P]),
    "ssa_surrogate_set_params": (_I, [_P, _P]),
    "ssa_surrogate_get_params": (_I, [_P, _P]),
    "ssa_surrogate_predict": (_I, [_P, _I, _P, _P, _P]),
    "ssa_surrogate_train_step": (_I, [_P, _I, _P, _P, ctypes.c_float, ctypes.c_float, _P, _P]),
    "ssa_surrogate_train": (_I, [_P, _I64, _I64, _P, _P, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I64,
                                 _P, _P]),
    "ssa_surrogate_gradients": (_I, [_P, _I, _P, _P, _P, _P]),
    "ssa_surrogate_get_state": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_I64)]),
    "ssa_surrogate_status": (_I, [_P]),
    "ssa_round16": (_I, [_P, _P, _I64, _I, _I, _I, _P, _P]),
    "ssa_histogram": (_I, [_P, _I64, _I64, _I, _P, _P]),
    "ssa_hist_w1": (_I, [_P, _P, _I64, _I, _P, _P]),
    "ssa_hist_w1_noise": (_I, [_P, _I64, _I, _D, _P, _P]),
    "ssa_count_histogram": (_I, [_P, _I, _I64, _I, _P, _P, _P]),
    "ssa_hist_ks_w1": (_I, [_P, _P, _I, _P, _P]),
    "ssa_dwell_histogram": (_I, [_P, _I, _I, _I64, _I64, _P, _P]),
    "ssa_last_error": (ctypes.c_char_p, []),
}

_LIB = None


class SSAError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"ssa error {code}: {message}")
        self.code = code


def lib():
    """Load the CUDA engine.  Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA engine not built ({LIB_PATH} missing): run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(rc):
    if rc != SSA_OK:
        raise SSAError(rc, lib().ssa_last_error().decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _dev_ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Model:
    """A reaction network (Sec. 2 problem statement), owned by the library."""

    def __init__(self, order, stoich, rate, law=None, hill=None, constant=None):
        self.order = np.ascontiguousarray(order, dtype=np.int32)
        M, N = self.order.shape
        self.N, self.M = N, M
        self.stoich = np.ascontiguousarray(stoich, dtype=np.int32).reshape(M, N)
        self.rate = np.ascontiguousarray(rate, dtype=np.float64).reshape(M)
        self.law = None if law is None else np.ascontiguousarray(law, dtype=np.int32)
        self.hill = None if hill is None else np.ascontiguousarray(hill, dtype=np.float64).reshape(M, 4)
        self.constant = None if constant is None else np.ascontiguousarray(constant, dtype=np.uint8)
        h = _P()
        _check(lib().ssa_model_create(N, M, _np_ptr(self.order), _np_ptr(self.stoich), _np_ptr(self.rate),
                                      _np_ptr(self.law), _np_ptr(self.hill), _np_ptr(self.constant), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_dict(cls, m):
        return cls(m["order"], m["stoich"], m["rate"], m.get("law"), m.get("hill"), m.get("constant"))

    @property
    def handle(self):
        return self._h

    @property
    def family(self):
        return FAMILIES[lib().ssa_model_kernel_family(self._h)]

    def close(self):
        if getattr(self, "_h", None):
            lib().ssa_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_launch_config(threads_per_block=0, blocks_per_sm=0, slice_pairs=0):
    """Launch shape for later runs (speed only; results do not depend on it).
    With no arguments, back to the library's defaults."""
    _check(lib().ssa_set_launch_config(int(threads_per_block), int(blocks_per_sm), int(slice_pairs)))


def set_tail_compaction(enabled=True):
    """Tail compaction of the direct-method kernel (speed only)."""
    _check(lib().ssa_set_tail_compaction(1 if enabled else 0))


def set_tail_lock_limit(spins=0):
    """Bound on one hand-off lock wait of tail compaction (0: the default)."""
    _check(lib().ssa_set_tail_lock_limit(int(spins)))


def tail_stats():
    """(trajectories moved between warps, lock waits given up, trajectories
    resumed at the end of a block) so far on the current device; synchronises
    it."""
    moved, timeouts, resumed = _I64(0), _I64(0), _I64(0)
    _check(lib().ssa_tail_stats(ctypes.byref(moved), ctypes.byref(timeouts), ctypes.byref(resumed)))
    return int(moved.value), int(timeouts.value), int(resumed.value)


def set_longest_first(mode=1, park_events=0):
    """Scheduling of direct-method ensemble runs: 0 off, 1 automatic (the
    default), 2 always; park_events 0 for the automatic parking point."""
    _check(lib().ssa_set_longest_first(int(mode), int(park_events)))


def direct_kernel_launches():
    """Kernels launched by the direct-method ensemble entry points so far."""
    n = _I64(0)
    _check(lib().ssa_direct_kernel_launches(ctypes.byref(n)))
    return int(n.value)


def _run_scalars(model, n_traj, traj_offset, x0, t_end, sample_times, precision, rounding, normalise, seed,
                 max_events, state_bytes):
    x0 = np.ascontiguousarray(x0, dtype=np.int32)
    st = np.ascontiguousarray(np.atleast_1d(sample_times), dtype=np.float64)
    prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
    rnd = ROUNDING[rounding] if isinstance(rounding, str) else int(rounding)
    return x0, st, prec, rnd


def _stored(model, out_species):
    """Number of stored species for an out_species mask (0: all)."""
    return model.N if not out_species else bin(int(out_species)).count("1")


def ensemble_run(model, n_traj, x0, t_end, sample_times, precision="fp64", rounding="rn", normalise=False, seed=0,
                 max_events=10**9, state_bytes=4, out=None, status=None, n_events=None, t_final=None,
                 stream=None, traj_offset=0, with_events=True, with_t_final=True, out_species=0):
    """Launch ssa_ensemble_run on CUDA tensors (allocated here when None).

    Returns a dict of device tensors: snapshots [K, Ns, n_traj] (Ns species
    stored per the out_species mask, 0 = all), status, n_events, t_final.
    Asynchronous on ``stream`` (a torch.cuda.Stream or None for the current
    stream)."""
    import torch
    x0, st, prec, rnd = _run_scalars(model, n_traj, traj_offset, x0, t_end, sample_times, precision, rounding,
                                     normalise, seed, max_events, state_bytes)
    dev = torch.device("cuda", torch.cuda.current_device())
    K = st.size
    if out is None:
        out = torch.empty((K, _stored(model, out_species), n_traj), dtype=torch.int16 if state_bytes == 2
                          else torch.int32, device=dev)
    if status is None:
        status = torch.empty(n_traj, dtype=torch.int32, device=dev)
    if n_events is None and with_events:
        n_events = torch.empty(n_traj, dtype=torch.int64, device=dev)
    if t_final is None and with_t_final:
        t_final = torch.empty(n_traj, dtype=torch.float64, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().ssa_ensemble_run(model.handle, int(n_traj), int(traj_offset), _np_ptr(x0), float(t_end), K,
                                  _np_ptr(st), prec, rnd, int(bool(normalise)), int(seed) & (2**64 - 1),
                                  int(max_events), int(state_bytes), int(out_species), _dev_ptr(out),
                                  _dev_ptr(status), _dev_ptr(n_events), _dev_ptr(t_final),
                                  ctypes.c_void_p(s.cuda_stream)))
    return {"snapshots": out, "status": status, "n_events": n_events, "t_final": t_final}


def ensemble_run_host(model, n_traj, x0, t_end, sample_times, precision="fp64", rounding="rn", normalise=False,
                      seed=0, max_events=10**9, state_bytes=4, out=None, status=None, n_events=None, t_final=None,
                      stream=None, traj_offset=0, out_species=0):
    """ssa_ensemble_run_host: host (numpy) outputs; synchronous."""
    x0, st, prec, rnd = _run_scalars(model, n_traj, traj_offset, x0, t_end, sample_times, precision, rounding,
                                     normalise, seed, max_events, state_bytes)
    K = st.size
    if out is None:
        out = np.empty((K, _stored(model, out_species), n_traj), dtype=np.int16 if state_bytes == 2 else np.int32)
    if status is None:
        status = np.empty(n_traj, dtype=np.uint32)
    if n_events is None:
        n_events = np.empty(n_traj, dtype=np.int64)
    if t_final is None:
        t_final = np.empty(n_traj, dtype=np.float64)
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream)
    _check(lib().ssa_ensemble_run_host(model.handle, int(n_traj), int(traj_offset), _np_ptr(x0), float(t_end), K,
                                       _np_ptr(st), prec, rnd, int(bool(normalise)), int(seed) & (2**64 - 1),
                                       int(max_events), int(state_bytes), int(out_species), _np_ptr(out),
                                       _np_ptr(status), _np_ptr(n_events), _np_ptr(t_final), sp))
    return {"snapshots": out, "status": status, "n_events": n_events, "t_final": t_final}


def tau_run(model, n_traj, x0, t_end, tau, sample_times, precision="fp64", rounding="rn", normalise=False, seed=0,
            state_bytes=4, out=None, status=None, n_events=None, t_final=None, stream=None, traj_offset=0):
    """Launch ssa_tau_run (fixed-leap tau-leaping) on CUDA tensors.

    Same outputs as ensemble_run; n_events counts reactions fired and t_final
    is the end of the last completed leap."""
    import torch
    x0, st, prec, rnd = _run_scalars(model, n_traj, traj_offset, x0, t_end, sample_times, precision, rounding,
                                     normalise, seed, 0, state_bytes)
    dev = torch.device("cuda", torch.cuda.current_device())
    K = st.size
    if out is None:
        out = torch.empty((K, model.N, n_traj), dtype=torch.int16 if state_bytes == 2 else torch.int32,
                          device=dev)
    if status is None:
        status = torch.empty(n_traj, dtype=torch.int32, device=dev)
    if n_events is None:
        n_events = torch.empty(n_traj, dtype=torch.int64, device=dev)
    if t_final is None:
        t_final = torch.empty(n_traj, dtype=torch.float64, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().ssa_tau_run(model.handle, int(n_traj), int(traj_offset), _np_ptr(x0), float(t_end), float(tau), K,
                             _np_ptr(st), prec, rnd, int(bool(normalise)), int(seed) & (2**64 - 1),
                             int(state_bytes), _dev_ptr(out), _dev_ptr(status), _dev_ptr(n_events),
                             _dev_ptr(t_final), ctypes.c_void_p(s.cuda_stream)))
    return {"snapshots": out, "status": status, "n_events": n_events, "t_final": t_final}


def rdme_run(model, dims, diffusion, x0, n_traj, t_end, sample_times, precision="fp64", rounding="rn",
             normalise=False, seed=0, max_events=10**9, state_bytes=4, out=None, status=None, n_events=None,
             t_final=None, stream=None, traj_offset=0):
    """Launch ssa_rdme_run on CUDA tensors: an nx x ny x nz lattice (dims),
    hop rates ``diffusion`` [N], initial counts ``x0`` [S, N].  Returns
    snapshots [K, S, N, n_traj], status, n_events (reactions and hops), t_final."""
    import torch
    nx, ny, nz = (list(dims) + [1, 1])[:3]
    S = nx * ny * nz
    x0 = np.ascontiguousarray(np.broadcast_to(np.asarray(x0, dtype=np.int32), (S, model.N)))
    D = np.ascontiguousarray(diffusion, dtype=np.float64)
    if D.shape != (model.N,):
        raise ValueError("diffusion must have one rate per species")
    _, st, prec, rnd = _run_scalars(model, n_traj, traj_offset, x0[0], t_end, sample_times, precision, rounding,
                                    normalise, seed, max_events, state_bytes)
    dev = torch.device("cuda", torch.cuda.current_device())
    K = st.size
    if out is None:
        out = torch.empty((K, S, model.N, n_traj), dtype=torch.int16 if state_bytes == 2 else torch.int32, device=dev)
    if status is None:
        status = torch.empty(n_traj, dtype=torch.int32, device=dev)
    if n_events is None:
        n_events = torch.empty(n_traj, dtype=torch.int64, device=dev)
    if t_final is None:
        t_final = torch.empty(n_traj, dtype=torch.float64, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().ssa_rdme_run(model.handle, int(nx), int(ny), int(nz), _np_ptr(D), int(n_traj), int(traj_offset),
                              _np_ptr(x0), float(t_end), K, _np_ptr(st), prec, rnd, int(bool(normalise)),
                              int(seed) & (2**64 - 1), int(max_events), int(state_bytes), _dev_ptr(out),
                              _dev_ptr(status), _dev_ptr(n_events), _dev_ptr(t_final), ctypes.c_void_p(s.cuda_stream)))
    return {"snapshots": out, "status": status, "n_events": n_events, "t_final": t_final}


class BatchGroup(ctypes.Structure):
    """Mirror of ssa_batch_group in include/ssa.h."""
    _fields_ = [("model", _P), ("n_sets", _I64), ("traj_per_set", _I64), ("rates", _P), ("hill", _P), ("x0", _P),
                ("traj_offset", _U64), ("out", _P), ("traj_status", _P), ("n_events", _P), ("t_final", _P)]


class Batch:
    """ssa_batch_*: several groups (model + parameter sweep) in one persistent launch.

    ``groups`` is a list of dicts with keys ``model`` (Model), ``x0`` [S, N],
    ``traj_per_set``, optional ``rates`` [S, M], ``hill`` [S, M, 2],
    ``traj_offset``.  Device outputs are allocated here (torch) and exposed as
    ``self.outputs[g]``."""

    def __init__(self, groups, t_end, sample_times, precision="mixed_f16", rounding="rn", normalise=False, seed=0,
                 max_events=10**9, state_bytes=4, host_outputs=False):
        """host_outputs: outputs in page-locked host memory (written by the
        kernel directly) instead of device memory."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        st = np.ascontiguousarray(np.atleast_1d(sample_times), dtype=np.float64)
        K = st.size
        self._keep = [st]
        self.outputs = []
        arr = (BatchGroup * len(groups))()
        for g, G in enumerate(groups):
            m = G["model"]
            x0 = np.ascontiguousarray(G["x0"], dtype=np.int32).reshape(-1, m.N)
            S = x0.shape[0]
            T = int(G["traj_per_set"])
            rates = G.get("rates")
            rates = None if rates is None else np.ascontiguousarray(rates, dtype=np.float64).reshape(S, m.M)
            hill = G.get("hill")
            hill = None if hill is None else np.ascontiguousarray(hill, dtype=np.float64).reshape(S, m.M, 2)
            n = S * T
            def alloc(shape, dtype):
                if host_outputs:
                    return torch.empty(shape, dtype=dtype).pin_memory()
                return torch.empty(shape, dtype=dtype, device=dev)
            o = {"snapshots": alloc((K, m.N, n), torch.int16 if state_bytes == 2 else torch.int32),
                 "status": alloc(n, torch.int32), "n_events": alloc(n, torch.int64),
                 "t_final": alloc(n, torch.float64)}
            self.outputs.append(o)
            self._keep += [x0, rates, hill, m]
            arr[g] = BatchGroup(m.handle, S, T, _np_ptr(rates), _np_ptr(hill), _np_ptr(x0), int(G.get("traj_offset", 0)),
                                o["snapshots"].data_ptr(), o["status"].data_ptr(), o["n_events"].data_ptr(),
                                o["t_final"].data_ptr())
        prec = PRECISION[precision] if isinstance(precision, str) else int(precision)
        rnd = ROUNDING[rounding] if isinstance(rounding, str) else int(rounding)
        h = _P()
        _check(lib().ssa_batch_create(len(groups), ctypes.cast(arr, _P), float(t_end), K, _np_ptr(st), prec, rnd,
                                      int(bool(normalise)), int(seed) & (2**64 - 1), int(max_events),
                                      int(state_bytes), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        """Asynchronous; a torch stream replays a captured CUDA graph."""
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(lib().ssa_batch_launch(self._h, sp))

    def autotune(self, stream=None):
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        b, p, sl, ms = _I(), _I(), _I(), _D()
        _check(lib().ssa_batch_autotune(self._h, sp, ctypes.byref(b), ctypes.byref(p), ctypes.byref(sl),
                                        ctypes.byref(ms)))
        return {"threads_per_block": b.value, "blocks_per_sm": p.value, "slice_pairs": sl.value, "ms": ms.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().ssa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Surrogate:
    """ssa_surrogate_*: the telegraph surrogate network (marshalling only)."""

    def __init__(self, max_batch, seed=0):
        h = _P()
        _check(lib().ssa_surrogate_create(int(max_batch), int(seed) & (2**64 - 1), ctypes.byref(h)))
        self._h = h
        self.n_params = int(lib().ssa_surrogate_param_count())

    def get_params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().ssa_surrogate_get_params(self._h, _np_ptr(out)))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.n_params
        _check(lib().ssa_surrogate_set_params(self._h, _np_ptr(theta)))

    def predict(self, features, probs=None, stream=None):
        import torch
        B = features.shape[0]
        if probs is None:
            probs = torch.empty((B, 128), dtype=torch.float32, device=features.device)
        _check(lib().ssa_surrogate_predict(self._h, B, _dev_ptr(features), _dev_ptr(probs), _stream_ptr(stream)))
        return probs

    def train_step(self, features, targets, lr, weight_decay=1e-4, loss=None, stream=None):
        _check(lib().ssa_surrogate_train_step(self._h, features.shape[0], _dev_ptr(features), _dev_ptr(targets),
                                              float(lr), float(weight_decay), _dev_ptr(loss), _stream_ptr(stream)))

    def train(self, features, targets, steps, batch_size, lr_max, lr_min, weight_decay=1e-4, loss_every=1,
              loss_trace=None, stream=None):
        """ssa_surrogate_train: `steps` AdamW steps replayed from one captured
        CUDA graph; step k uses rows (k * batch_size + j) mod n of features /
        targets (CUDA tensors).  loss_trace: CUDA float tensor of
        ceil(steps / loss_every) entries, or None.  Synchronous."""
        _check(lib().ssa_surrogate_train(self._h, int(steps), int(features.shape[0]), _dev_ptr(features),
                                         _dev_ptr(targets), int(batch_size), float(lr_max), float(lr_min),
                                         float(weight_decay), int(loss_every), _dev_ptr(loss_trace),
                                         _stream_ptr(stream)))

    def gradients(self, features, targets):
        g = np.empty(self.n_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        _check(lib().ssa_surrogate_gradients(self._h, features.shape[0], _dev_ptr(features), _dev_ptr(targets),
                                             _np_ptr(g), _np_ptr(loss)))
        return float(loss[0]), g

    def get_state(self):
        """ssa_surrogate_get_state: (theta, m, v, grad, adam_steps), host arrays."""
        arrs = [np.empty(self.n_params, dtype=np.float32) for _ in range(4)]
        t = ctypes.c_int64(0)
        _check(lib().ssa_surrogate_get_state(self._h, *[_np_ptr(a) for a in arrs], ctypes.byref(t)))
        return (*arrs, int(t.value))

    def status(self):
        _check(lib().ssa_surrogate_status(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().ssa_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def round16(x, rbits=None, fmt="f16", rounding="rn", half=0, out=None, stream=None):
    """ssa_round16 on CUDA tensors: x float32, rbits int32/uint32 words (SR);
    returns the rounded values widened to float32."""
    import torch
    if out is None:
        out = torch.empty_like(x, dtype=torch.float32)
    _check(lib().ssa_round16(_dev_ptr(x), _dev_ptr(rbits), int(x.numel()), {"f16": 0, "bf16": 1}[fmt],
                             {"rn": 0, "sr": 1}[rounding], int(half), _dev_ptr(out), _stream_ptr(stream)))
    return out


def histogram(counts, n_sets, traj_per_set, bins=128, hist=None, stream=None):
    """Normalised per-set histograms (device) of device int32 counts."""
    import torch
    if hist is None:
        hist = torch.empty((n_sets, bins), dtype=torch.float32, device=counts.device)
    _check(lib().ssa_histogram(_dev_ptr(counts), int(n_sets), int(traj_per_set), int(bins), _dev_ptr(hist),
                               _stream_ptr(stream)))
    return hist


def hist_w1(p, q, out=None, stream=None):
    """Row-wise Wasserstein-1 distance between device histograms."""
    import torch
    rows, bins = p.shape
    if out is None:
        out = torch.empty(rows, dtype=torch.float32, device=p.device)
    _check(lib().ssa_hist_w1(_dev_ptr(p), _dev_ptr(q), int(rows), int(bins), _dev_ptr(out), _stream_ptr(stream)))
    return out


# ------------------------------------------------------- ensemble statistics

def hist_w1_noise(p, n_draws, out=None, stream=None):
    """Expected W1 sampling noise of an n-draw histogram of each row's law."""
    import torch
    if out is None:
        out = torch.empty(p.shape[0], dtype=torch.float32, device=p.device)
    _check(lib().ssa_hist_w1_noise(_dev_ptr(p), int(p.shape[0]), int(p.shape[1]), float(n_draws), _dev_ptr(out),
                                   _stream_ptr(stream)))
    return out


def count_histogram(values, bins, hist=None, clamped=None, stream=None):
    """ssa_count_histogram on a contiguous int32/int16 CUDA tensor; returns
    (hist uint64-as-int64 [bins], clamped [1]) device tensors (accumulated
    into the given ones, else fresh zeros)."""
    import torch
    if values.dtype not in (torch.int32, torch.int16) or not values.is_contiguous():
        raise ValueError("values must be a contiguous int32 or int16 tensor")
    if hist is None:
        hist = torch.zeros(bins, dtype=torch.int64, device=values.device)
    if clamped is None:
        clamped = torch.zeros(1, dtype=torch.int64, device=values.device)
    _check(lib().ssa_count_histogram(_dev_ptr(values), values.element_size(), values.numel(), int(bins),
                                     _dev_ptr(hist), _dev_ptr(clamped), _stream_ptr(stream)))
    return hist, clamped


def hist_ks_w1(ha, hb, out=None, stream=None):
    """ssa_hist_ks_w1: device float64 [2] = (KS statistic D, Wasserstein-1)."""
    import torch
    if ha.numel() != hb.numel():
        raise ValueError("histograms must have the same bins")
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=ha.device)
    _check(lib().ssa_hist_ks_w1(_dev_ptr(ha), _dev_ptr(hb), ha.numel(), _dev_ptr(out), _stream_ptr(stream)))
    return out


def dwell_histogram(snapshots, species, hist=None, stream=None):
    """ssa_dwell_histogram of species `species` of snapshots [K, N, n]
    (contiguous CUDA tensor): device int64 [K] of completed OFF-interval lengths."""
    import torch
    if not snapshots.is_contiguous() or snapshots.dim() != 3:
        raise ValueError("snapshots must be a contiguous [K, N, n] tensor")
    K, N, n = snapshots.shape
    if hist is None:
        hist = torch.zeros(K, dtype=torch.int64, device=snapshots.device)
    base = snapshots[0, species]
    _check(lib().ssa_dwell_histogram(_dev_ptr(base), snapshots.element_size(), K, n, N * n, _dev_ptr(hist),
                                     _stream_ptr(stream)))
    return hist

"""Measurement runs for the batched-sweep and scale configurations.

    python -m paper_2605_00479_gb300.experiments batch  [sets=10000] [traj=256]
    python -m paper_2605_00479_gb300.experiments scale  [n_traj=1000000] [t_end=1000] [fp64_traj=20000]

batch: telegraph (kon, koff log-uniform in [0.05, 5], km in [5, 100], gamma 1),
  dimerisation (k1, k2 log-uniform in [x0.5, x2] around 1e-3, 0.1; M0 = 300)
  and repressilator (alpha, beta log-uniform in [x0.5, x2] around 216, 5)
  sweeps, `sets` parameter sets per model x `traj` trajectories, t_end = 200,
  one snapshot at t_end; all three models in ONE persistent launch (longest
  first), autotuned, replayed from a CUDA graph; mixed fp16 RN and uniform
  bf16 SR.
scale: repressilator, `n_traj` trajectories to t_end with 200 snapshots
  streamed to HBM; state stored int32 and int16; propensities in fp16
  (mixed_f16), fp32 and fp64 (fp64 on a subsample of `fp64_traj`
  trajectories: GB300's FP64 rate makes the full ensemble take minutes).
Each prints one JSON line.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import presets as P
from . import ssa


def _timed(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def batch(sets=10000, traj=256, seed=3):
    import torch
    tel, dm, rp = P.telegraph(), P.dimer(), P.repressilator()
    tr = P.telegraph_sweep(sets, seed=seed)
    dr = P.dimer_sweep(sets, seed=seed + 1)
    rr, rh = P.repressilator_sweep(sets, seed=seed + 2)
    models = {"repressilator": ssa.Model.from_dict(rp), "telegraph": ssa.Model.from_dict(tel),
              "dimer": ssa.Model.from_dict(dm)}
    groups = [
        {"model": models["repressilator"], "x0": np.tile(P.REPRESSILATOR_X0, (sets, 1)), "rates": rr,
         "hill": rh[:, :, :2], "traj_per_set": traj, "traj_offset": 0},
        {"model": models["telegraph"], "x0": np.tile(P.TELEGRAPH_X0, (sets, 1)), "rates": tr, "traj_per_set": traj,
         "traj_offset": sets * traj},
        {"model": models["dimer"], "x0": np.tile(P.dimer_x0(300), (sets, 1)), "rates": dr, "traj_per_set": traj,
         "traj_offset": 2 * sets * traj},
    ]
    out = {"config": f"batched sweep: 3 models x {sets} sets x {traj} trajectories, t_end=200, K=1",
           "n_traj": 3 * sets * traj, "modes": {}}
    for prec, rnd in [("mixed_f16", "rn"), ("uniform_bf16", "sr")]:
        b = ssa.Batch(groups, 200.0, [200.0], prec, rnd, seed=seed, max_events=10**7)
        s = torch.cuda.Stream()
        t0 = time.perf_counter()
        cfg = b.autotune(s)
        tune_s = time.perf_counter() - t0
        b.launch(s)                      # capture + first replay (warm-up)
        s.synchronize()
        with torch.cuda.stream(s):
            dt = _timed(lambda: b.launch(s), reps=2)
        ev = {name: int(b.outputs[g]["n_events"].sum()) for g, name in enumerate(["repressilator", "telegraph", "dimer"])}
        st = {name: int((b.outputs[g]["status"] != 0).sum()) for g, name in
              enumerate(["repressilator", "telegraph", "dimer"])}
        total = sum(ev.values())
        out["modes"][f"{prec}:{rnd}"] = {"events": total, "events_per_model": ev, "nonzero_status": st,
                                         "seconds": dt, "events_per_s": total / dt, "autotune": cfg,
                                         "autotune_s": tune_s}
        b.close()
    return out


def scale(n_traj=1_000_000, t_end=1000.0, fp64_traj=20000, seed=5):
    import torch
    rp = P.repressilator()
    m = ssa.Model.from_dict(rp)
    samples = P.even_samples(t_end, 200)
    out = {"config": f"repressilator scale run: {n_traj} trajectories, t_end={t_end}, 200 snapshots",
           "n_traj": n_traj, "runs": {}}
    free, total = torch.cuda.mem_get_info()
    out["hbm_free_gb"] = free / 1e9
    for prec, sb, n in [("mixed_f16", 4, n_traj), ("mixed_f16", 2, n_traj), ("fp32", 4, n_traj), ("fp32", 2, n_traj),
                        ("fp64", 4, fp64_traj), ("fp64", 2, fp64_traj)]:
        snap = torch.empty((200, 6, n), dtype=torch.int16 if sb == 2 else torch.int32, device="cuda")
        st = torch.empty(n, dtype=torch.int32, device="cuda")
        ev = torch.empty(n, dtype=torch.int64, device="cuda")

        def go():
            ssa.ensemble_run(m, n, P.REPRESSILATOR_X0, t_end, samples, prec, "rn", False, seed, 10**9, sb, out=snap,
                             status=st, n_events=ev, t_final=None, with_t_final=False)

        go()   # warm-up
        dt = _timed(go)
        events = int(ev.sum())
        bytes_out = snap.numel() * snap.element_size()
        out["runs"][f"{prec}:int{8 * sb}"] = {
            "n_traj": n, "events": events, "seconds": dt, "events_per_s": events / dt,
            "snapshot_bytes_per_traj": 200 * 6 * sb, "snapshot_hbm_gbs": bytes_out / dt / 1e9,
            "state_range_flags": int(((st & 4) != 0).sum()), "max_abs_state": int(snap.abs().max())}
        del snap, st, ev
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    cmd = sys.argv[1]
    kw = {}
    for arg in sys.argv[2:]:
        k, v = arg.split("=")
        kw[k] = float(v) if k == "t_end" else int(v)
    print(json.dumps({"batch": batch, "scale": scale}[cmd](**kw)), flush=True)

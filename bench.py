"""Benchmark: SSA reaction events/s on one GB300 for the 16-bit precision modes,
against the same engine's fp64 mode.

Workload (the Schloegl configuration): the bistable Schloegl model (c1 = 3e-7,
c2 = 1e-4, c3 = 1e-3, c4 = 3.5, reservoirs A = 1e5 and B = 2e5 folded into the
rate constants), X0 = 250, 10^6 trajectories per GPU, t_end = 10, 50 evenly
spaced snapshots.  One step runs the five 16-bit modes (mixed fp16 RN, mixed
bf16 RN, uniform fp16 RN, uniform fp16 SR, uniform bf16 SR) over the whole
ensemble; fp64 is timed the same way beside it.  Trajectories are
independent, so N GPUs run N disjoint trajectory-id ranges (weak scaling, no
collective on the data path).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                      [--workload schlogl|tau|rdme]
(--workload tau / rdme: the tau-leaping and RDME extensions, same contract;
see the section above run_ext.)
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_00479_gb300 import presets as P  # noqa: E402

METRIC = "SSA reaction events/s on 1 GB300, 16-bit modes vs fp64, at KS p>0.05 vs oracle"
MODES16 = [("mixed_f16", "rn"), ("mixed_bf16", "rn"), ("uniform_f16", "rn"), ("uniform_f16", "sr"),
           ("uniform_bf16", "sr")]
# reported beside the step (timed alone, not part of the timed step): selective SR
EXTRA_MODES = [("uniform_f16", "sra"), ("uniform_bf16", "sra")]
N_TRAJ = 1_000_000
T_END = 10.0
K_SAMPLES = 50
MAX_EVENTS = 200_000
SEED = 2605
SEED_FP64 = 2606     # independent fp64 ensemble for the KS / W1 comparison


def workload():
    m = P.schlogl()
    return m, P.schlogl_x0(m), P.even_samples(T_END, K_SAMPLES)


# ----------------------------------------------------------- op accounting
# Algorithmic 32-bit operations per event for the Schloegl structure with the
# reservoirs folded (chains: X(X-1) in reaction 1, X(X-1)(X-2) in reaction 2,
# X in reaction 4; reaction 3 is a constant).  Counted from the method:
#   Philox4x32-10 block: 10 rounds x (2 mul-hi + 2 mul-lo + 4 xor + 2 add) = 100
#   uniforms: half a block per step (two steps per block) + 2 x 4 to scale
#   log: 25 (exponent split 6, s = (m-1)/(m+1) 3, z and series 8, recombine 8)
#   tau division, target multiply, clock add: 3
#   mass-action factor: subtract, convert, multiply = 3 (+2 roundings in 16 bit)
#   partial sums: M - 1 adds (+ M - 1 roundings in uniform mode)
#   selection M compares + branch 2, update 2, snapshot compare 1, loop 4
SCHLOGL_FACTORS = 6  # X(X-1): 2, X(X-1)(X-2): 3, X: 1
M_REACTIONS = 4


def ops_per_event(prec, rnd):
    philox = 100
    ops = philox * 0.5 + 8 + 25 + 3
    ops += SCHLOGL_FACTORS * 3
    ops += (M_REACTIONS - 1)
    ops += M_REACTIONS + 2 + 2 + 1 + 4
    if prec.startswith(("mixed", "uniform")):
        ops += SCHLOGL_FACTORS * 2          # cvt to and from the 16-bit type
    if prec.startswith("uniform"):
        ops += (M_REACTIONS - 1 + 5) * 2    # rounded sums, E, U2, tau, target, t
    if rnd == "sr":
        n_sr = SCHLOGL_FACTORS * 2 + (M_REACTIONS - 1 + 5 if prec.startswith("uniform") else 0)
        ops += philox * ((n_sr + 7) // 8)   # stochastic-rounding blocks per step
    if rnd == "sra":
        ops += philox * ((M_REACTIONS + 7) // 8)   # sums and clock only
    return float(ops)


# ------------------------------------------------------------ ncu traffic
# DRAM bytes (read + write) per trajectory of the step's kernels, from one ncu
# capture (the uniform_f16 RN kernel profile; a 3e5-trajectory launch scaled
# per trajectory: the traffic is the snapshot stream, proportional to the
# trajectories).  Valid only for the kernel source it was measured on: the
# key includes a hash of the device code, and a changed kernel reports null.
NCU_TRAFFIC_PER_TRAJ = {
    # uniform_f16 RN, 3e5 trajectories, default launch shape (256 threads chosen for this
    # kernel, 32 step pairs per refill check, tail compaction): 269,713,408 B read +
    # 438,277,376 B written
    ("9411da1654565aeb", "uniform_f16:rn"): (269713408 + 438277376) / 300000,
}


def device_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("ssa_device.cuh", "ssa_models.h", "ssa_launch.h"):
        with open(os.path.join(ROOT, "paper_2605_00479_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(mode_key, n_traj):
    v = NCU_TRAFFIC_PER_TRAJ.get((device_source_hash(), mode_key))
    return None if v is None else v * n_traj


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                           "--format=csv,noheader,nounits", "-lms", "200"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._proc = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------- the CPU oracle
def oracle_sample(n_per_mode, modes, workers):
    """Time the oracle (as it stands) on a bounded sample of the workload."""
    import oracle
    m, x0, samples = workload()
    events = 0
    t0 = time.perf_counter()
    for prec, rnd in modes:
        r = oracle.run_parallel(m, x0, n_per_mode, T_END, samples, workers=workers, precision=prec, rounding=rnd,
                                normalise=True, seed=SEED, max_events=MAX_EVENTS)
        events += int(r["n_events"].sum())
    dt = time.perf_counter() - t0
    return events, dt


def run_reference(args, world, rank):
    """--impl reference: the oracle on the host cores, same metric and config."""
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    n_per_mode = 32 * workers
    for _ in range(args.warmup):
        oracle_sample(max(workers, 16), MODES16, workers)
    times, evs = [], []
    for _ in range(args.steps):
        e, dt = oracle_sample(n_per_mode, MODES16, workers)
        times.append(dt)
        evs.append(e)
    total_t, total_e = sum(times), sum(evs)
    value = total_e / total_t
    sample = f"{n_per_mode} trajectories per 16-bit mode per step (of {N_TRAJ}), trajectory ids 0..{n_per_mode - 1}"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16,bf16",
        "data": "synthetic", "config": config_block(),
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block():
    return {"workload": f"schlogl bistable, {N_TRAJ} trajectories per GPU, t_end={T_END}, {K_SAMPLES} snapshots, "
                        "reservoirs folded (normalise), int32 state",
            "model": "schlogl", "n_traj_per_gpu": N_TRAJ, "t_end": T_END, "n_samples": K_SAMPLES,
            "modes": [f"{p}:{r}" for p, r in MODES16], "baseline_mode": "fp64", "max_events": MAX_EVENTS,
            "l2": "no input reuse; each launch writes 600 MB of snapshots (> 129 MB L2)"}


# ------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import torch
    from scipy import stats as sst
    from paper_2605_00479_gb300 import ssa

    torch.cuda.set_device(local)
    ssa.lib()
    m_dict, x0, samples = workload()
    model = ssa.Model.from_dict(m_dict)
    offset = rank * N_TRAJ
    dev = torch.device("cuda", local)
    modes_all = MODES16 + EXTRA_MODES + [("fp64", "rn")]
    # one output set per mode, so that the modes of a step can run concurrently
    bufs = {m: (torch.empty((K_SAMPLES, model.N, N_TRAJ), dtype=torch.int32, device=dev),
                torch.empty(N_TRAJ, dtype=torch.int32, device=dev),
                torch.empty(N_TRAJ, dtype=torch.int64, device=dev),
                torch.empty(N_TRAJ, dtype=torch.float64, device=dev)) for m in modes_all}
    streams = {m: torch.cuda.Stream() for m in modes_all}
    main = torch.cuda.current_stream()

    def launch(m, seed, stream):
        out, status, nev, tfin = bufs[m]
        ssa.ensemble_run(model, N_TRAJ, x0, T_END, samples, m[0], m[1], True, seed, MAX_EVENTS, 4, out=out,
                         status=status, n_events=nev, t_final=tfin, stream=stream, traj_offset=offset)

    def record_results(modes, record):
        for m in modes:
            out, status, nev, _ = bufs[m]
            record.setdefault(m, []).append((nev.sum(), out[-1, 0].clone(), status.clone()))

    def sequential_step(modes, seed, record):
        """Modes one after the other on the main stream, each timed alone."""
        per = []
        for m in modes:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            launch(m, seed, main)
            e1.record(main)
            per.append((m, e0, e1))
        if record is not None:
            record_results(modes, record)
        return per

    def concurrent_step(modes, seed, record):
        """All modes at once on their own streams: the end-of-queue tail of one
        persistent kernel overlaps the start of the next."""
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(main)
        per = []
        for m in modes:
            s = streams[m]
            s.wait_event(start)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            launch(m, seed, s)
            e1.record(s)
            per.append((m, e0, e1))
        for m in modes:
            main.wait_stream(streams[m])
        stop.record(main)
        if record is not None:
            record_results(modes, record)
        return start, stop, per

    # warm-up (untimed): concurrent steps, then one sequential pass that gives
    # each mode's own rate, and the fp64 reference
    for _ in range(max(0, args.warmup - 1)):
        if (not args.concurrent):
            sequential_step(MODES16, SEED, None)
        else:
            concurrent_step(MODES16, SEED, None)
    rec_alone = {}
    alone = sequential_step(MODES16 + EXTRA_MODES, SEED, rec_alone)
    sequential_step([("fp64", "rn")], SEED_FP64, None)
    torch.cuda.synchronize()
    alone_ms = {m: e0.elapsed_time(e1) for m, e0, e1 in alone}

    # timed: K steps of the five 16-bit modes
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    rec = {}
    t0 = time.perf_counter()
    if (not args.concurrent):
        steps = [sequential_step(MODES16, SEED, rec) for _ in range(args.steps)]
    else:
        steps = [concurrent_step(MODES16, SEED, rec) for _ in range(args.steps)]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(world)
    clocks.stop()
    kernel_ms = {}
    if (not args.concurrent):
        step_ms = []
        for per in steps:
            for m, e0, e1 in per:
                kernel_ms.setdefault(m, []).append(e0.elapsed_time(e1))
            step_ms.append(sum(e0.elapsed_time(e1) for _, e0, e1 in per))
    else:
        step_ms = []
        for start, stop, per in steps:
            for m, e0, e1 in per:
                kernel_ms.setdefault(m, []).append(e0.elapsed_time(e1))
            step_ms.append(start.elapsed_time(stop))
    local_time = sum(step_ms) / 1e3
    events = {k: float(sum(float(v[0]) for v in vals)) for k, vals in rec.items()}
    local_events = sum(events.values())

    # fp64 beside it, same number of launches
    rec64 = {}
    steps64 = [sequential_step([("fp64", "rn")], SEED_FP64, rec64) for _ in range(args.steps)]
    torch.cuda.synchronize()
    fp64_ms = [e0.elapsed_time(e1) for per in steps64 for _, e0, e1 in per]
    fp64_events = sum(float(v[0]) for v in rec64[("fp64", "rn")])
    fp64_rate = fp64_events / (sum(fp64_ms) / 1e3)
    model_out = bufs[MODES16[0]]

    # end to end through the host-buffer entry point (pinned host memory)
    del model_out
    h_out = torch.empty((K_SAMPLES, model.N, N_TRAJ), dtype=torch.int32).pin_memory()
    h_st = torch.empty(N_TRAJ, dtype=torch.int32).pin_memory()
    h_ev = torch.empty(N_TRAJ, dtype=torch.int64).pin_memory()
    h_tf = torch.empty(N_TRAJ, dtype=torch.float64).pin_memory()
    e2e_events, e2e_time = 0.0, 0.0
    h2d = d2h = 0
    for prec, rnd in MODES16:
        t1 = time.perf_counter()
        ssa.ensemble_run_host(model, N_TRAJ, x0, T_END, samples, prec, rnd, True, SEED, MAX_EVENTS, 4,
                              out=h_out.numpy(), status=h_st.numpy().view(np.uint32), n_events=h_ev.numpy(),
                              t_final=h_tf.numpy(), traj_offset=offset)
        e2e_time += time.perf_counter() - t1
        e2e_events += float(h_ev.numpy().sum())
        h2d += x0.nbytes + samples.nbytes
        d2h += h_out.numel() * 4 + h_st.numel() * 4 + h_ev.numel() * 8 + h_tf.numel() * 8

    # whole-job numbers
    job_time = max_over_ranks(world, local_time)
    job_events = sum_over_ranks(world, local_events)
    e2e_time = max_over_ranks(world, e2e_time)
    e2e_events = sum_over_ranks(world, e2e_events)
    fp64_rate_job = sum_over_ranks(world, fp64_rate)
    if rank != 0:
        return

    # accuracy of each mode against the independent fp64 ensemble (last step)
    ref = rec64[("fp64", "rn")][-1][1].cpu().numpy()
    modes_out = {}
    for (prec, rnd), vals in rec.items():
        xs = vals[-1][1].cpu().numpy()
        st = vals[-1][2].cpu().numpy()
        D, p = sst.ks_2samp(ref, xs)
        D4, p4 = sst.ks_2samp(ref[:10000], xs[:10000])
        ev_alone = float(rec_alone[(prec, rnd)][0][0])
        rate = ev_alone / (alone_ms[(prec, rnd)] / 1e3)
        modes_out[f"{prec}:{rnd}"] = {
            "events_per_s": rate, "ms_per_launch_alone": alone_ms[(prec, rnd)],
            "ms_per_launch_in_step": float(np.mean(kernel_ms[(prec, rnd)])), "speedup_vs_fp64": rate / fp64_rate,
            "ks_p_vs_fp64": float(p), "ks_p_vs_fp64_n1e4": float(p4),
            "w1_vs_fp64": float(sst.wasserstein_distance(ref, xs)),
            "mean": float(xs.mean()), "var": float(xs.var()), "frac_max_events": float(np.mean((st & 2) != 0)),
            "ops_per_event": ops_per_event(prec, rnd)}
    for prec, rnd in EXTRA_MODES:
        out_x, st_x = bufs[(prec, rnd)][0], bufs[(prec, rnd)][1]
        xs = rec_alone[(prec, rnd)][0][1].cpu().numpy()
        ev_alone = float(rec_alone[(prec, rnd)][0][0])
        rate = ev_alone / (alone_ms[(prec, rnd)] / 1e3)
        modes_out[f"{prec}:{rnd}"] = {
            "events_per_s": rate, "ms_per_launch_alone": alone_ms[(prec, rnd)], "in_step": False,
            "speedup_vs_fp64": rate / fp64_rate, "ks_p_vs_fp64": float(sst.ks_2samp(ref, xs)[1]),
            "ks_p_vs_fp64_n1e4": float(sst.ks_2samp(ref[:10000], xs[:10000])[1]),
            "w1_vs_fp64": float(sst.wasserstein_distance(ref, xs)),
            "mean": float(xs.mean()), "var": float(xs.var()), "ops_per_event": ops_per_event(prec, rnd)}
    modes_out["fp64:rn"] = {"events_per_s": fp64_rate, "ms_per_launch": float(np.mean(fp64_ms)),
                            "mean": float(ref.mean()), "var": float(ref.var())}

    # the metric's KS criterion: which modes of the step match the fp64
    # ensemble at p > 0.05 (10^4 trajectories of each), and their own rate
    passing = [m for m in MODES16 if modes_out[f"{m[0]}:{m[1]}"]["ks_p_vs_fp64_n1e4"] > 0.05]
    pass_ms = sum(sum(kernel_ms[m]) for m in passing)
    ks_block = {"test": "two-sample KS of X at t_end vs the independent fp64 ensemble, 10^4 trajectories each",
                "passing_modes": [f"{p}:{r}" for p, r in passing],
                "events_per_s_passing": (sum(events[m] for m in passing) / (pass_ms / 1e3)) if passing else None}

    # roofline of the dominant kernel (largest share of the step)
    dom = max(kernel_ms, key=lambda k: sum(kernel_ms[k]))
    dom_ms = float(np.mean(kernel_ms[dom]))     # on its own stream, inside the timed steps
    dom_events = events[dom] / args.steps
    clk = clocks.summary()
    sm_mhz = clk["sm_mhz"] or 1455.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_gops = sms * 128 * sm_mhz * 1e6 / 1e9            # 4 schedulers x 32 lanes per SM per clock
    achieved_gops = ops_per_event(*dom) * dom_events / (dom_ms / 1e3) / 1e9
    value = job_events / job_time
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * job_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16,bf16", "data": "synthetic", "config": config_block(),
        "gpu_launches": len(MODES16) * args.steps,
        "roofline": {"bound": "alu", "kernel": f"ssa_kernel<schlogl,{dom[0]},{dom[1]}>",
                     "achieved": achieved_gops, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved_gops / peak_gops, "traffic": traffic_per_launch(f"{dom[0]}:{dom[1]}", N_TRAJ),
                     "traffic_unit": "bytes per launch", "source_hash": device_source_hash(),
                     "peak_basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock sampled in the run)",
                     "snapshot_hbm_gbs": (K_SAMPLES * model.N * N_TRAJ * 4) / (dom_ms / 1e3) / 1e9},
        "fp64_events_per_s": fp64_rate_job, "speedup_vs_fp64": value / fp64_rate_job,
        "ks_criterion": ks_block,
        "modes": modes_out,
        "e2e": {"value": e2e_events / e2e_time, "unit": "events/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk,
        "wall_s_timed": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        workers = os.cpu_count() or 1
        n_per_mode = 32 * workers
        e, dt = oracle_sample(n_per_mode, MODES16, workers)
        line["cpu_baseline"] = {"value": e / dt, "unit": "events/s", "cores": workers, "kind": "oracle",
                                "sample": f"{n_per_mode} trajectories per 16-bit mode (ids 0..{n_per_mode - 1}) "
                                          f"of the same workload, one process per core"}
    print(json.dumps(line), flush=True)


# ===================================================== tau-leaping and RDME
# The same contract for the two approximate / spatial extensions of the path:
#   --workload tau   fixed-leap tau-leaping on the Schloegl configuration above
#                    (10^6 trajectories per GPU, t_end = 10, 50 snapshots,
#                    tau = 0.005 = 2000 leaps); unit: reactions fired (the sum
#                    of the Poisson counts) per second;
#   --workload rdme  the spatial Schloegl chain: 32 voxels in a line, each the
#                    Schloegl system above, X hopping at D = 1 per molecule to
#                    each neighbour, 2^17 lattices per GPU, t_end = 2, one
#                    snapshot; unit: events (reactions + hops) per second.
# A step runs the listed modes one after the other, each timed with CUDA
# events on the launching stream; fp64 is timed beside the step on a smaller
# ensemble.  Roofline: the kernels are bound by instruction issue (state in
# registers / shared memory, HBM carries only snapshots), so `achieved` is the
# warp-instruction rate = (warp instructions per unit from one ncu count,
# keyed by the device-source hash) x (units per second measured here) and
# `peak` = SMs x 4 warp instructions per clock x the sampled SM clock.
TAU_STEP = 0.005
TAU_MODES = [("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_bf16", "rn"), ("uniform_f16", "sr"), ("uniform_bf16", "sr")]
TAU_N_TRAJ = 1_000_000
TAU_FP64_TRAJ = 200_000
RDME_S = 32
RDME_D = [1.0, 0.0, 0.0]
RDME_T_END = 2.0
RDME_MODES = [("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_bf16", "rn"), ("mixed_f16", "sr")]
RDME_N = 131_072
RDME_FP64_N = 8192
RDME_CAP = 4_000_000

# ncu counts per unit (warp instructions; DRAM bytes), keyed by (device-source
# hash, workload, mode); a changed kernel reports null until re-counted.
NCU_PER_UNIT = {
    # tau, 2e5 trajectories, one launch per mode (compiled Schloegl structure)
    ("cd94fe69908757f8", "tau", "fp32:rn"): {"warp_inst": 6.275, "dram_bytes": 0.01362},
    ("cd94fe69908757f8", "tau", "mixed_f16:rn"): {"warp_inst": 6.364, "dram_bytes": 0.01471},
    ("cd94fe69908757f8", "tau", "mixed_bf16:rn"): {"warp_inst": 6.246, "dram_bytes": 0.01422},
    ("cd94fe69908757f8", "tau", "uniform_f16:sr"): {"warp_inst": 6.540, "dram_bytes": 0.01391},
    ("cd94fe69908757f8", "tau", "uniform_bf16:sr"): {"warp_inst": 6.440, "dram_bytes": 0.01381},
    # rdme, 32768 lattices, one launch per mode
    ("5413161c178d66ef", "rdme", "fp32:rn"): {"warp_inst": 30.169, "dram_bytes": 0.00012},
    ("5413161c178d66ef", "rdme", "mixed_f16:rn"): {"warp_inst": 32.493, "dram_bytes": 0.00012},
    ("5413161c178d66ef", "rdme", "mixed_bf16:rn"): {"warp_inst": 32.519, "dram_bytes": 0.00065},
    ("5413161c178d66ef", "rdme", "mixed_f16:sr"): {"warp_inst": 43.923, "dram_bytes": 0.00110},
}


def ext_source_hash(workload):
    import hashlib
    h = hashlib.sha256()
    files = ["ssa_device.cuh", "ssa_models.h", "ssa_launch.h"]
    files += (["tau_device.cuh", "tau_launch.h", "ssa_k_tau.cu", "ssa_k_tau_schlogl.cu"] if workload == "tau" else
              ["rdme_device.cuh", "ssa_k_rdme.cu", "ssa_k_rdme_schlogl.cu"])
    for f in files:
        with open(os.path.join(ROOT, "paper_2605_00479_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ext_spec(workload, n_traj=None):
    m = P.schlogl()
    x0 = P.schlogl_x0(m)
    if workload == "tau":
        n = n_traj or TAU_N_TRAJ
        samples = P.even_samples(T_END, K_SAMPLES)
        return {"metric": "tau-leaping reactions/s on 1 GB300 (Schloegl, tau = 0.005), 16-bit and fp32 modes vs fp64",
                "unit": "reactions/s", "modes": TAU_MODES, "n": n, "n64": min(n, TAU_FP64_TRAJ), "model": m,
                "x0": x0, "samples": samples, "flush_l2": False,
                "config": {"workload": f"schlogl bistable tau-leaping, {n} trajectories per GPU, t_end={T_END}, "
                                       f"tau={TAU_STEP} ({int(round(T_END / TAU_STEP))} leaps), {K_SAMPLES} "
                                       "snapshots, reservoirs folded, int32 state",
                           "model": "schlogl", "n_traj_per_gpu": n, "tau": TAU_STEP, "t_end": T_END,
                           "n_samples": K_SAMPLES, "modes": [f"{p}:{r}" for p, r in TAU_MODES],
                           "baseline_mode": "fp64", "l2": "no input reuse; each launch writes 600 MB of snapshots "
                                                          "(> 129 MB L2)"}}
    n = n_traj or RDME_N
    lat = np.tile(x0, (RDME_S, 1)).astype(np.int32)
    return {"metric": "RDME events/s on 1 GB300 (spatial Schloegl chain, 32 voxels), 16-bit and fp32 modes vs fp64",
            "unit": "events/s", "modes": RDME_MODES, "n": n, "n64": min(n, RDME_FP64_N), "model": m, "x0": lat,
            "samples": [RDME_T_END], "flush_l2": True,
            "config": {"workload": f"RDME spatial schlogl chain, {RDME_S} voxels, D=1 for X, {n} lattices per GPU, "
                                   f"t_end={RDME_T_END}, 1 snapshot, reservoirs folded, int32 state",
                       "model": "schlogl", "lattice": [RDME_S, 1, 1], "diffusion": RDME_D, "n_traj_per_gpu": n,
                       "t_end": RDME_T_END, "n_samples": 1, "modes": [f"{p}:{r}" for p, r in RDME_MODES],
                       "baseline_mode": "fp64", "max_events": RDME_CAP,
                       "l2": "lattice state lives in shared memory; a 256 MB buffer is written between launches "
                             "(L2 flush)"}}


def ext_launch(ssa, workload, spec, model, mode, n, seed, offset, stream, bufs=None):
    prec, rnd = mode
    kw = {} if bufs is None else dict(out=bufs[0], status=bufs[1], n_events=bufs[2], t_final=bufs[3])
    if workload == "tau":
        return ssa.tau_run(model, n, spec["x0"], T_END, TAU_STEP, spec["samples"], prec, rnd, True, seed, 4,
                           stream=stream, traj_offset=offset, **kw)
    return ssa.rdme_run(model, (RDME_S,), RDME_D, spec["x0"], n, RDME_T_END, spec["samples"], prec, rnd, True, seed,
                        RDME_CAP, 4, stream=stream, traj_offset=offset, **kw)


def ext_oracle_sample(workload, spec, modes, n_per_mode, workers):
    """The oracle (as it stands) on a bounded sample: trajectory ids 0..n-1."""
    import oracle
    units = 0
    t0 = time.perf_counter()
    for prec, rnd in modes:
        if workload == "tau":
            r = oracle.events_parallel("tau_run", n_per_mode, workers=workers, model=spec["model"], x0=spec["x0"],
                                       t_end=T_END, tau=TAU_STEP, sample_times=spec["samples"], precision=prec,
                                       rounding=rnd, normalise=True, seed=SEED)
        else:
            r = oracle.events_parallel("rdme_run", n_per_mode, workers=workers, model=spec["model"],
                                       dims=(RDME_S,), diffusion=RDME_D, x0=spec["x0"], t_end=RDME_T_END,
                                       sample_times=spec["samples"], precision=prec, rounding=rnd, normalise=True,
                                       seed=SEED, max_events=RDME_CAP)
        units += int(r["n_events"].sum())
    return units, time.perf_counter() - t0


def ext_oracle_n(workload, workers):
    return (64 if workload == "tau" else 16) * workers


def run_ext_reference(args, world, rank, workload):
    if rank != 0:
        return
    spec = ext_spec(workload)
    workers = os.cpu_count() or 1
    n = ext_oracle_n(workload, workers)
    for _ in range(args.warmup):
        ext_oracle_sample(workload, spec, spec["modes"], workers, workers)
    times, units = [], []
    for _ in range(args.steps):
        u, dt = ext_oracle_sample(workload, spec, spec["modes"], n, workers)
        times.append(dt)
        units.append(u)
    value = sum(units) / sum(times)
    sample = f"{n} trajectories per mode per step (of {spec['n']}), ids 0..{n - 1}"
    print(json.dumps({
        "impl": "reference", "metric": spec["metric"], "value": value, "unit": spec["unit"], "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32,f16,bf16",
        "data": "synthetic", "config": spec["config"],
        "cpu_baseline": {"value": value, "unit": spec["unit"], "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": spec["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def run_ext(args, world, rank, local, workload):
    import torch
    from scipy import stats as sst
    from paper_2605_00479_gb300 import ssa

    torch.cuda.set_device(local)
    ssa.lib()
    spec = ext_spec(workload, args.n_traj)
    if args.modes:
        spec["modes"] = [tuple(m.split(":")) for m in args.modes.split(",")]
    model = ssa.Model.from_dict(spec["model"])
    n, n64 = spec["n"], spec["n64"]
    offset = rank * n
    main = torch.cuda.current_stream()
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device="cuda") if spec["flush_l2"] else None

    N = model.N
    shape = (len(spec["samples"]), N, n) if workload == "tau" else (len(spec["samples"]), RDME_S, N, n)

    def buffers(count):
        sh = shape[:-1] + (count,)
        return (torch.empty(sh, dtype=torch.int32, device="cuda"), torch.empty(count, dtype=torch.int32, device="cuda"),
                torch.empty(count, dtype=torch.int64, device="cuda"),
                torch.empty(count, dtype=torch.float64, device="cuda"))

    bufs = {mode: buffers(n) for mode in spec["modes"]}
    bufs[("fp64", "rn")] = buffers(n64)

    def step(modes, seed, count):
        per = []
        for mode in modes:
            if flush is not None:
                flush.fill_(1)                  # between launches, outside the timed interval
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            r = ext_launch(ssa, workload, spec, model, mode, count, seed, offset, main, bufs[mode])
            e1.record(main)
            per.append((mode, e0, e1, r))
        torch.cuda.synchronize()
        out = {}
        for mode, e0, e1, r in per:
            out[mode] = (e0.elapsed_time(e1), float(r["n_events"].double().sum()),
                         r["snapshots"][-1, 0].cpu().numpy() if workload == "tau" else
                         r["snapshots"][-1, RDME_S // 2, 0].cpu().numpy(),
                         int(((r["status"].cpu().numpy() & 0x9) != 0).sum()))
        return out

    for _ in range(args.warmup):
        step(spec["modes"], SEED, n)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = [step(spec["modes"], SEED, n) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    barrier(world)
    clocks.stop()
    local_time = sum(v[0] for st in steps for v in st.values()) / 1e3
    local_units = sum(v[1] for st in steps for v in st.values())
    job_time = max_over_ranks(world, local_time)
    job_units = sum_over_ranks(world, local_units)

    # fp64 beside the step (smaller ensemble), and its states for accuracy
    step([("fp64", "rn")], SEED + 1, n64)
    r64 = step([("fp64", "rn")], SEED + 1, n64)[("fp64", "rn")]
    fp64_rate = r64[1] / (r64[0] / 1e3)

    # end to end through the public call: inputs from the host, results read back
    h2d = d2h = 0
    e2e_units, e2e_time = 0.0, 0.0
    pinned = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory()
              for k, v in zip(("snapshots", "status", "n_events", "t_final"), bufs[spec["modes"][0]])}
    host_out = tuple(pinned[k] for k in ("snapshots", "status", "n_events", "t_final"))
    for mode in spec["modes"]:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        # inputs from the host; the kernel writes its results straight into the
        # page-locked host buffers (the ABI accepts them as output pointers)
        ext_launch(ssa, workload, spec, model, mode, n, SEED, offset, main, host_out)
        torch.cuda.synchronize()
        e2e_time += time.perf_counter() - t1
        e2e_units += float(pinned["n_events"].double().sum())
        h2d += np.asarray(spec["x0"]).size * 4 + 8 * len(spec["samples"])
        d2h += sum(v.numel() * v.element_size() for v in pinned.values())
    e2e_time = max_over_ranks(world, e2e_time)
    e2e_units = sum_over_ranks(world, e2e_units)
    if rank != 0:
        return

    ref = r64[2]
    modes_out = {"fp64:rn": {"units_per_s": fp64_rate, "ms_per_launch": r64[0], "n_traj": n64,
                             "mean": float(ref.mean()), "var": float(ref.var())}}
    for mode in spec["modes"]:
        ms = [st[mode][0] for st in steps]
        u = sum(st[mode][1] for st in steps)
        xs = steps[-1][mode][2]
        modes_out[f"{mode[0]}:{mode[1]}"] = {
            "units_per_s": u / (sum(ms) / 1e3), "ms_per_launch": float(np.mean(ms)),
            "units_per_launch": steps[-1][mode][1],
            "speedup_vs_fp64": (u / (sum(ms) / 1e3)) / fp64_rate,
            "ks_p_vs_fp64": float(sst.ks_2samp(ref, xs)[1]), "w1_vs_fp64": float(sst.wasserstein_distance(ref, xs)),
            "mean": float(xs.mean()), "var": float(xs.var()), "stopped": steps[-1][mode][3]}
    dom = max(spec["modes"], key=lambda m: sum(st[m][0] for st in steps))
    dom_ms = float(np.mean([st[dom][0] for st in steps]))
    dom_units = float(np.mean([st[dom][1] for st in steps]))
    clk = clocks.summary()
    sm_mhz = clk["sm_mhz"] or 1455.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    key = (ext_source_hash(workload), workload, f"{dom[0]}:{dom[1]}")
    counts = NCU_PER_UNIT.get(key)
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    achieved = None if counts is None else counts["warp_inst"] * dom_units / (dom_ms / 1e3) / 1e9
    value = job_units / job_time
    line = {
        "metric": spec["metric"], "value": value, "unit": spec["unit"], "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * job_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32,f16,bf16", "data": "synthetic",
        "config": spec["config"], "gpu_launches": len(spec["modes"]) * args.steps,
        "roofline": {"bound": "issue", "kernel": f"{workload}_kernel<schlogl,{dom[0]},{dom[1]}>",
                     "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s",
                     "frac": None if achieved is None else achieved / peak,
                     "traffic": None if counts is None else counts["dram_bytes"] * dom_units,
                     "traffic_unit": "bytes per launch", "source_hash": key[0],
                     "peak_basis": f"{sms} SMs x 4 warp instructions per clock x {sm_mhz:.0f} MHz (median SM clock "
                                   "sampled in the run)",
                     "count_basis": "ncu smsp__inst_executed.sum per unit of the same kernel and source, times the "
                                    "units per second measured here"},
        "fp64_units_per_s": fp64_rate, "speedup_vs_fp64": value / fp64_rate, "modes": modes_out,
        "e2e": {"value": e2e_units / e2e_time, "unit": spec["unit"], "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk, "wall_s_timed": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        workers = os.cpu_count() or 1
        nn = ext_oracle_n(workload, workers)
        u, dt = ext_oracle_sample(workload, spec, spec["modes"], nn, workers)
        line["cpu_baseline"] = {"value": u / dt, "unit": spec["unit"], "cores": workers, "kind": "oracle",
                                "sample": f"{nn} trajectories per mode (ids 0..{nn - 1}) of the same workload, "
                                          "one process per core"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--concurrent", action="store_true",
                    help="run the modes of a step on concurrent streams (overlaps the kernels' end-of-queue tails)")
    ap.add_argument("--n-traj", type=int, default=None,
                    help="trajectories per GPU (default 10^6; smaller values are for profiling only)")
    ap.add_argument("--modes", default=None, help="comma list like mixed_f16:rn (profiling only)")
    ap.add_argument("--workload", choices=["schlogl", "tau", "rdme"], default="schlogl",
                    help="schlogl: the direct-method benchmark (default); tau: tau-leaping; rdme: spatial RDME")
    args = ap.parse_args()
    global N_TRAJ, MODES16
    if args.n_traj:
        N_TRAJ = args.n_traj
    if args.modes:
        MODES16 = [tuple(m.split(":")) for m in args.modes.split(",")]
    world, rank, local = dist_setup(args)
    if args.workload != "schlogl":
        if args.impl == "reference":
            run_ext_reference(args, world, rank, args.workload)
        else:
            run_ext(args, world, rank, local, args.workload)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
